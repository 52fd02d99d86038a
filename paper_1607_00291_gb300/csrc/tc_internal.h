// Internal types shared by the planner and the kernels of libtc.
#pragma once

#include <cstddef>
#include <cstdint>

#include "tc.h"

namespace tc {

constexpr int kMaxRank = TC_MAX_RANK;

// One index bundle after normalisation: lengths and the strides of the bundle
// dims in the two tensors that hold it (I: A, C; J: B, C; P: A, B).  The
// bundle's linearised index runs colexicographically over the dims (dim 0
// fastest), which is the matrix index of Section 6.1.
struct Bundle {
  int32_t nd;
  int64_t len[kMaxRank];
  int64_t s0[kMaxRank];
  int64_t s1[kMaxRank];
  // Blocked row bundle (the packed form's two-dimensional row tiles, built by
  // block_row_bundle): for each of the nblk pairs p, dims blk_lo[p] and
  // blk_hi[p] split one original dim of extent blk_lim[p] into blk_b[p] and
  // ceil(blk_lim[p] / blk_b[p]); a linear index whose digits give
  // u_lo + blk_b[p] u_hi >= blk_lim[p] is a hole, whose scatter entry is kHole.
  int32_t nblk;
  int32_t blk_lo[2], blk_hi[2];
  int64_t blk_b[2], blk_lim[2];
};

// The scatter entry of a hole of a blocked bundle: no element; every kernel
// that reads a blocked bundle's entries skips it.
constexpr int64_t kHole = INT64_MIN / 4;

// The matrix view of one contraction: C_{IJ} (m x n) = A_{IP} (m x k) B_{PJ} (k x n).
struct Layout {
  int64_t m, n, k;
  Bundle I;  // s0 = stride in A, s1 = stride in C
  Bundle J;  // s0 = stride in B, s1 = stride in C
  Bundle P;  // s0 = stride in A, s1 = stride in B
};

// A planned contraction (host side).  a/b are the operands in their matrix
// roles, i.e. already exchanged when info.swapped.
struct Planned {
  Layout L;
  tc_plan_info info;
  const void* a;
  const void* b;
  void* c;
};

// Validation + Section 7.3 normalisation.  Returns TC_OK or an error code.
int plan_problem(const tc_tensor* A, const tc_tensor* B, const tc_tensor* C, Planned* out);

// The packed form's blocked row order: when A is read along its rows and its
// unit-stride dim is the second row dim, behind C's (GPU step 7's interleave),
// out = L with those two dims split into 16 x ceil(E0 / 16) and 8 x ceil(E1 / 8)
// and ordered (lo0, lo1, hi0, hi1, rest): every 128-row tile is one 16 x 8
// block, over which C's unit-stride runs are 16 long and A's 8 long.  Rows
// past an original extent are holes (kHole entries).  Returns false (out
// untouched) when the layout does not qualify.
bool block_row_bundle(const Layout& L, bool a_k_contig, Layout* out);

// Exchange the matrix roles of A and B (C^T = B^T A^T: I and J swap, P's two
// stride sets swap, and the operands and their access flags with them), as
// Section 7.3's step 4 does.  Used by packed batch plans for problems whose
// rows pad far more than their columns would.
void swap_roles(Planned* p);

// Scatter-vector section offsets inside a workspace (int64 entries).
struct ScatterOffsets {
  int64_t rA, cA, rB, cB, rC, cC;        // scatter vectors
  int64_t rbsA, cbsA, rbsB, cbsB, rbsC, cbsC;  // block-scatter vectors
  int64_t total;                           // entries
};
#if defined(__CUDACC__)
#define TC_HD __host__ __device__
#else
#define TC_HD
#endif

TC_HD inline ScatterOffsets scatter_offsets(const Layout& L, int32_t b) {
  ScatterOffsets o;
  const int64_t m = L.m, n = L.n, k = L.k;
  const int64_t nm = (m + b - 1) / b, nn = (n + b - 1) / b, nk = (k + b - 1) / b;
  int64_t p = 0;
  o.rA = p; p += m;
  o.cA = p; p += k;
  o.rB = p; p += k;
  o.cB = p; p += n;
  o.rC = p; p += m;
  o.cC = p; p += n;
  o.rbsA = p; p += nm;
  o.cbsA = p; p += nk;
  o.rbsB = p; p += nk;
  o.cbsB = p; p += nn;
  o.rbsC = p; p += nm;
  o.cbsC = p; p += nn;
  o.total = p;
  return o;
}

// Block size of the block-scatter vectors the mainloops consult.
constexpr int32_t kBsBlock = 4;

// Device error word codes (shared by all kernels).
constexpr int32_t kDevOk = 0;
constexpr int32_t kDevTimeout = 1;
constexpr int32_t kDevBounds = 2;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace tc
