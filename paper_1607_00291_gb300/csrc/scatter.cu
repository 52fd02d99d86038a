// K1: device construction of the scatter and block-scatter vectors.
//
// Section 6.1: for a bundle with dims (n_0, s_0), (n_1, s_1), ... the scatter
// vector maps the linearised index x (dim 0 fastest) to the tensor offset
// scat[x] = sum_d u_d(x) s_d.  A matrix view C_{IJ} of a tensor then has
// loc(C_{IJ}) = rscat_I(C) + cscat_J(C); A uses rscat over I and cscat over P,
// B rscat over P and cscat over J.
// Section 6.2: the block-scatter vector with blocking parameter b holds, per
// block of b consecutive entries, the common difference s > 0 of the entries
// when there is one and 0 otherwise (one-element blocks get 1).
//
// GPU form: one thread per output entry; each block-scatter entry recomputes
// the scatter values of its own block, so the kernel needs no second pass.
#include <cstdlib>

#include "kernels.h"

namespace tc {
namespace {

// Entry x of a bundle's scatter vector over its s0 (first) or s1 strides;
// kHole where the digits of x fall past an original extent of a blocked
// bundle.
__device__ __forceinline__ int64_t scat_at(const Bundle& B, bool first, int64_t x) {
  const int64_t* s = first ? B.s0 : B.s1;
  int64_t v = 0, lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
  for (int d = 0; d < B.nd; ++d) {
    const int64_t q = x / B.len[d];
    const int64_t u = x - q * B.len[d];
    v += u * s[d];
    if (B.nblk > 0) {
      if (d == B.blk_lo[0]) lo0 = u;
      if (d == B.blk_hi[0]) hi0 = u;
      if (d == B.blk_lo[1]) lo1 = u;
      if (d == B.blk_hi[1]) hi1 = u;
    }
    x = q;
  }
  if (B.nblk > 0 && lo0 + B.blk_b[0] * hi0 >= B.blk_lim[0]) return kHole;
  if (B.nblk > 1 && lo1 + B.blk_b[1] * hi1 >= B.blk_lim[1]) return kHole;
  return v;
}

struct Section {
  const Bundle* B;
  bool first;
  int64_t l;
};

__device__ __forceinline__ Section section(const Layout& L, int which) {
  // 0 rA: I/A   1 cA: P/A   2 rB: P/B   3 cB: J/B   4 rC: I/C   5 cC: J/C
  switch (which) {
    case 0: return {&L.I, true, L.m};
    case 1: return {&L.P, true, L.k};
    case 2: return {&L.P, false, L.k};
    case 3: return {&L.J, true, L.n};
    case 4: return {&L.I, false, L.m};
    default: return {&L.J, false, L.n};
  }
}

// Entry t of the concatenated vectors of one problem (layout of tc.h).
__device__ __forceinline__ int64_t scatter_entry(const Layout& L, const ScatterOffsets& o,
                                                 int32_t b, int64_t t) {
  const int64_t starts[12] = {o.rA, o.cA, o.rB, o.cB, o.rC, o.cC,
                              o.rbsA, o.cbsA, o.rbsB, o.cbsB, o.rbsC, o.cbsC};
  int sec = 0;
  while (sec < 11 && t >= starts[sec + 1]) ++sec;
  const int64_t x = t - starts[sec];
  if (sec < 6) {
    Section S = section(L, sec);
    return scat_at(*S.B, S.first, x);
  }
  Section S = section(L, sec - 6);
  const int64_t lo = x * b;
  const int64_t hi = lo + b < S.l ? lo + b : S.l;
  int64_t prev = scat_at(*S.B, S.first, lo);
  if (prev == kHole) return 0;  // a block with a hole makes no claim
  if (hi - lo <= 1) return 1;
  int64_t cur = scat_at(*S.B, S.first, lo + 1);
  if (cur == kHole) return 0;
  const int64_t st = cur - prev;
  bool ok = st > 0;
  for (int64_t j = lo + 2; j < hi && ok; ++j) {
    prev = cur;
    cur = scat_at(*S.B, S.first, j);
    ok = cur != kHole && (cur - prev) == st;
  }
  return ok ? st : 0;
}

__global__ void k_build_scatter(const Layout L, const int32_t b, const ScatterOffsets o,
                                int64_t* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < o.total;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = scatter_entry(L, o, b, t);
}

// All problems of a batch: entry t belongs to the problem p with
// offsets[p] <= t < offsets[p + 1] (binary search).
__global__ void k_build_scatter_batched(const Layout* __restrict__ layouts,
                                        const int64_t* __restrict__ offsets, int32_t count,
                                        int64_t total, int32_t b, int64_t* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = count;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (offsets[mid] <= t) lo = mid; else hi = mid;
    }
    const Layout& L = layouts[lo];
    out[t] = scatter_entry(L, scatter_offsets(L, b), b, t - offsets[lo]);
  }
}

// ---- checks: entry t of one problem's vectors against its vector's range,
// block-scatter entries against the differences of their block -------------
__device__ __forceinline__ bool entry_ok(const Layout& L, const ScatterOffsets& o, int32_t b,
                                         const CheckBounds& cb, const int64_t* v, int64_t t) {
  const int64_t starts[13] = {o.rA,   o.cA,   o.rB,   o.cB,   o.rC,   o.cC,   o.rbsA,
                              o.cbsA, o.rbsB, o.cbsB, o.rbsC, o.cbsC, o.total};
  int sec = 0;
  while (sec < 11 && t >= starts[sec + 1]) ++sec;
  // a hole of a blocked row bundle (rA, rC) names no element
  if (sec < 6) return (v[t] >= cb.lo[sec] && v[t] <= cb.hi[sec]) ||
                      (v[t] == kHole && (sec == 0 || sec == 4) && L.I.nblk > 0);
  const int vs = sec - 6;  // the scatter vector this block-scatter vector describes
  const int64_t len = starts[vs + 1] - starts[vs];
  const int64_t lo = (t - starts[sec]) * b, hi = lo + b < len ? lo + b : len;
  const int64_t st = v[t];
  if (st < 0) return false;
  if (st == 0) return true;  // no claim: the kernels gather this block element by element
  const int64_t* sv = v + starts[vs];
  for (int64_t j = lo + 1; j < hi; ++j)
    if (sv[j] - sv[j - 1] != st) return false;
  return true;
}

__global__ void k_check_scatter(const Layout L, const int32_t b, const ScatterOffsets o,
                                const CheckBounds cb, const int64_t* __restrict__ v,
                                int32_t* __restrict__ err) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < o.total;
       t += (int64_t)gridDim.x * blockDim.x)
    if (!entry_ok(L, o, b, cb, v, t)) atomicMax(err, kDevBounds);
}

__global__ void k_check_scatter_batched(const Layout* __restrict__ layouts,
                                        const int64_t* __restrict__ offsets,
                                        const CheckBounds* __restrict__ cbs, int32_t count,
                                        int64_t total, int32_t b, const int64_t* __restrict__ v,
                                        int32_t* __restrict__ err) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = count;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (offsets[mid] <= t) lo = mid; else hi = mid;
    }
    const Layout& L = layouts[lo];
    if (!entry_ok(L, scatter_offsets(L, b), b, cbs[lo], v + offsets[lo], t - offsets[lo]))
      atomicMax(err, kDevBounds);
  }
}

template <typename T>
__global__ void k_scale_c(T* __restrict__ c, const int64_t* __restrict__ rC,
                          const int64_t* __restrict__ cC, int64_t m, int64_t n, double beta,
                          const int32_t* __restrict__ gate) {
  if (gate && *gate == kDevBounds) return;
  const int64_t total = m * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % m, j = t / m;
    const int64_t r = rC[i];
    if (r == kHole) continue;  // a hole of a blocked row bundle
    T* p = c + r + cC[j];
    *p = beta == 0.0 ? T(0) : T(beta * (double)*p);
  }
}

}  // namespace

ScatterPtrs scatter_ptrs(const int64_t* base, const ScatterOffsets& o) {
  ScatterPtrs p;
  p.rA = base + o.rA;
  p.cA = base + o.cA;
  p.rB = base + o.rB;
  p.cB = base + o.cB;
  p.rC = base + o.rC;
  p.cC = base + o.cC;
  p.rbsA = base + o.rbsA;
  p.cbsA = base + o.cbsA;
  p.rbsB = base + o.rbsB;
  p.cbsB = base + o.cbsB;
  p.rbsC = base + o.rbsC;
  p.cbsC = base + o.cbsC;
  return p;
}

cudaError_t launch_build_scatter(const Layout& L, int32_t b, int64_t* out, cudaStream_t s) {
  const ScatterOffsets o = scatter_offsets(L, b);
  if (o.total == 0) return cudaSuccess;
  int64_t blocks = (o.total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_build_scatter<<<(int)blocks, 256, 0, s>>>(L, b, o, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_build_scatter_batched(const Layout* layouts, const int64_t* offsets,
                                         int32_t count, int64_t total, int32_t b, int64_t* out,
                                         cudaStream_t s) {
  if (total == 0 || count == 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  k_build_scatter_batched<<<(int)blocks, 256, 0, s>>>(layouts, offsets, count, total, b, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_scale_c(tc_dtype dt, void* c, const ScatterPtrs& sp, int64_t m, int64_t n,
                           double beta, cudaStream_t s, const int32_t* gate) {
  if (beta == 1.0 || m == 0 || n == 0) return cudaSuccess;
  int64_t blocks = (m * n + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (dt == TC_F64)
    k_scale_c<double><<<(int)blocks, 256, 0, s>>>((double*)c, sp.rC, sp.cC, m, n, beta, gate);
  else
    k_scale_c<float><<<(int)blocks, 256, 0, s>>>((float*)c, sp.rC, sp.cC, m, n, beta, gate);
  note_launch();
  return cudaGetLastError();
}

// Least and largest entry of each scatter vector: over the bundle's dims,
// sum of (len - 1) * stride where negative, resp. positive -- the range of
// offsets the dims can reach in the operand (the vectors of one operand add
// up to the operand's whole span; folded dims reach what their parts reach).
CheckBounds check_bounds(const Layout& L) {
  CheckBounds cb;
  const Bundle* bs[6] = {&L.I, &L.P, &L.P, &L.J, &L.I, &L.J};
  const bool first[6] = {true, true, false, true, false, false};  // s0 or s1
  for (int v = 0; v < 6; ++v) {
    int64_t lo = 0, hi = 0;
    for (int d = 0; d < bs[v]->nd; ++d) {
      const int64_t reach = (bs[v]->len[d] - 1) * (first[v] ? bs[v]->s0[d] : bs[v]->s1[d]);
      if (reach < 0) lo += reach; else hi += reach;
    }
    cb.lo[v] = lo;
    cb.hi[v] = hi;
  }
  // TC_CHECK_SHRINK=v (0..5): test hook that hands the checker a range one
  // element short at the top for vector v (the operands stay whole), so that
  // the check fires without any access outside an operand
  if (const char* e = std::getenv("TC_CHECK_SHRINK")) {
    const int v = std::atoi(e);
    if (e[0] >= '0' && e[0] <= '5' && e[1] == 0) cb.hi[v] -= 1;
  }
  return cb;
}

cudaError_t launch_check_scatter(const Layout& L, int32_t b, const int64_t* scat,
                                 const CheckBounds& cb, int32_t* err, cudaStream_t s) {
  const ScatterOffsets o = scatter_offsets(L, b);
  if (o.total == 0) return cudaSuccess;
  if (!err) return cudaErrorInvalidValue;
  int64_t blocks = (o.total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_check_scatter<<<(int)blocks, 256, 0, s>>>(L, b, o, cb, scat, err);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_check_scatter_batched(const Layout* layouts, const int64_t* offsets,
                                         const CheckBounds* cbs, int32_t count, int64_t total,
                                         int32_t b, const int64_t* scat, int32_t* err,
                                         cudaStream_t s) {
  if (total == 0 || count == 0) return cudaSuccess;
  if (!err) return cudaErrorInvalidValue;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  k_check_scatter_batched<<<(int)blocks, 256, 0, s>>>(layouts, offsets, cbs, count, total, b,
                                                      scat, err);
  note_launch();
  return cudaGetLastError();
}

}  // namespace tc
