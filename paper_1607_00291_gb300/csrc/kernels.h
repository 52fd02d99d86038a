// Launch wrappers of the device kernels (one translation unit each).
#pragma once

#include <cuda_runtime.h>

#include "tc_internal.h"

namespace tc {

// Bookkeeping shared by every launch wrapper (defined in api.cu).
void note_launch(int n = 1);
// Events the caller asked to have recorded around the next mainloop launch.
void mainloop_event_before(cudaStream_t s);
void mainloop_event_after(cudaStream_t s);

// K1 (scatter.cu): scatter + block-scatter vectors of Section 6.1/6.2 into `out`.
cudaError_t launch_build_scatter(const Layout& L, int32_t b, int64_t* out, cudaStream_t s);

// Pointers to the six scatter vectors and six block-scatter vectors in a workspace.
struct ScatterPtrs {
  const int64_t *rA, *cA, *rB, *cB, *rC, *cC;
  const int64_t *rbsA, *cbsA, *rbsB, *cbsB, *rbsC, *cbsC;
};
ScatterPtrs scatter_ptrs(const int64_t* base, const ScatterOffsets& o);

// C := beta * C over the m x n matrix view (alpha == 0 or an empty P range).
cudaError_t launch_scale_c(tc_dtype dt, void* c, const ScatterPtrs& sp, int64_t m, int64_t n,
                           double beta, cudaStream_t s);

// K2 + K5 (f64.cu): FP64 mainloop with the fused scattered alpha/beta epilogue.
struct F64Launch {
  tc_dtype dtype;
  const void* a;
  const void* b;
  void* c;
  ScatterPtrs sp;
  int64_t m, n, k;
  double alpha, beta;
  int a_k_contig, b_k_contig;
  double* partial;   // stream-K partial tiles (f64_partial_bytes(max_ctas)), or null
  int64_t max_ctas;  // CTAs for stream-K (one per SM); ignored without `partial`
  int32_t* err;
};
cudaError_t launch_f64(const F64Launch& p, cudaStream_t s);
int64_t f64_grid(int64_t m, int64_t n, int64_t k, int64_t max_ctas, bool can_split);
size_t f64_partial_bytes(int64_t max_ctas);

// K3 + K5 (+ K4 when splits > 1) (bf16x3.cu): tcgen05 BF16x3 mainloop.
struct Bf16Launch {
  const void* a;
  const void* b;
  void* c;
  float* partial;  // splits * m * n FP32, used when splits > 1
  ScatterPtrs sp;
  int64_t m, n, k;
  double alpha, beta;
  int a_k_contig, b_k_contig;
  int bn;          // 128 or 256
  int pieces;      // bf16 pieces per operand: 2 (BF16x3) or 3 (BF16x6)
  int splits;      // CTAs along the contracted range
  int64_t k_per_split;  // multiple of 32
  int32_t* err;
};
cudaError_t launch_bf16x3(const Bf16Launch& q, cudaStream_t s);

}  // namespace tc
