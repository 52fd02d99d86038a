// tc_contract_noalloc: the FP64 contraction without any device allocation.
//
// Some callers cannot call cudaMalloc at all: code running while a CUDA graph
// is being captured elsewhere on the device, real-time or embedded hosts whose
// device memory is carved up once at start-up, and plug-in or interop layers
// whose host application owns every allocation.  For them this entry point
// keeps the only scratch the FP64 path needs -- the scatter and block-scatter
// vectors -- in one fixed array compiled into the library.  The caller still
// supplies A, B and C; nothing else is allocated, by the library or by any
// routine it calls.
#include <mutex>

#include "host_common.h"
#include "kernels.h"

namespace tc {
int aliases(const tc_tensor* A, const tc_tensor* B, const tc_tensor* C, size_t es);
}

namespace {

using namespace tc;

constexpr size_t kScratchBytes = TC_NOALLOC_SCRATCH_BYTES;
constexpr int64_t kScratchEntries = (int64_t)(kScratchBytes / sizeof(int64_t));

// The fixed scratch: every GPU that loads libtc holds these bytes until the
// process exits.  All calls on a device share it.
static __device__ __align__(256) int64_t g_noalloc_scratch[kScratchEntries];

std::mutex g_scratch_mu;
int64_t* g_scratch_ptr[64] = {};

// Device address of the scratch array on the current device.  The first call
// on each device looks it up (cudaGetSymbolAddress, with that device current);
// later calls reuse the cached address.  In host code the array's name is only
// a host-side stand-in, never a device address, so kernels get this pointer.
int scratch_on_current_device(int64_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TC_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return TC_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<int64_t*>(p);
  }
  *out = g_scratch_ptr[dev];
  return TC_OK;
}

}  // namespace

extern "C" int tc_contract_noalloc(tc_dtype dtype, double alpha, const tc_tensor* A,
                                   const tc_tensor* B, double beta, const tc_tensor* C,
                                   void* stream) {
  NvtxRange range("tc_contract_noalloc");
  if (dtype != TC_F64 && dtype != TC_F32) return TC_ERR_ARG;
  Planned p;
  int rc = plan_problem(A, B, C, &p);
  if (rc != TC_OK) return rc;
  if (tc::aliases(A, B, C, dtype == TC_F64 ? 8 : 4)) return TC_ERR_OVERLAP;
  const Layout& L = p.L;
  if (L.m == 0 || L.n == 0) return TC_OK;
  const ScatterOffsets o = scatter_offsets(L, kBsBlock);
  if (o.total > kScratchEntries) return TC_ERR_SCRATCH_LIMIT;
  int64_t* scat = nullptr;
  if ((rc = scratch_on_current_device(&scat)) != TC_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Every entry the kernels read below is written by the scatter builder
  // first, in stream order, so nothing in the array has to start at zero.
  if (launch_build_scatter(L, kBsBlock, scat, s) != cudaSuccess) return TC_ERR_CUDA;
  // the library's device error word (a static array too: no allocation)
  int32_t* ew = err_word();
  if (!ew) return TC_ERR_CUDA;
  const int32_t* gate = nullptr;
  if (checks_on()) {
    if (launch_check_scatter(L, kBsBlock, scat, check_bounds(L), ew, s) != cudaSuccess)
      return TC_ERR_CUDA;
    gate = ew;
  }
  const ScatterPtrs sp = scatter_ptrs(scat, o);
  if (L.k == 0 || alpha == 0.0)
    return launch_scale_c(dtype, p.c, sp, L.m, L.n, beta, s, gate) == cudaSuccess ? TC_OK
                                                                                  : TC_ERR_CUDA;
  F64Launch f;
  f.dtype = dtype;
  f.a = p.a;
  f.b = p.b;
  f.c = p.c;
  f.sp = sp;
  f.m = L.m;
  f.n = L.n;
  f.k = L.k;
  f.alpha = alpha;
  f.beta = beta;
  f.a_k_contig = p.info.a_k_contig;
  f.b_k_contig = p.info.b_k_contig;
  f.partial = nullptr;  // plain tiling only: no stream-K partials in the fixed array
  f.max_ctas = 0;
  f.err = ew;
  f.gate = gate;
  return launch_f64(f, s) == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}
