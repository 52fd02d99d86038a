// Host helpers shared by the single-contraction (api.cu) and batch (batch.cu)
// entry points.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>  // header-only: the ranges cost nothing without a profiler

#include "tc_internal.h"

namespace tc {

// A named NVTX range around an entry point's host work and launches (visible
// in timeline profilers; inert otherwise).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// TC_LOG=1: one line per contraction or plan on stderr describing its plan.
bool log_enabled();

// Device error word of the current device (looked up once per device).
int32_t* err_word();
size_t elem_size(tc_dtype dt);
// Valid dtype/mode combination?  TC_OK or an error code.
int check_modes(tc_dtype dt, tc_mode mode);
// SMs of the current device (152 when no device can be queried).
int sm_count();
// plan_problem + the C-aliases-A/B check.
int plan_checked(tc_dtype dt, const tc_tensor* A, const tc_tensor* B, const tc_tensor* C,
                 Planned* p);

// Tile width and k-split of the tensor-core mainloop.
struct TcChoice {
  int bn, splits;
  int64_t kps;
};
TcChoice choose_tc(const Layout& L, int pieces, int sms, int bn_force = 0, int split_mult = 1);

}  // namespace tc
