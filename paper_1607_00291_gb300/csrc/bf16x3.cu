// K3 + K5: BF16x3 mainloop on the fifth-generation tensor cores (tcgen05).
//
// FP32 operands are gathered in place through the scatter vectors of
// Section 6.1 (coalesced along each operand's own unit-stride index, 16-byte
// vector loads wherever the block-scatter vectors of Section 6.2 report a unit
// stride), split on the fly into x = hi + lo with hi = RN_bf16(x) and
// lo = RN_bf16(x - hi), and written into shared memory in the tensor core's
// K-major canonical layout.  One elected thread issues, per 16-wide k-slice,
// three tcgen05.mma (hi*hi, hi*lo, lo*hi) into an FP32 accumulator in Tensor
// Memory; the lo*lo term (relative size 2^-16) is dropped.  The epilogue reads
// the accumulator with tcgen05.ld and either applies alpha/beta through
// rscat(C) + cscat(C) or, when the contracted range is split across CTAs,
// stores FP32 partials that K4 reduces in FP64.
//
// Roles (288 threads): warps 0-7 load (one k-tile ahead, in registers),
// convert and stage (producers), and later run the epilogue; warp 8 owns the Tensor Memory allocation and its lane 0 issues the
// MMAs.  Stages are handed over through mbarriers: `full` (producers -> MMA)
// and `empty` (tcgen05.commit -> producers).  Every wait is bounded; on expiry
// the CTA records TC_ERR_DEVICE_TIMEOUT in the device error word and unwinds.
#include <cuda_bf16.h>

#include "kernels.h"
#include "sm100_ptx.cuh"

namespace tc {
namespace {

using namespace ptx;

constexpr int BM = 128, BK = 32;
constexpr int NPROD = 256;
constexpr int NT = NPROD + 32;
constexpr int MMA_WARP = NPROD / 32;

// Shared-memory plan for NS bf16 pieces per operand.  Per stage:
// [A piece 0 .. NS-1][B piece 0 .. NS-1], each piece an R x BK K-major panel.
template <int BN, int NS>
struct Lay {
  static constexpr int STAGES = NS == 2 ? 4 : 3;
  static constexpr int A_BYTES = BM * BK * 2;  // one bf16 piece of the A panel
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int B_OFF = NS * A_BYTES;
  static constexpr int STAGE = NS * A_BYTES + NS * B_BYTES;
  static constexpr int OPS = STAGES * STAGE;
  static constexpr int SCAT = OPS;  // int64: rA[BM] rC[BM] cB[BN] cC[BN]
  static constexpr int BARS = SCAT + (2 * BM + 2 * BN) * 8;
  static constexpr int MISC = BARS + (2 * STAGES + 1) * 8;  // tmem slot + abort flag
  static constexpr int END = MISC + 16;
  static constexpr int ALLOC = END + 1024;  // + alignment of the base to 1 KB
  static_assert(ALLOC <= 227 * 1024, "shared memory plan exceeds the per-CTA limit");
};

// Split 8 FP32 values into NS bf16 pieces: piece 0 = RN_bf16(x), piece i =
// RN_bf16(x - pieces 0..i-1) (each residual is exact in FP32), stored to the
// NS panels at byte offset `off` (one 16-byte core-matrix row each).
template <int NS>
__device__ __forceinline__ void split8_store(float (&v)[8], uint8_t* piece0, int piece_bytes,
                                             uint32_t off) {
#pragma unroll
  for (int sidx = 0; sidx < NS; ++sidx) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
      if (sidx + 1 < NS) {
        const float2 f = __bfloat1622float2(b);
        v[2 * j] -= f.x;
        v[2 * j + 1] -= f.y;
      }
      w[j] = *reinterpret_cast<uint32_t*>(&b);
    }
    *reinterpret_cast<uint4*>(piece0 + sidx * piece_bytes + off) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// byte offset of (row r, k-chunk q of 8 elements) in an R-row K-major panel
template <int R>
__device__ __forceinline__ uint32_t panel_off(int r, int q) {
  return (uint32_t)((q * (R / 8) + (r >> 3)) * 128 + (r & 7) * 16);
}

struct Args {
  const float* a;
  const float* b;
  float* c;
  float* partial;
  ScatterPtrs sp;
  int64_t m, n, k;
  double alpha, beta;
  int a_kc, b_kc;
  int64_t tiles_n;
  int64_t k_per_split;
  int splits;
  int32_t* err;
};

// Register-staged gather of one R x BK FP32 panel.  Each producer thread owns
// a fixed set of chunks, so a panel can be loaded into registers one k-tile
// ahead of its conversion:
//  * k-contiguous operand: chunks of (1 row, 8 consecutive k), two 16-byte
//    loads where the block-scatter entry says the 4-run has unit stride and
//    the address is 16-byte aligned, scalar loads through the scatter vectors
//    otherwise;
//  * row-contiguous operand: chunks of (2 consecutive rows, 8 k), one 8-byte
//    load per k where the two rows are adjacent, scalar loads otherwise.
// Consecutive threads take consecutive chunks along the unit-stride index, so
// a warp's loads are coalesced.
template <int R>
struct PanelRegs {
  static constexpr int E = R * BK / NPROD;  // floats per thread (16 or 32)
  float v[E];
};

template <int R>
__device__ __forceinline__ void panel_load(PanelRegs<R>& pr, int tid,
                                           const float* __restrict__ base, const int64_t* rowsc,
                                           int rows_valid, const int64_t* __restrict__ ksc,
                                           const int64_t* __restrict__ kbs, int64_t k0,
                                           int64_t kend, bool kcontig) {
  constexpr int E = PanelRegs<R>::E;
  if (kcontig) {
#pragma unroll
    for (int i = 0; i < E / 8; ++i) {
      const int c = tid + i * NPROD;
      const int r = c >> 2, q = c & 3;
      const int64_t kk = k0 + q * 8;
      float* v = pr.v + 8 * i;
      if (r < rows_valid) {
        const float* rowp = base + rowsc[r];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int64_t kq = kk + 4 * h;
          const float* p = kq < kend ? rowp + ksc[kq] : rowp;
          if (kq + 3 < kend && kbs[kq >> 2] == 1 &&
              ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
            const float4 f = __ldg(reinterpret_cast<const float4*>(p));
            v[4 * h] = f.x;
            v[4 * h + 1] = f.y;
            v[4 * h + 2] = f.z;
            v[4 * h + 3] = f.w;
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
              v[4 * h + j] = (kq + j < kend) ? __ldg(rowp + ksc[kq + j]) : 0.f;
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = 0.f;
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < E / 16; ++i) {
      const int c = tid + i * NPROD;
      const int g = c % (R / 2), q = c / (R / 2);
      const int r0 = 2 * g;
      const int64_t kk = k0 + q * 8;
      float* v = pr.v + 16 * i;
      const bool r0v = r0 < rows_valid, r1v = r0 + 1 < rows_valid;
      const int64_t o0 = rowsc[r0], o1 = rowsc[r0 + 1];
      const bool pair = r1v && o1 == o0 + 1;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int64_t k = kk + j;
        if (k < kend) {
          const int64_t ko = ksc[k];
          const float* p = base + o0 + ko;
          if (pair && ((reinterpret_cast<uintptr_t>(p) & 7) == 0)) {
            const float2 f = __ldg(reinterpret_cast<const float2*>(p));
            v[j] = f.x;
            v[8 + j] = f.y;
          } else {
            v[j] = r0v ? __ldg(p) : 0.f;
            v[8 + j] = r1v ? __ldg(base + o1 + ko) : 0.f;
          }
        } else {
          v[j] = 0.f;
          v[8 + j] = 0.f;
        }
      }
    }
  }
}

template <int R, int NS>
__device__ __forceinline__ void panel_store(const PanelRegs<R>& pr, int tid, bool kcontig,
                                            uint8_t* piece0) {
  constexpr int E = PanelRegs<R>::E;
  constexpr int PB = R * BK * 2;
  if (kcontig) {
#pragma unroll
    for (int i = 0; i < E / 8; ++i) {
      const int c = tid + i * NPROD;
      float w[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) w[j] = pr.v[8 * i + j];
      split8_store<NS>(w, piece0, PB, panel_off<R>(c >> 2, c & 3));
    }
  } else {
#pragma unroll
    for (int i = 0; i < E / 16; ++i) {
      const int c = tid + i * NPROD;
      const int g = c % (R / 2), q = c / (R / 2);
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        float w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) w[j] = pr.v[16 * i + 8 * rr + j];
        split8_store<NS>(w, piece0, PB, panel_off<R>(2 * g + rr, q));
      }
    }
  }
}

__device__ __forceinline__ void record_timeout(volatile int* abort, int32_t* err) {
  *abort = 1;
  if (err) atomicCAS(err, 0, kDevTimeout);
}

template <int BN, int NS>
__global__ void __launch_bounds__(NT, 1) k_bf16x3(const Args p) {
  using Ly = Lay<BN, NS>;
  constexpr int STAGES = Ly::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  int64_t* sRA = reinterpret_cast<int64_t*>(smem + Ly::SCAT);
  int64_t* sRC = sRA + BM;
  int64_t* sCB = sRC + BM;
  int64_t* sCC = sCB + BN;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Ly::BARS);
  uint64_t* empty = full + STAGES;
  uint64_t* accfull = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + Ly::MISC);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + Ly::MISC + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t tile = blockIdx.x;
  const int64_t m0 = (tile / p.tiles_n) * BM, n0 = (tile % p.tiles_n) * BN;
  const int ks = blockIdx.y;
  const int64_t kbeg = (int64_t)ks * p.k_per_split;
  const int64_t kend = kbeg + p.k_per_split < p.k ? kbeg + p.k_per_split : p.k;
  const int64_t KT = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
  const int rows_a = (int)(p.m - m0 < BM ? p.m - m0 : BM);
  const int rows_b = (int)(p.n - n0 < BN ? p.n - n0 : BN);

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], NPROD);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accfull, 1);
    *abort = 0;
    fence_mbar_init();
  }
  if (warp == MMA_WARP) {
    tmem_alloc(tmem_slot, BN);
    tmem_relinquish();
  }
  for (int i = tid; i < BM; i += NT) {
    sRA[i] = i < rows_a ? p.sp.rA[m0 + i] : 0;
    sRC[i] = i < rows_a ? p.sp.rC[m0 + i] : 0;
  }
  for (int i = tid; i < BN; i += NT) {
    sCB[i] = i < rows_b ? p.sp.cB[n0 + i] : 0;
    sCC[i] = i < rows_b ? p.sp.cC[n0 + i] : 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp < MMA_WARP) {
    // ---- producers: gather one k-tile ahead, split, stage ----
    PanelRegs<BM> ra0, ra1;
    PanelRegs<BN> rb0, rb1;
    auto load = [&](int64_t kt, PanelRegs<BM>& ra, PanelRegs<BN>& rb) {
      const int64_t k0 = kbeg + kt * BK;
      panel_load<BM>(ra, tid, p.a, sRA, rows_a, p.sp.cA, p.sp.cbsA, k0, kend, p.a_kc);
      panel_load<BN>(rb, tid, p.b, sCB, rows_b, p.sp.rB, p.sp.rbsB, k0, kend, p.b_kc);
    };
    auto stage = [&](int64_t kt, const PanelRegs<BM>& ra, const PanelRegs<BN>& rb) -> bool {
      const int s = (int)(kt % STAGES);
      const uint32_t ph = (uint32_t)((kt / STAGES) & 1);
      if (!mbar_wait(&empty[s], ph ^ 1, abort)) {
        record_timeout(abort, p.err);
        return false;
      }
      uint8_t* st = smem + s * Ly::STAGE;
      panel_store<BM, NS>(ra, tid, p.a_kc, st);
      panel_store<BN, NS>(rb, tid, p.b_kc, st + Ly::B_OFF);
      fence_proxy_async_smem();
      mbar_arrive(&full[s]);
      return true;
    };
    if (KT > 0) load(0, ra0, rb0);
    for (int64_t kt = 0; kt < KT; kt += 2) {
      if (kt + 1 < KT) load(kt + 1, ra1, rb1);
      if (!stage(kt, ra0, rb0)) break;
      if (kt + 1 >= KT) break;
      if (kt + 2 < KT) load(kt + 2, ra0, rb0);
      if (!stage(kt + 1, ra1, rb1)) break;
    }
    // ---- epilogue ----
    bool have_acc = KT > 0;
    if (have_acc && !*abort) {
      if (!mbar_wait(accfull, 0, abort)) {
        record_timeout(abort, p.err);
      }
    }
    tc_fence_after();
    const int q = warp & 3, hsel = warp >> 2;
    const int row = 32 * q + lane;
    const bool mv = row < rows_a;
    const bool ok = !*abort;
    for (int cb = hsel * (BN / 2); cb < (hsel + 1) * (BN / 2); cb += 16) {
      float v[16];
      if (have_acc && ok) {
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)cb, v);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
      }
      if (!ok) continue;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = cb + j;
        if (mv && col < rows_b) {
          if (p.splits == 1) {
            float* cp = p.c + sRC[row] + sCC[col];
            double r = p.alpha * (double)v[j];
            if (p.beta != 0.0) r += p.beta * (double)*cp;
            *cp = (float)r;
          } else {
            p.partial[((int64_t)ks * p.n + (n0 + col)) * p.m + (m0 + row)] = v[j];
          }
        }
      }
    }
  } else if (lane == 0) {
    // ---- MMA issue (one thread) ----
    constexpr uint32_t idesc = idesc_bf16_f32(BM, BN);
    const uint32_t base = smem_u32(smem);
    for (int64_t kt = 0; kt < KT; ++kt) {
      const int s = (int)(kt % STAGES);
      const uint32_t ph = (uint32_t)((kt / STAGES) & 1);
      if (!mbar_wait(&full[s], ph, abort)) {
        record_timeout(abort, p.err);
        break;
      }
      tc_fence_after();
      const uint32_t st = base + s * Ly::STAGE;
#pragma unroll
      for (int ksl = 0; ksl < BK / 16; ++ksl) {
        // k-slice ksl covers k-chunks 2*ksl, 2*ksl+1 (LBO apart); row groups SBO = 128 B apart
        const uint32_t ao = ksl * 2 * (BM / 8) * 128, bo = ksl * 2 * (BN / 8) * 128;
        uint64_t dA[NS], dB[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
          dA[i] = smem_desc(st + i * Ly::A_BYTES + ao, (BM / 8) * 128, 128);
          dB[i] = smem_desc(st + Ly::B_OFF + i * Ly::B_BYTES + bo, (BN / 8) * 128, 128);
        }
        // every product of pieces i, j with i + j < NS: the terms of relative
        // size above 2^-8NS (three for NS = 2, six for NS = 3)
        mma_bf16_ss(tmem, dA[0], dB[0], idesc, (kt > 0 || ksl > 0) ? 1u : 0u);
#pragma unroll
        for (int tsum = 1; tsum < NS; ++tsum)
#pragma unroll
          for (int i = 0; i <= tsum; ++i) mma_bf16_ss(tmem, dA[i], dB[tsum - i], idesc, 1u);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(accfull);
  }

  // ---- teardown: every MMA has completed before Tensor Memory is released ----
  if (warp == MMA_WARP && lane == 0 && KT > 0) {
    if (!mbar_wait(accfull, 0, abort)) record_timeout(abort, p.err);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    tmem_dealloc(tmem, BN);
  }
}

__global__ void k_splitk_reduce(const float* __restrict__ partial, float* __restrict__ c,
                                const int64_t* __restrict__ rC, const int64_t* __restrict__ cC,
                                int64_t M, int64_t N, int S, double alpha, double beta) {
  const int64_t total = M * N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = t % M, n = t / M;
    double s = 0.0;
    for (int ks = 0; ks < S; ++ks) s += (double)partial[((int64_t)ks * N + n) * M + m];
    float* cp = c + rC[m] + cC[n];
    double r = alpha * s;
    if (beta != 0.0) r += beta * (double)*cp;
    *cp = (float)r;
  }
}

template <int BN, int NS>
cudaError_t launch_bn(const Bf16Launch& q, cudaStream_t s) {
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_bf16x3<BN, NS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Lay<BN, NS>::ALLOC);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  Args a;
  a.a = (const float*)q.a;
  a.b = (const float*)q.b;
  a.c = (float*)q.c;
  a.partial = q.partial;
  a.sp = q.sp;
  a.m = q.m;
  a.n = q.n;
  a.k = q.k;
  a.alpha = q.alpha;
  a.beta = q.beta;
  a.a_kc = q.a_k_contig;
  a.b_kc = q.b_k_contig;
  a.tiles_n = (q.n + BN - 1) / BN;
  a.splits = q.splits;
  a.k_per_split = q.k_per_split;
  a.err = q.err;
  const int64_t tiles = ((q.m + BM - 1) / BM) * a.tiles_n;
  if (tiles == 0) return cudaSuccess;
  if (tiles > 0x7fffffffLL || q.splits > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)tiles, (unsigned)q.splits);
  mainloop_event_before(s);
  k_bf16x3<BN, NS><<<grid, NT, Lay<BN, NS>::ALLOC, s>>>(a);
  note_launch();
  if (q.splits > 1) {
    int64_t blocks = (q.m * q.n + 255) / 256;
    if (blocks > 16384) blocks = 16384;
    k_splitk_reduce<<<(int)blocks, 256, 0, s>>>(q.partial, (float*)q.c, q.sp.rC, q.sp.cC, q.m,
                                                 q.n, q.splits, q.alpha, q.beta);
    note_launch();
  }
  mainloop_event_after(s);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_bf16x3(const Bf16Launch& q, cudaStream_t s) {
  if (q.pieces == 3) return q.bn == 256 ? launch_bn<256, 3>(q, s) : launch_bn<128, 3>(q, s);
  return q.bn == 256 ? launch_bn<256, 2>(q, s) : launch_bn<128, 2>(q, s);
}

}  // namespace tc
