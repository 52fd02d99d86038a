// K3 + K5: the FP32 contraction on the fifth-generation tensor cores (tcgen05),
// persistent over output tiles (of one problem, or of a batch of problems).
//
// Each operand panel reaches a raw FP32 stage in shared memory in one of two
// ways.  Gathered in place through the scatter vectors of Section 6.1 --
// 16-byte cp.async copies wherever the block-scatter vectors of Section 6.2
// (or the row scatter entries) show a unit-stride run of four, 4-byte copies
// otherwise, zero-filled past the end of the contracted range -- or, when the
// tiles of both operands are boxes in their own dims (the BOX form), as one
// TMA box per operand and k-tile, which lands in exactly the layout the gather
// produces.  Converter warps split every value into bf16 pieces
// (x = b0 + b1 [+ b2], each b_i = RN_bf16 of the residual left so far, every
// residual exact in FP32): A's pieces straight into Tensor Memory
// (tcgen05.st; one thread per row, the tensor core's A-in-TMEM layout), B's
// into shared memory in the tensor core's K-major canonical layout.  One
// elected thread issues, per 16-wide k-slice, a tcgen05.mma (A from Tensor
// Memory, B from shared memory) for every piece pair (i, j) with i + j <
// pieces -- three for two pieces (BF16x3), six for three (BF16x6) -- into an
// FP32 accumulator in Tensor Memory.  Keeping A's pieces out of shared memory
// cuts the shared-memory traffic per k-tile, which with the tensor core's
// operand reads is what sets the pace, by a quarter or more.
//
// Accumulation: the tensor core adds in FP32 with unspecified rounding, and
// over thousands of terms that alone exceeds 1e-5 of sum|a||b| (measured on
// the spiky 4096^3 workload: 2.25e-5 with 4096-term chains).  So a tile's
// contracted range is processed in chunks of at most 1024 terms, each into a
// fresh accumulator, and the epilogue warps add the finished chunks into a
// running FP32 sum that stays in Tensor Memory, releasing the accumulator to
// the next chunk's MMAs as soon as they have read it.  A work item holds at
// most 16 chunks (the planner splits longer ranges across items), so the
// folds add at most 16 roundings of 2^-24 of the sum's magnitude (below 1e-6
// of sum|a||b|).  After the last chunk they apply alpha/beta through
// rscat(C) + cscat(C), or -- when a tile's range is split across items --
// store the FP32 partial that K4 sums with compensated (two-sum) arithmetic.
//
// Warp roles (672 threads; 704 in the BOX form): warps 0-7 load (cp.async),
// or in the BOX form convert, warps 8-15 convert, warps 16-19 run the
// epilogue (one per Tensor Memory lane quarter), warp 20 owns the Tensor
// Memory allocation (512 columns: the accumulator, the running sum, A's piece
// stages) and its lane 0 issues the MMAs, and in the
// BOX form lane 0 of warp 21 issues the boxes.  The output stores of one tile
// overlap the MMAs of the next.  Hand-offs go through mbarriers: raw_full
// (cp.async completion, or the boxes' transaction count) / raw_empty,
// mma_full / mma_empty (tcgen05.commit), acc_full (tcgen05.commit) /
// acc_empty.
// Every mbarrier wait is bounded: on expiry the CTA records
// TC_ERR_DEVICE_TIMEOUT in the device error word and raises a CTA-wide abort
// flag; the roles leave their loops together (barrier reductions of the
// flag), the MMA thread waits for its issued MMAs to drain, the box warp for
// its boxes in flight, and Tensor Memory is always released.
//
// Rows of a panel beyond the operand's edge are not gathered (a box reads
// them as zeros): a row of A (or B) only reaches the matching row (column) of
// the accumulator, which the epilogue skips.  Past the end of the contracted
// range the panels are zero-filled, since those entries reach every output.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "kernels.h"
#include "sm100_ptx.cuh"

namespace tc {
namespace {

using namespace ptx;

constexpr int BM = 128, BK = 32;
constexpr int NLOAD = 256, NCONV = 256, NEPI = 128;
// threads of a CTA: + the MMA warp, and the box warp in the BOX form
constexpr int nthreads(bool box) { return NLOAD + NCONV + NEPI + (box ? 64 : 32); }
constexpr int CONV_W0 = NLOAD / 32;
constexpr int EPI_W0 = (NLOAD + NCONV) / 32;
constexpr int MMA_WARP = (NLOAD + NCONV + NEPI) / 32;
constexpr int BOX_WARP = MMA_WARP + 1;  // issues the TMA box loads (BOX instantiation)
constexpr int BAR_LOAD = 1, BAR_CONV = 2, BAR_EPI = 3;
constexpr int KRING = 2;
// Batches take their work items from a shared counter: loader thread 0 claims
// items up to QPUB ahead of the loaders and publishes them in a ring of QR
// entries that every role reads in order.  A role lags the loaders by at most
// the pipeline's depth in items (raw and MMA stages plus the accumulator),
// well inside the ring.
constexpr int QR = 16, QPUB = 2;
constexpr int KSLOT = 2 * BK + 2 * (BK / 4);  // cA[32] rB[32] cbsA[8] rbsB[8]
constexpr int BNMAX = 128;        // widest output tile (columns)
constexpr int CHUNK_KT = 32;      // k-tiles per accumulation chunk (1024 terms)
constexpr int MAX_CHUNKS = 16;    // chunks per work item (longer ranges are split)
// Tensor Memory columns: accumulator, running sum, A's piece stages (16
// columns per piece and k-tile: 32 bf16 k-values, two per column)
constexpr uint32_t TM_ACC = 0, TM_SUM = BNMAX, TM_A = 2 * BNMAX, TM_COLS = 512;

// Shared-memory plan.  Raw FP32 stages hide the load latency; bf16 MMA stages
// (B's pieces in shared memory, A's in Tensor Memory) let the converters run
// ahead of the tensor core.
// PAIR: B's panels are half as wide (the pair splits the tile's columns), so
// a raw stage is 24 instead of 32 KB and seven of them fit.
template <int NS, bool BOX, bool PAIR = false>
struct Lay {
  static constexpr int RB = PAIR ? BNMAX / 2 : BNMAX;  // B rows per CTA
  // bf16 MMA stages, as many as Tensor Memory (A's pieces: NS x 16 of its 256
  // free columns per stage) and shared memory (B's pieces) allow: the ring of
  // MMA stages, each returned by a tcgen05.commit, paces the pipeline
  static constexpr int MS = PAIR ? (NS == 3 ? 5 : 8) : (NS == 3 ? 3 : 5);
  static constexpr int RS = PAIR ? 6 : 4;        // raw FP32 stages
  static constexpr int PB = RB * BK * 2;         // one bf16 piece of B
  static constexpr int MMA_STAGE = NS * PB;
  static constexpr uint32_t TA_STAGE = NS * 16;  // Tensor Memory columns of A's pieces
  static_assert(TM_A + MS * TA_STAGE <= TM_COLS, "Tensor Memory plan");
  static constexpr int RAW_A = BM * BK * 4;
  static constexpr int RAW_STAGE = RAW_A + RB * BK * 4;
  static constexpr int MMA0 = 0;
  static constexpr int RAW0 = MMA0 + MS * MMA_STAGE;
  static constexpr int SCAT = RAW0 + RS * RAW_STAGE;  // int64 rA[BM] cB[BNMAX] rC[BM] cC[BNMAX]
  static constexpr int KR = SCAT + (2 * BM + 2 * BNMAX) * 8;  // k ring: KRING x KSLOT int64
  static constexpr int PROB = KR + KRING * KSLOT * 8;
  static constexpr int BARS = PROB + (int)((sizeof(DevProblem) + 15) / 16 * 16);
  static constexpr int NBARS = 2 * RS + 2 * MS + 5;
  static constexpr int MISC = BARS + NBARS * 8;
  static constexpr int WQ = MISC + 16;  // work queue: QR int64 entries, QR full + QR empty barriers
  static constexpr int END = WQ + 3 * QR * 8;
  static constexpr int ALLOC = END + 1024;
  static_assert(ALLOC <= 227 * 1024, "shared memory plan exceeds the per-CTA limit");
  static_assert(BNMAX % NEPI == 0 && BM == NEPI && NLOAD % 32 == 0 && BK % (NLOAD / 32) == 0,
                "thread maps of the loaders and the epilogue");
};

// byte offset of (row r, k-chunk q of 8) in an R-row K-major bf16 panel:
// 8-row x 16-byte core matrices, rows 16 B apart inside one, row groups 128 B
// apart (SBO), k-chunks R*16 B apart (LBO)
template <int R>
__device__ __forceinline__ uint32_t panel_off(int r, int q) {
  return (uint32_t)((q * (R / 8) + (r >> 3)) * 128 + (r & 7) * 16);
}

// Split 8 FP32 values into NS bf16 pieces and store one 16-byte core-matrix
// row per piece (pieces `piece_bytes` apart).
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

struct Args {
  CUtensorMap tm[2];  // tensor maps of the single problem's box operands (A, B)
  DevProblem single;
  const DevProblem* probs;
  const WorkItem* items;
  int64_t nitems;
  int64_t tiles_single;
  int32_t* err;
  int fault;  // 1: injected timeout (see TcLaunch::fault)
  unsigned long long* counter;  // batch: the shared work counter (dynamic items), or null
  const int32_t* gate;  // checked launch: no work if *gate == kDevBounds (or null)
  int dbuf;  // every work item is one chunk: alternate two accumulators (see the epilogue)
};

__device__ __forceinline__ void record_timeout(volatile int* abort, int32_t* err) {
  *abort = 1;
  if (err) atomicCAS(err, 0, kDevTimeout);
}

struct __align__(16) Item {
  const DevProblem* d;
  int64_t m0, n0, kbeg, kend, KT;
  int split;
  int rows_a, rows_b;
  int nchunks;
};

// Output tile `tile` of problem d over k-split `split`.
// PAIR: the CTA pair's tile has 256 rows; CTA `crank` of the pair takes rows
// 128 crank .. 128 crank + 127 of it (all of its columns).
template <bool PAIR = false>
__device__ __forceinline__ Item item_of_tile(const DevProblem* d, int64_t tile, int split,
                                             uint32_t crank = 0) {
  Item it;
  it.d = d;
  it.split = split;
  it.m0 = (tile / d->tiles_n) * (PAIR ? 2 * BM : BM) + (PAIR ? (int64_t)BM * crank : 0);
  it.n0 = (tile % d->tiles_n) * d->bn;
  it.kbeg = (int64_t)it.split * d->kps;
  it.kend = it.kbeg + d->kps < d->k ? it.kbeg + d->kps : d->k;
  it.KT = it.kend > it.kbeg ? (it.kend - it.kbeg + BK - 1) / BK : 0;
  it.rows_a = (int)(d->m - it.m0 < BM ? d->m - it.m0 : BM);
  it.rows_b = (int)(d->n - it.n0 < d->bn ? d->n - it.n0 : d->bn);
  it.nchunks = it.KT > 0 ? (int)((it.KT + CHUNK_KT - 1) / CHUNK_KT) : 1;
  return it;
}

template <bool PAIR = false>
__device__ __forceinline__ Item get_item(const Args& a, const DevProblem* single, int64_t w,
                                         uint32_t crank = 0) {
  if (a.probs) {
    const WorkItem wi = a.items[w];
    return item_of_tile<PAIR>(a.probs + wi.prob, wi.tile, wi.split, crank);
  }
  return item_of_tile<PAIR>(single, w % a.tiles_single, (int)(w / a.tiles_single), crank);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// ---- loader: one raw FP32 panel of R rows x BK k through cp.async ----------------------
// Layouts of a raw stage:
//  * k-contiguous operand: raw[row][BK], the eight 16-byte chunks of a row
//    stored at position (chunk ^ (row & 7)), so that both the loaders' writes
//    and the converters' reads touch all 32 banks once per quarter-warp;
//  * row-contiguous operand: raw[BK][R].
// The k side of every address comes from a small ring in shared memory that
// holds, per k-tile, the 32 scatter entries of each operand along k and their
// 8 block-scatter entries; loader thread i < KSLOT owns entry i: it keeps the
// entries of the next four k-tiles in flight in registers and stores one
// per k-tile into the ring, so the latency of the scatter vectors stays off
// the critical path.  The row side of every address
// comes from the row scatter entries of the tile, also in shared memory.
// Consecutive threads walk each operand's unit-stride index.
// Entry `i` (< KSLOT) of the k-side ring: which vector it reads and where.
struct KSlotSrc {
  const int64_t* vec;
  int off;
  bool block;  // a block-scatter entry (k blocks of 4) rather than a scatter entry
};

__device__ __forceinline__ KSlotSrc kslot_src(int i, const DevProblem* d) {
  if (i < BK) return {d->sp.cA, i, false};
  if (i < 2 * BK) return {d->sp.rB, i - BK, false};
  if (i < 2 * BK + BK / 4) return {d->sp.cbsA, i - 2 * BK, true};
  return {d->sp.rbsB, i - 2 * BK - BK / 4, true};
}

__device__ __forceinline__ int64_t kslot_fetch(const KSlotSrc& src, int64_t k0, int64_t kend) {
  if (src.block) {
    const int64_t kb = (k0 >> 2) + src.off;
    return (kb << 2) < kend ? __ldg(src.vec + kb) : 0;
  }
  return k0 + src.off < kend ? __ldg(src.vec + k0 + src.off) : 0;
}

// ---- box loads (operands whose tiles are TMA boxes) ------------------------------
// Issued by one lane of the box warp; coordinates live in its registers.
//
// Coordinates of the box whose rows start at linear row r0 and whose k-tile
// starts at linear k index k0: the mixed-radix digits of r0 and k0 over the
// two bundles' extents (the last dim of each bundle keeps the quotient, which
// may point past its end: the box reads zeros there).  Once per work item.
__device__ __forceinline__ void box_coords(const BoxAccess& x, uint32_t r0, uint32_t k0,
                                           int32_t (&c)[5]) {
  uint32_t v1 = x.kfirst ? k0 : r0, v2 = x.kfirst ? r0 : k0;
  const int rank = x.rank, nf = x.nfirst;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    c[i] = 0;
    if (i < rank) {
      const bool first = i < nf;
      const bool lastdim = i == nf - 1 || i == rank - 1;
      const uint32_t v = first ? v1 : v2;
      const uint32_t len = (uint32_t)x.len[i];
      c[i] = (int32_t)(lastdim ? v : v % len);
      const uint32_t q = lastdim ? 0u : v / len;
      if (first) v1 = q; else v2 = q;
    }
  }
}

// The next k-tile's box: one step along the dim the k-tile ends in, carried
// into the k bundle's higher dims (the step divides that dim's extent, so a
// wrap lands exactly on 0; the bundle's last dim is not wrapped).
__device__ __forceinline__ void box_advance(const BoxAccess& x, int32_t (&c)[5]) {
  const int sd = x.kstep_dim, kl = x.klast;
  bool carry = false;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    if (i == sd) c[i] += x.kstep;
    else if (carry) c[i] += 1;
    carry = i >= sd && i < kl && c[i] >= x.len[i];
    if (carry) c[i] = 0;
  }
}

template <int R>
__device__ __forceinline__ void load_panel(int t, uint32_t raw, const float* __restrict__ base,
                                           const int64_t* rowsc, int rows_valid,
                                           const int64_t* ks, const int64_t* kbs, int64_t k0,
                                           int64_t kend, bool kcontig, bool vec_ok) {
  if (kcontig) {
    constexpr int RSTEP = NLOAD / 8;  // rows per pass of the loaders
    const int q4 = t & 7;
    const int64_t kq = k0 + 4 * q4;
    const bool vec = vec_ok && kq + 3 < kend && kbs[q4] == 1;
    int64_t ko[4];
    uint32_t valid = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      ko[j] = ks[4 * q4 + j];
      valid |= (uint32_t)(kq + j < kend) << j;
    }
#pragma unroll
    for (int i = 0; i < R / RSTEP; ++i) {
      const int r = (t >> 3) + RSTEP * i;
      if (r < rows_valid) {
        const uint32_t dst = raw + (uint32_t)(r * BK * 4 + ((q4 ^ (r & 7)) << 4));
        const float* rowp = base + rowsc[r];
        const float* p = rowp + ko[0];
        if (vec && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
          cp_async16(dst, p, 16);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const bool ok = (valid >> j) & 1;
            cp_async4(dst + 4 * j, ok ? rowp + ko[j] : base, ok ? 4u : 0u);
          }
        }
      }
    }
  } else {
    constexpr int KSTEP = NLOAD / 32;  // k positions per pass of the loaders
    const int kk0 = t >> 5;
#pragma unroll
    for (int u = 0; u < R / 128; ++u) {
      const int r0 = 4 * ((t & 31) + 32 * u);
      if (r0 >= rows_valid) continue;
      const int64_t o0 = rowsc[r0];
      const bool quad = vec_ok && r0 + 3 < rows_valid && rowsc[r0 + 1] == o0 + 1 &&
                        rowsc[r0 + 2] == o0 + 2 && rowsc[r0 + 3] == o0 + 3;
#pragma unroll
      for (int v = 0; v < BK / KSTEP; ++v) {
        const int kk = kk0 + KSTEP * v;
        const uint32_t dst = raw + (uint32_t)(kk * R + r0) * 4;
        const bool ok = k0 + kk < kend;
        const int64_t ko = ks[kk];
        const float* p = base + o0 + ko;
        if (ok && quad && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
          cp_async16(dst, p, 16);
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            if (r0 + i < rows_valid)
              cp_async4(dst + 4 * i, ok ? base + rowsc[r0 + i] + ko : base, ok ? 4u : 0u);
          }
        }
      }
    }
  }
}

// ---- converter: raw panel -> NS bf16 pieces in the canonical layout ------------------
// Task c = (row r = c % R, k-chunk q = c / R): a warp covers 32 consecutive
// rows of one k-chunk, so its 16-byte core-matrix row stores are contiguous.
template <int R, int NS, int NTH>
__device__ __forceinline__ void convert_panel(int t, const uint8_t* raw, uint8_t* piece0,
                                              bool kcontig, int rstride) {
  constexpr int TASKS = R * BK / 8;
  constexpr int PBY = R * BK * 2;
  static_assert(TASKS % NTH == 0 || NTH % TASKS == 0, "converter tasks per thread");
  const float* rf = reinterpret_cast<const float*>(raw);
  if (TASKS < NTH && t >= TASKS) return;  // fewer tasks than threads: one each
#pragma unroll
  for (int i = 0; i < (TASKS + NTH - 1) / NTH; ++i) {
    const int c = t + i * NTH;
    const int r = c % R, q = c / R;
    float v[8];
    if (kcontig) {
      const float* row = rf + r * BK;
      const float4 x0 = *reinterpret_cast<const float4*>(row + (((2 * q) ^ (r & 7)) << 2));
      const float4 x1 = *reinterpret_cast<const float4*>(row + (((2 * q + 1) ^ (r & 7)) << 2));
      v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
      v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = rf[(8 * q + j) * rstride + r];
    }
    split8_store<NS>(v, piece0, PBY, panel_off<R>(r, q));
  }
}
// A's raw panel (BM rows x BK k) into NS bf16 pieces in Tensor Memory at
// column `tcol` (+16 per piece).  Converter warp cw (of NCVW) may access only
// its Tensor Memory lane quarter cw % 4 (its warp index in the CTA is cw plus
// a multiple of 4), so it converts rows 32 (cw % 4) + lane, and of each row
// the 8-value k-chunks cw / 4, cw / 4 + NCVW / 4, ...; a chunk's pieces are
// four columns each.
template <int NS, int NCVW>
__device__ __forceinline__ void convert_a_tmem(int cw, int lane, const uint8_t* raw,
                                               uint32_t tmem, uint32_t tcol, bool kcontig) {
  static_assert(NCVW % 4 == 0 && 4 % (NCVW / 4) == 0, "converter warps per lane quarter");
  const float* rf = reinterpret_cast<const float*>(raw);
  const int q = cw & 3, r = 32 * q + lane;
  const uint32_t base = tmem + ((uint32_t)(32 * q) << 16) + tcol;
#pragma unroll
  for (int c = cw >> 2; c < BK / 8; c += NCVW / 4) {
    float v[8];
    if (kcontig) {
      const float* row = rf + r * BK;
      const float4 x0 = *reinterpret_cast<const float4*>(row + (((2 * c) ^ (r & 7)) << 2));
      const float4 x1 = *reinterpret_cast<const float4*>(row + (((2 * c + 1) ^ (r & 7)) << 2));
      v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
      v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = rf[(8 * c + j) * BM + r];
    }
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
      tmem_st4(base + (uint32_t)(sidx * 16 + c * 4), w);
    }
  }
}

// BOX = false: the loader warps gather every operand through the scatter
// vectors (no box code at all).  BOX = true: both operands of every work item
// are TMA boxes, issued by the box warp; there are no loaders, and their eight
// warps convert alongside the converters.
template <int NS, bool BOX, bool PAIR>
__global__ void __launch_bounds__(nthreads(BOX), 1) k_tc(const __grid_constant__ Args a) {
  static_assert(BOX || !PAIR, "the pair form loads both operands as boxes");
  constexpr int NCV = BOX ? NLOAD + NCONV : NCONV;  // converter threads
  // B rows per CTA: the pair splits the tile's columns between its two CTAs
  // (its bf16 pieces then lie RB * BK * 2 bytes apart in a stage)
  constexpr int RB = PAIR ? BNMAX / 2 : BNMAX;
  using Ly = Lay<NS, BOX, PAIR>;
  static_assert(RB == Ly::RB, "B rows per CTA");
  constexpr int RS = Ly::RS, MS = Ly::MS;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // align to 1 KB by offsetting the shared-memory pointer itself, so that the
  // compiler keeps every access below in the shared state space
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  int64_t* sRA = reinterpret_cast<int64_t*>(smem + Ly::SCAT);  // loaders' rows
  int64_t* sRC = sRA + BM + BNMAX;                            // epilogue's rows
  int64_t* sCC = sRC + BM;
  int64_t* kring = reinterpret_cast<int64_t*>(smem + Ly::KR);
  DevProblem* sProb = reinterpret_cast<DevProblem*>(smem + Ly::PROB);
  uint64_t* raw_full = reinterpret_cast<uint64_t*>(smem + Ly::BARS);
  uint64_t* raw_empty = raw_full + RS;
  uint64_t* mma_full = raw_empty + RS;
  uint64_t* mma_empty = mma_full + MS;
  uint64_t* acc_full = mma_empty + MS;  // [0], and [1] with two accumulators
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + Ly::MISC);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + Ly::MISC + 4);
  volatile int64_t* wq = reinterpret_cast<volatile int64_t*>(smem + Ly::WQ);
  uint64_t* wq_full = reinterpret_cast<uint64_t*>(smem + Ly::WQ + QR * 8);
  uint64_t* wq_empty = wq_full + QR;
  // one release per entry from every warp of the loaders, converters and
  // epilogue, and from the MMA thread
  constexpr int NWQ = (NLOAD + NCV + NEPI) / 32 + 1;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < RS; ++s) {
      // BOX: the box warp's one arrival, with the transaction count
      mbar_init(&raw_full[s], BOX ? 1 : NLOAD);
      mbar_init(&raw_empty[s], NCV / 32);  // one arrival per converter warp
    }
    // pair form: the even CTA's mma_full and acc_empty also count the odd
    // CTA's converter warps and epilogue threads (remote arrivals)
    for (int s = 0; s < MS; ++s) {
      mbar_init(&mma_full[s], (PAIR ? 2 : 1) * NCV / 32);
      mbar_init(&mma_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], (PAIR ? 2 : 1) * NEPI);
    }
    mbar_init(drain, 1);
    for (int q = 0; q < QR; ++q) {
      mbar_init(&wq_full[q], 1);
      mbar_init(&wq_empty[q], NWQ);
    }
    // a checked launch whose scatter-vector check failed starts aborted: every
    // role leaves its loop at once, nothing is loaded or stored
    *abort = (a.gate && *a.gate == kDevBounds) ? 2 : 0;
    *sProb = a.single;
    fence_mbar_init();
  }
  // the pair's two CTAs allocate together: the same columns in both
  if (warp == MMA_WARP) {
    if constexpr (PAIR) {
      tmem_alloc2(tmem_slot, TM_COLS);
      tmem_relinquish2();
    } else {
      tmem_alloc(tmem_slot, TM_COLS);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  // both CTAs' barriers are initialised before any arrival from the other
  if constexpr (PAIR) cluster_sync();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int64_t nitems = a.nitems;
  // pair form: the pair (cluster) takes work items, both CTAs the same ones
  const uint32_t crank = PAIR ? cluster_ctarank() : 0u;
  const int64_t w0 = PAIR ? blockIdx.x / 2 : blockIdx.x, dw = PAIR ? gridDim.x / 2 : gridDim.x;
  // dynamic items (batches, gather form): the j-th item of this CTA is entry
  // j of the work queue; otherwise items w0, w0 + dw, ...
  const bool dyn = !BOX && a.counter != nullptr;
  auto item_of = [&](int64_t j) -> int64_t {
    if (!dyn) return w0 + j * dw;
    const int q = (int)(j % QR);
    if (!mbar_wait(&wq_full[q], (uint32_t)((j / QR) & 1), abort)) {
      record_timeout(abort, a.err);
      return nitems;
    }
    return wq[q];
  };
  // this warp has read entry j (its warps' lanes converge first)
  auto release_item = [&](int64_t j) {
    if (!dyn) return;
    __syncwarp();
    if (lane == 0) mbar_arrive(&wq_empty[j % QR]);
  };

  if (!BOX && warp < CONV_W0) {
    // ---- loaders ----
    const int t = tid;
    int64_t g = 0;  // k-tiles staged by this CTA so far
    // row scatter entries (A rows then B rows) of the next item, fetched one item ahead
    constexpr int NR = (BM + BNMAX + NLOAD - 1) / NLOAD;
    int64_t pre[NR];
    auto fetch_rows = [&](const Item& it) {
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        const int r = t + i * NLOAD;
        pre[i] = 0;
        if (r < BM) {
          if (r < it.rows_a) pre[i] = __ldg(it.d->sp.rA + it.m0 + r);
        } else if (r < BM + BNMAX) {
          if (r - BM < it.rows_b) pre[i] = __ldg(it.d->sp.cB + it.n0 + (r - BM));
        }
      }
    };
    // the claimer (thread 0): entries up to `last` claimed and published
    int64_t pub = 0;
    bool pub_end = false;
    auto publish_upto = [&](int64_t last) {
      while (!pub_end && pub <= last) {
        const int q = (int)(pub % QR);
        if (!mbar_wait(&wq_empty[q], (uint32_t)(((pub / QR) & 1) ^ 1), abort)) {
          record_timeout(abort, a.err);
          pub_end = true;
          return;
        }
        int64_t wc = pub == 0 ? w0 : dw + (int64_t)atomicAdd(a.counter, 1ull);
        if (wc >= nitems) {
          wc = nitems;  // the end of this CTA's sequence
          pub_end = true;
        }
        wq[q] = wc;
        mbar_arrive(&wq_full[q]);
        ++pub;
      }
    };
    if (dyn && t == 0) publish_upto(QPUB - 1);
    int64_t w = item_of(0);
    if (w < nitems) fetch_rows(get_item<PAIR>(a, sProb, w, crank));
    for (int64_t j = 0;; ++j) {
      // uniform exit; previous rows consumed
      if (bar_or(BAR_LOAD, NLOAD, *abort || w >= nitems)) break;
      if (dyn && t == 0) publish_upto(j + QPUB);
      const Item it = get_item<PAIR>(a, sProb, w, crank);
      const DevProblem* d = it.d;
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        const int r = t + i * NLOAD;
        if (r < BM + BNMAX) sRA[r] = pre[i];  // B rows follow A rows
      }
      w = item_of(j + 1);
      release_item(j);
      if (w < nitems) fetch_rows(get_item<PAIR>(a, sProb, w, crank));
      const float* A = static_cast<const float*>(d->a);
      const float* B = static_cast<const float*>(d->b);
      const bool akc = d->a_kc, bkc = d->b_kc;
      const bool vec_ok = d->elem_gather == 0;
      // k ring: entry t of k-tile 0 now, of k-tiles 1..4 in flight in p0..p3
      KSlotSrc src{nullptr, 0, false};
      int64_t p0 = 0, p1 = 0, p2 = 0, p3 = 0;
      if (t < KSLOT) {
        src = kslot_src(t, d);
        auto kf = [&](int64_t kt) { return kt < it.KT ? kslot_fetch(src, it.kbeg + kt * BK, it.kend) : 0; };
        const int64_t v0 = kf(0);
        p0 = kf(1);
        p1 = kf(2);
        p2 = kf(3);
        p3 = kf(4);
        if (it.KT > 0) kring[t] = v0;
      }
      bar_sync(BAR_LOAD, NLOAD);
      for (int64_t kt = 0; kt < it.KT; ++kt, ++g) {
        if (t < KSLOT) {  // publish k-tile kt+1, fetch k-tile kt+5
          if (kt + 1 < it.KT) kring[((kt + 1) % KRING) * KSLOT + t] = p0;
          p0 = p1;
          p1 = p2;
          p2 = p3;
          p3 = kt + 5 < it.KT ? kslot_fetch(src, it.kbeg + (kt + 5) * BK, it.kend) : 0;
        }
        const int s = (int)(g % RS);
        const bool ok = mbar_wait(&raw_empty[s], (uint32_t)(((g / RS) & 1) ^ 1), abort);
        if (!ok) record_timeout(abort, a.err);
        if (ok) {
          const uint32_t raw = smem_u32(smem + Ly::RAW0 + s * Ly::RAW_STAGE);
          const int64_t* slot = kring + (kt % KRING) * KSLOT;
          const int64_t k0 = it.kbeg + kt * BK;
          load_panel<BM>(t, raw, A, sRA, it.rows_a, slot, slot + 2 * BK, k0, it.kend, akc,
                         vec_ok);
          load_panel<BNMAX>(t, raw + Ly::RAW_A, B, sRA + BM, it.rows_b, slot + BK,
                            slot + 2 * BK + BK / 4, k0, it.kend, bkc, vec_ok);
          cp_async_arrive(&raw_full[s]);
        }
        // slot kt+1 now complete and slot kt free for reuse; a timeout anywhere
        // makes every loader leave together
        if (bar_or(BAR_LOAD, NLOAD, !ok)) break;
      }
    }
    // no copy into shared memory may outlive the CTA (matters only after an abort)
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  } else if (warp < EPI_W0) {
    // ---- converters ----
    const int t = BOX ? tid : tid - NLOAD;
    int64_t g = 0;
    int64_t w = item_of(0);
    for (int64_t j = 0;; ++j) {
      if (bar_or(BAR_CONV, NCV, *abort || w >= nitems)) break;  // uniform exit
      const Item it = get_item<PAIR>(a, sProb, w, crank);
      w = item_of(j + 1);
      release_item(j);
      const bool akc = it.d->a_kc, bkc = it.d->b_kc;
      // a row-contiguous B box holds k-rows of bn floats (pair form: bn / 2);
      // the gather's k-rows hold BNMAX
      const int rsB = BOX && !it.d->b_kc ? (PAIR ? it.d->bn / 2 : it.d->bn) : BNMAX;
      for (int64_t kt = 0; kt < it.KT; ++kt, ++g) {
        const int rs = (int)(g % RS), ms = (int)(g % MS);
        const bool ok = mbar_wait(&raw_full[rs], (uint32_t)((g / RS) & 1), abort) &&
                        mbar_wait<PAIR>(&mma_empty[ms], (uint32_t)(((g / MS) & 1) ^ 1), abort);
        if (!__all_sync(0xffffffffu, ok)) {  // the warp leaves together (it arrives as one)
          record_timeout(abort, a.err);
          break;
        }
        tc_fence_after();  // the MMAs that read this stage's A pieces are complete
        const uint8_t* raw = smem + Ly::RAW0 + rs * Ly::RAW_STAGE;
        uint8_t* st = smem + Ly::MMA0 + ms * Ly::MMA_STAGE;
        convert_a_tmem<NS, NCV / 32>(t >> 5, lane, raw, tmem, TM_A + (uint32_t)ms * Ly::TA_STAGE,
                                     akc);
        if (!BOX || rsB == RB)  // the common k-row pitch as a constant: immediate offsets
          convert_panel<RB, NS, NCV>(t, raw + Ly::RAW_A, st, bkc, RB);
        else
          convert_panel<RB, NS, NCV>(t, raw + Ly::RAW_A, st, bkc, rsB);
        // every lane's pieces in Tensor Memory and visible to the tensor
        // core's proxy in shared memory, every lane's raw reads done, then one
        // arrival per warp on each barrier
        tmem_st_wait();
        tc_fence_before();
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          if constexpr (PAIR) mbar_arrive_cluster(&mma_full[ms], 0);  // the even CTA issues
          else mbar_arrive(&mma_full[ms]);
          mbar_arrive(&raw_empty[rs]);
        }
      }
    }
  } else if (warp < MMA_WARP) {
    // ---- epilogue: one thread per accumulator row ----
    const int t = tid - NLOAD - NCONV;
    const int wq = warp & 3;  // Tensor Memory lane quarter of this warp
    const int row = 32 * wq + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * wq) << 16);
    constexpr int NB = BNMAX / NEPI;
    int64_t pre_r = 0, pre_c[NB];
    auto fetch_rows = [&](const Item& it) {
      pre_r = t < it.rows_a ? __ldg(it.d->sp.rC + it.m0 + t) : 0;
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        const int c = t + i * NEPI;
        pre_c[i] = c < it.rows_b ? __ldg(it.d->sp.cC + it.n0 + c) : 0;
      }
    };
    int64_t w = item_of(0);
    if (w < nitems) fetch_rows(get_item<PAIR>(a, sProb, w, crank));
    int64_t gc = 0;  // chunks finished by this CTA
    for (int64_t j = 0;; ++j) {
      // uniform exit; previous rows consumed
      if (bar_or(BAR_EPI, NEPI, *abort || w >= nitems)) break;
      const Item it = get_item<PAIR>(a, sProb, w, crank);
      const DevProblem* d = it.d;
      sRC[t] = pre_r;
#pragma unroll
      for (int i = 0; i < NB; ++i) sCC[t + i * NEPI] = pre_c[i];
      w = item_of(j + 1);
      release_item(j);
      if (w < nitems) fetch_rows(get_item<PAIR>(a, sProb, w, crank));
      bar_sync(BAR_EPI, NEPI);
      const bool have = it.KT > 0;
      // descriptor fields in registers: the stores below could alias them as
      // far as the compiler knows, which would reload them per element
      const int bn = d->bn;
      const bool direct = d->splits == 1;
      const float al = (float)d->alpha, be = (float)d->beta;
      float* const crow = static_cast<float*>(d->c) + sRC[row];
      float* const prow = direct ? nullptr
                                 : static_cast<float*>(d->partial) +
                                       ((int64_t)it.split * d->n + it.n0) * d->m + it.m0 + row;
      const int64_t pm = d->m;
      const bool mv = row < it.rows_a;
      const int cols = it.rows_b;
      bool ok = true;
      // output of 8 columns of the tile: alpha * (hi + lo) [+ beta * C], or the
      // partial.  The three cases are separate loops so that no load of C is
      // ever issued when beta == 0 (C is then only written), and the loads of
      // C for beta != 0 are all in flight before the first store.
      auto out8 = [&](int cb, const float (&hi)[8], const float (&lo)[8]) {
        if (!mv) return;
        if (!direct) {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (cb + q < cols) prow[(int64_t)(cb + q) * pm] = __fadd_rn(hi[q], lo[q]);
        } else if (be == 0.f) {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (cb + q < cols) crow[sCC[cb + q]] = __fmaf_rn(al, hi[q], al * lo[q]);
        } else {
          float old[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) old[q] = cb + q < cols ? crow[sCC[cb + q]] : 0.f;
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (cb + q < cols)
              crow[sCC[cb + q]] = __fmaf_rn(be, old[q], __fmaf_rn(al, hi[q], al * lo[q]));
        }
      };
      for (int ch = 0; ch < it.nchunks; ++ch, ++gc) {
        const bool first = ch == 0, last = ch + 1 == it.nchunks;
        // two accumulators (every item one chunk): the running-sum columns
        // serve as the second, and items alternate between them
        const int buf = a.dbuf ? (int)(gc & 1) : 0;
        const uint32_t use = (uint32_t)(a.dbuf ? gc >> 1 : gc);  // earlier uses of buf
        if (have && !*abort) {
          if (!mbar_wait<PAIR>(&acc_full[buf], use & 1u, abort)) record_timeout(abort, a.err);
        }
        tc_fence_after();
        ok = __all_sync(0xffffffffu, !*abort);
        // A short tile (one chunk of at most four k-tiles), or any tile when
        // there are two accumulators, is written straight from its
        // accumulator -- the running sum would hold the same values -- which
        // saves the round trip through the sum; with one accumulator that
        // holds it until the stores are issued, and for longer tiles the next
        // tile's MMAs gain more from having it released first.
        const bool direct_out = a.dbuf || (first && last && it.KT <= 4);
        if (ok && direct_out) {
          // 16 columns per Tensor Memory load and wait (bn is a multiple of 16)
          const uint32_t accc = buf ? TM_SUM : TM_ACC;
          float z[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) z[q] = 0.f;
          for (int cb = 0; cb < bn; cb += 16) {
            float v[16];
            if (have) {
              tmem_ld16(lane_base + accc + (uint32_t)cb, v);
            } else {
#pragma unroll
              for (int q = 0; q < 16; ++q) v[q] = 0.f;
            }
#pragma unroll
            for (int p8 = 0; p8 < 2; ++p8) {
              float v8[8];
#pragma unroll
              for (int q = 0; q < 8; ++q) v8[q] = v[8 * p8 + q];
              out8(cb + 8 * p8, v8, z);
            }
          }
        } else if (ok) {
          // fold the chunk into the running sum
          for (int cb = 0; cb < bn; cb += 8) {
            float v[8], sum[8];
            if (have) {
              tmem_ld8(lane_base + TM_ACC + (uint32_t)cb, v);
            } else {
#pragma unroll
              for (int q = 0; q < 8; ++q) v[q] = 0.f;
            }
            if (first) {
#pragma unroll
              for (int q = 0; q < 8; ++q) sum[q] = v[q];
            } else {
              tmem_ld8(lane_base + TM_SUM + (uint32_t)cb, sum);
#pragma unroll
              for (int q = 0; q < 8; ++q) sum[q] = __fadd_rn(sum[q], v[q]);
            }
            tmem_st8(lane_base + TM_SUM + (uint32_t)cb, sum);
          }
          tmem_st_wait();
        }
        // the accumulator is free for the next chunk's MMAs
        tc_fence_before();
        if constexpr (PAIR) mbar_arrive_cluster(&acc_empty[buf], 0);
        else mbar_arrive(&acc_empty[buf]);
        if (!ok) break;
        if (!last || direct_out) continue;  // (a short tile is written above)
        // the tile's output from the running sum
        for (int cb = 0; cb < bn; cb += 8) {
          float sum[8], z[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) z[q] = 0.f;
          tmem_ld8(lane_base + TM_SUM + (uint32_t)cb, sum);
          out8(cb, sum, z);
        }
      }
    }
  } else if (BOX && warp == BOX_WARP) {
    // ---- box loads (BOX instantiation): one lane issues every TMA box ----
    // Per k-tile it waits for the raw stage to be free, raises the stage's
    // transaction count by the bytes of its two boxes, issues them, and
    // arrives.  Its arrival follows its transaction count, so the phase
    // cannot complete before the boxes have landed.
    if (BOX && lane == 0) {
      int64_t g = 0, g_iss = -1;  // the last k-tile whose boxes were issued
      for (int64_t w = w0; w < nitems && !*abort; w += dw) {
        const Item it = get_item<PAIR>(a, sProb, w, crank);
        const DevProblem* d = it.d;
        const BoxAccess bxA = d->boxA, bxB = d->boxB;
        const CUtensorMap* maps = a.probs ? d->tmaps : a.tm;
        if (a.probs) {  // maps in the plan's device buffer (kernel parameters need no fence)
          fence_tensormap_acquire(maps);
          fence_tensormap_acquire(maps + 1);
        }
        const uint32_t bytes = (uint32_t)bxA.bytes + (uint32_t)bxB.bytes;
        int32_t cA[5], cB[5];
        box_coords(bxA, (uint32_t)it.m0, (uint32_t)it.kbeg, cA);
        box_coords(bxB, (uint32_t)(it.n0 + (PAIR ? crank * (uint32_t)(d->bn / 2) : 0u)),
                   (uint32_t)it.kbeg, cB);
        bool failed = false;
        for (int64_t kt = 0; kt < it.KT; ++kt, ++g) {
          const int s = (int)(g % RS);
          if (!mbar_wait(&raw_empty[s], (uint32_t)(((g / RS) & 1) ^ 1), abort)) {
            record_timeout(abort, a.err);
            failed = true;
            break;
          }
          const uint32_t raw = smem_u32(smem + Ly::RAW0 + s * Ly::RAW_STAGE);
          mbar_expect_tx(&raw_full[s], bytes);
          tma_load(raw, maps, cA, bxA.rank, &raw_full[s]);
          tma_load(raw + Ly::RAW_A, maps + 1, cB, bxB.rank, &raw_full[s]);
          box_advance(bxA, cA);
          box_advance(bxB, cB);
          mbar_arrive(&raw_full[s]);
          g_iss = g;
        }
        if (failed) break;
      }
      // no box load may outlive the CTA (matters only after an abort): a fill
      // that a later fill of the same stage followed was consumed before that
      // one began, so only the last RS k-tiles can be in flight; wait for
      // their phases.  A box lands within microseconds of its issue; the wait
      // is bounded (about 10 ms per stage) all the same.
      if (g_iss >= 0) {
        for (int64_t gi = g_iss - RS + 1 > 0 ? g_iss - RS + 1 : 0; gi <= g_iss; ++gi) {
          const long long t0 = clock64();
          while (!mbar_try_wait(&raw_full[gi % RS], (uint32_t)((gi / RS) & 1)) &&
                 clock64() - t0 < 20000000LL) {
          }
        }
      }
    }
  } else if (lane == 0) {
    // ---- MMA issue (pair form: the even CTA issues for both; the odd one
    // only waits, before releasing Tensor Memory, for the MMAs writing it) ----
    const uint32_t base = smem_u32(smem + Ly::MMA0);
    int64_t g = 0, gc = 0;
    bool failed = false;
    const bool issuer = !PAIR || crank == 0;
    if (issuer && a.fault == 1) {
      // injected failure: a bounded wait (about 10 ms) on a barrier nothing
      // arrives on yet; it expires, and the CTA unwinds through the abort path
      if (!mbar_wait(drain, 0, abort, 20000000LL)) {
        record_timeout(abort, a.err);
        failed = true;
      }
    }
    int64_t w = (failed || !issuer) ? nitems : item_of(0);
    for (int64_t j = 0; w < nitems && !*abort && !failed; ++j) {
      const Item it = get_item<PAIR>(a, sProb, w, crank);
      w = item_of(j + 1);
      if (dyn) mbar_arrive(&wq_empty[j % QR]);  // (this thread alone reads the queue here)
      const uint32_t idesc = idesc_bf16_f32(PAIR ? 2 * BM : BM, (uint32_t)it.d->bn);
      for (int ch = 0; ch < it.nchunks && !failed; ++ch, ++gc) {
        const int buf = a.dbuf ? (int)(gc & 1) : 0;
        const int64_t use = a.dbuf ? gc >> 1 : gc;  // earlier uses of this accumulator
        // the epilogue has read (or folded) this accumulator's previous chunk
        if (use > 0 && !mbar_wait<PAIR>(&acc_empty[buf], (uint32_t)((use - 1) & 1), abort)) {
          record_timeout(abort, a.err);
          failed = true;
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + (buf ? TM_SUM : TM_ACC);
        const int64_t kt0 = (int64_t)ch * CHUNK_KT;
        const int64_t kt1 = kt0 + CHUNK_KT < it.KT ? kt0 + CHUNK_KT : it.KT;
        for (int64_t kt = kt0; kt < kt1; ++kt, ++g) {
          const int ms = (int)(g % MS);
          if (!mbar_wait<PAIR>(&mma_full[ms], (uint32_t)((g / MS) & 1), abort)) {
            record_timeout(abort, a.err);
            failed = true;
            break;
          }
          tc_fence_after();
          const uint32_t st = base + ms * Ly::MMA_STAGE;
          const uint32_t ta = tmem + TM_A + (uint32_t)ms * Ly::TA_STAGE;
#pragma unroll
          for (int ksl = 0; ksl < BK / 16; ++ksl) {
            const uint32_t bo = ksl * 2 * (RB / 8) * 128;
            uint32_t tA[NS];
            uint64_t dB[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) {
              tA[i] = ta + (uint32_t)(i * 16 + ksl * 8);
              dB[i] = smem_desc(st + i * Ly::PB + bo, (RB / 8) * 128, 128);
            }
            auto mma = [&](uint32_t ta_, uint64_t db_, uint32_t accum) {
              if constexpr (PAIR) mma_bf16_ts2(acc, ta_, db_, idesc, accum);
              else mma_bf16_ts(acc, ta_, db_, idesc, accum);
            };
            mma(tA[0], dB[0], (kt > kt0 || ksl > 0) ? 1u : 0u);
#pragma unroll
            for (int ts = 1; ts < NS; ++ts)
#pragma unroll
              for (int i = 0; i <= ts; ++i) mma(tA[i], dB[ts - i], 1u);
          }
          if constexpr (PAIR) mma_commit2(&mma_empty[ms], 0x3);  // both CTAs' stages
          else mma_commit(&mma_empty[ms]);
        }
        if (failed) break;
        if (kt1 > kt0) {
          if constexpr (PAIR) mma_commit2(&acc_full[buf], 0x3);
          else mma_commit(&acc_full[buf]);
        } else if constexpr (PAIR) {  // nothing to accumulate: hand over at once
          mbar_arrive_cluster(&acc_full[buf], 0);
          mbar_arrive_cluster(&acc_full[buf], 1);
        } else {
          mbar_arrive(&acc_full[buf]);
        }
      }
    }
    // every MMA this thread issued has completed once this commit arrives (in
    // the pair form on both CTAs' drain barriers)
    if (issuer) {
      if constexpr (PAIR) mma_commit2(drain, 0x3);
      else mma_commit(drain);
    }
    if (!mbar_wait(drain, 0, abort)) {
      // even on abort, wait for the drain itself (bounded) before releasing TMEM
      const long long t0 = clock64();
      while (!mbar_try_wait(drain, 0) && clock64() - t0 < 4000000000LL) {
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync();  // both CTAs are done with both Tensor Memories
  if (warp == MMA_WARP) {
    tc_fence_after();
    if constexpr (PAIR) tmem_dealloc2(tmem, TM_COLS);
    else tmem_dealloc(tmem, TM_COLS);
  }
}

// K4: C = alpha * (sum of the FP32 partials of the k-splits) + beta * C.
// The partials are added with error-free transformations (Knuth's two-sum,
// then the collected errors once: the cascade "Sum2" of Ogita, Rump and
// Oishi), which yields the sum as if computed in twice FP32's precision
// before the final rounding -- for S <= 64 FP32 partials as good as an FP64
// sum -- while running on the FP32 pipes: on GB300 FP64 arithmetic is slow
// enough (about 1.1 TFLOP/s) that an FP64 reduction of tens of millions of
// elements costs a large share of the contraction itself.
// Grid: x over m, y over n, both with stride loops; no integer division per
// element.

// Columns [n0, n1) of one problem (the single-problem launch strides its
// block rows over all columns; the batched one hands each block row one).
// F64: the partials are summed in FP64 instead, alpha and beta applied in FP64,
// one rounding to FP32 at the end (the selectable tc_set_split_reduction form).
template <bool F64>
__device__ __forceinline__ void reduce_one(const DevProblem& d, int64_t n0, int64_t n1) {
  const int64_t M = d.m, plane = M * d.n;
  const int S = d.splits;
  const float* part = static_cast<const float*>(d.partial);
  float* c = static_cast<float*>(d.c);
  const float alpha = (float)d.alpha, beta = (float)d.beta;
  const bool stride_y = n1 - n0 > 1;
  for (int64_t n = n0 + (stride_y ? blockIdx.y : 0); n < n1; n += stride_y ? gridDim.y : 1) {
    const int64_t cn = __ldg(d.sp.cC + n);
    const float* pn = part + n * M;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
      const int64_t rm = __ldg(d.sp.rC + m);
      if (rm == kHole) continue;  // a hole of a blocked row bundle
      if constexpr (F64) {
        double sum = 0.0;
        for (int ks = 0; ks < S; ++ks) sum += (double)__ldg(pn + ks * plane + m);
        float* cp = c + rm + cn;
        double r = d.alpha * sum;
        if (d.beta != 0.0) r += d.beta * (double)*cp;
        *cp = (float)r;
        continue;
      }
      float hi = __ldg(pn + m), lo = 0.f;
      for (int ks = 1; ks < S; ++ks) {
        float e;
        two_sum(hi, __ldg(pn + ks * plane + m), hi, e);
        lo = __fadd_rn(lo, e);
      }
      float* cp = c + rm + cn;
      // alpha * (hi + lo) [+ beta * C], the small term folded in first; C is
      // only read when beta != 0
      const float r = __fmaf_rn(alpha, hi, alpha * lo);
      if (beta == 0.f) *cp = r;
      else *cp = __fmaf_rn(beta, *cp, r);
    }
  }
}

// One launch for the single problem, or for every split problem of a batch:
// block row y walks the flattened list of (problem, column) pairs, found from
// the prefix sums of the problems' column counts.
template <bool F64>
__global__ void k_reduce_partials(const DevProblem single, const DevProblem* probs,
                                  const int32_t* split_probs, const int64_t* col_prefix,
                                  int32_t n_split, const int32_t* gate) {
  if (gate && *gate == kDevBounds) return;
  if (!probs) {
    reduce_one<F64>(single, 0, single.n);
    return;
  }
  const int64_t total = col_prefix[n_split];
  for (int64_t r = blockIdx.y; r < total; r += gridDim.y) {
    int lo = 0, hi = n_split;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (col_prefix[mid] <= r) lo = mid; else hi = mid;
    }
    const int64_t n = r - col_prefix[lo];
    reduce_one<F64>(probs[split_probs[lo]], n, n + 1);
  }
}

// ---- the packed form (BLIS-style packing of Section 5, on the GPU) -------------------
// BLIS packs each operand's panels into a contiguous buffer once and reuses
// them across every block of the other operand; the paper (Sections 5-6) has
// the packing read the tensor through the scatter vectors, so that no tensor
// is ever transposed.  The packed form does the same in two steps:
//  * k_pack reads A (B) through its scatter vectors once, splits every value
//    into bf16 pieces exactly as the converters do, and writes each 128-row
//    (bn-row) x 32-k unit of the operand, all pieces, contiguously in the
//    tensor core's K-major canonical layout (units ordered row tile by row
//    tile, k-tile by k-tile);
//  * k_tcp streams the units of each work item into shared memory with one
//    bulk copy per operand and k-tile, and issues the same MMAs in the same
//    order as k_tc (A from shared memory), with the same chunked accumulation
//    and the same scattered epilogue.
// Gathering once instead of once per output tile across from the operand cuts
// the gathers by the operand's reuse (ceil(n / bn) for A, ceil(m / 128) for
// B), and the mainloop then has no loaders and no converters; the price is
// one write and one read of the packed operands (as many bytes as the FP32
// operands for two pieces).  The results equal k_tc's bit for bit.
// Units of every packing job in one launch: a single contraction's A and B
// (jobs in the parameter block), or those of every problem of a batch (jobs
// and their prefix sums of unit groups in device memory).
struct PackLaunch {
  PackJob local[2];
  int64_t local_prefix[3];
  const PackJob* jobs;    // batch: the jobs (device), or null
  const int64_t* prefix;  // batch: prefix sums of the jobs' unit groups (device, njobs + 1)
  int32_t njobs;
  int64_t total;          // unit groups of all jobs
  unsigned long long* claim;  // batch: the claim counter (zero at launch)
  int64_t chunk;              // batch: unit groups per claim
  const int32_t* gate;
};

// Units [u0, u1) of a job.  Task c = (row r = c % R, k-chunk q = c / R) of a
// unit packs eight values of one row (k past the range as zeros; rows past
// the operand are skipped); eight elements that the block-scatter vector
// shows at unit stride, from a 16-byte boundary, take two 16-byte loads.
// Each thread takes PK_TPT tasks at a time, a block's width apart, and
// issues all their loads before it splits and stores any of them: the launch
// is bound by the latency of its loads.  Two tasks per thread at five CTAs of
// 256 threads per SM (48 registers) measured best on the 512-problem batch:
// resident warps count for more than tasks per thread (four tasks at three
// CTAs per SM were slower than one task at four).
constexpr int PK_TPT = 2;
template <int NS>
__device__ __forceinline__ void pack_units(const PackJob& p, int64_t u0, int64_t u1) {
  const int R = p.R, per_unit = R * (BK / 8);
  const int nt = (int)((u1 - u0) * per_unit);  // a launch's share: far below 2^31
  const int unit_bytes = NS * R * BK * 2;
  for (int base = threadIdx.x; base < nt; base += PK_TPT * blockDim.x) {
    float v[PK_TPT][8];
    int uls[PK_TPT];  // the task's unit (from u0), or -1: nothing to store
    uint32_t off[PK_TPT];
#pragma unroll
    for (int i = 0; i < PK_TPT; ++i) {
      const int tt = base + i * (int)blockDim.x;
      uls[i] = -1;
      off[i] = 0;
      if (tt >= nt) continue;
      const int ul = tt / per_unit, c = tt - ul * per_unit;
      // a job's units number far below 2^32 (each is 2 KB or more)
      const uint32_t u = (uint32_t)u0 + (uint32_t)ul, KT = (uint32_t)p.KT;
      // a blocked unit's row r = lo0 + 16 lo1: consecutive threads take
      // consecutive lo1, the operand's unit-stride dim
      const int r = p.swz ? (c % R) / 8 + 16 * ((c % R) % 8) : c % R, q = c / R;
      const uint32_t tr = u / KT, kt = u - tr * KT;
      const int64_t row = (int64_t)tr * R + r;
      const int64_t kk0 = (int64_t)kt * BK + 8 * q;
      const int64_t ro = row < p.rows ? __ldg(p.rs + row) : kHole;
      // a row past the operand or a hole of a blocked bundle is not written: it
      // reaches only its own accumulator row (column), which is never stored
      if (ro == kHole) continue;
      uls[i] = ul;
      off[i] = (uint32_t)((q * (R / 8) + (r >> 3)) * 128 + (r & 7) * 16);
      const float* xr = p.x + ro;
      bool vec = false;
      if (kk0 + 7 < p.k) {
        const int64_t o = __ldg(p.ks + kk0);
        if (__ldg(p.kbs + (kk0 >> 2)) == 1 && __ldg(p.kbs + (kk0 >> 2) + 1) == 1 &&
            __ldg(p.ks + kk0 + 4) == o + 4 && (reinterpret_cast<uintptr_t>(xr + o) & 15) == 0) {
          const float4 x0 = __ldg(reinterpret_cast<const float4*>(xr + o));
          const float4 x1 = __ldg(reinterpret_cast<const float4*>(xr + o + 4));
          v[i][0] = x0.x; v[i][1] = x0.y; v[i][2] = x0.z; v[i][3] = x0.w;
          v[i][4] = x1.x; v[i][5] = x1.y; v[i][6] = x1.z; v[i][7] = x1.w;
          vec = true;
        }
      }
      if (!vec) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int64_t kk = kk0 + j;
          v[i][j] = kk < p.k ? __ldg(xr + __ldg(p.ks + kk)) : 0.f;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < PK_TPT; ++i)
      if (uls[i] >= 0) split8_store<NS>(v[i], p.out + (u0 + uls[i]) * (int64_t)unit_bytes, R * BK * 2, off[i]);
  }
}

// A single contraction's two jobs: the CTAs take the unit groups round robin
// (neighbouring units, which share sectors of the operand, are packed side by
// side).  A batch: the CTAs claim runs of `chunk` consecutive unit groups from
// a counter, so that the cost of a group, which varies with its operand's
// layout by several times, evens out over the CTAs (fixed contiguous ranges
// per CTA left the launch waiting on its slowest ranges); a run's job -- a
// binary search over the prefix sums -- is looked up only when it crosses
// into another job, and each job's part of a run is packed in one pass.
template <int NS>
__global__ void __launch_bounds__(256, 5) k_pack(const __grid_constant__ PackLaunch p) {
  if (p.gate && *p.gate == kDevBounds) return;
  if (!p.jobs) {
    for (int64_t g = blockIdx.x; g < p.total; g += gridDim.x) {
      const int j = g < p.local_prefix[1] ? 0 : 1;
      const PackJob& J = p.local[j];
      const int64_t u0 = (g - p.local_prefix[j]) * J.G;
      pack_units<NS>(J, u0, u0 + J.G < J.units ? u0 + J.G : J.units);
    }
    return;
  }
  // the claim and the current job live in shared memory (the job's fields,
  // held in registers, would cost the launch resident CTAs)
  __shared__ PackJob sJ;
  __shared__ int64_t s_claim, s_jlo, s_jhi;
  for (;;) {
    if (threadIdx.x == 0) s_claim = (int64_t)atomicAdd(p.claim, (unsigned long long)p.chunk);
    __syncthreads();
    const int64_t g0 = s_claim;
    if (g0 >= p.total) break;
    const int64_t g1 = g0 + p.chunk < p.total ? g0 + p.chunk : p.total;
    for (int64_t g = g0; g < g1;) {
      if (threadIdx.x == 0) {
        int lo = 0, hi = p.njobs;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (__ldg(p.prefix + mid) <= g) lo = mid; else hi = mid;
        }
        sJ = p.jobs[lo];
        s_jlo = __ldg(p.prefix + lo);
        s_jhi = __ldg(p.prefix + lo + 1);
      }
      __syncthreads();
      const int64_t jlo = s_jlo, jhi = s_jhi;
      const int64_t ge = jhi < g1 ? jhi : g1;  // this job's groups in the run: [g, ge)
      const int64_t ue = (ge - jlo) * sJ.G;
      pack_units<NS>(sJ, (g - jlo) * sJ.G, ue < sJ.units ? ue : sJ.units);
      __syncthreads();  // every thread is done with the job (and the claim) before they change
      g = ge;
    }
  }
}

struct PackedArgs {
  DevProblem single;           // the problem of a single call (probs == null)
  const DevProblem* probs;     // batch descriptors (device), or null
  const WorkItem* items;       // batch work list (device), or null
  int64_t nitems, tiles_single;
  int32_t* err;
  const int32_t* gate;
  int fault;  // 1: injected timeout (see TcLaunch::fault)
  int dual;   // two epilogue groups taking the work items in turn (see the epilogue)
  unsigned long long* counter;  // batch (single CTAs): the item claim counter (zero at launch), or null
  const Item* pitems;           // batch (single CTAs): the work items decoded at plan creation, or null
};

// Warps: producer, MMA, two groups of four epilogue warps (the second works
// for batches and for single contractions whose items are one accumulation
// chunk each: the groups then take the items in turn, each with its own
// accumulator); in the pair form also a relay warp that tells the pair's MMA
// issuer when its CTA's stage has landed.
constexpr int pk_threads(bool pair) { return pair ? 352 : 320; }
constexpr int PK_EPI_W0 = 2, PK_RELAY_WARP = 10;

// PAIR: CTA pairs (cta_group::2) on 256-row tiles; each CTA stages its own
// 128 rows of A and half of the tile's B rows (B is packed in half-tile
// units for it), which cuts every SM's operand bytes per k-tile by a quarter.
// A stage holds U consecutive k-tiles (units) of both operands: with two
// pieces, two k-tiles, so that each wait and commit of the MMA thread covers
// twelve MMAs; the tensor core takes a new MMA only about as fast as it
// finishes one, so the thread's fixed costs per stage (the barrier test, the
// commit, the loop) otherwise leave it idle for a third of the time.
template <int NS, bool PAIR = false>
struct PLay {
  static constexpr int U = NS == 2 ? 2 : 1;
  static constexpr int A_BYTES = NS * BM * BK * 2;  // one unit of A
  static constexpr int B_BYTES = NS * (PAIR ? BNMAX / 2 : BNMAX) * BK * 2;  // the widest unit of B
  static constexpr int STAGE = U * (A_BYTES + B_BYTES);  // U units of A, then U of B
  static constexpr int NSTG = PAIR ? (NS == 3 ? 5 : 4) : (NS == 3 ? 4 : 3);
  static constexpr int SCAT = NSTG * STAGE;  // per epilogue group int64 rC[BM] cC[BNMAX]
  static constexpr int PROB = SCAT + 2 * (BM + BNMAX) * 8;
  static constexpr int BARS = PROB + (int)((sizeof(DevProblem) + 15) / 16 * 16);
  static constexpr int NBARS = 3 * NSTG + 5;
  static constexpr int MISC = BARS + NBARS * 8;
  // decoded work items: the producer decodes each item once (for a batch,
  // from the work list and the problem's descriptor in device memory) and
  // hands it to the other roles through a ring in shared memory
  static constexpr int QRP = 16;
  // Item[QRP] (16-byte aligned: items are copied 16 bytes at a time), then
  // QRP full and QRP empty barriers
  static constexpr int RING = (MISC + 16 + 15) / 16 * 16;
  static constexpr int END = RING + QRP * (int)sizeof(Item) + 2 * QRP * 8;
  static constexpr int ALLOC = END + 1024;
  static_assert(ALLOC <= 227 * 1024, "shared memory plan exceeds the per-CTA limit");
  static_assert(sizeof(Item) % 16 == 0 && RING % 16 == 0 && (QRP & (QRP - 1)) == 0, "item ring layout");
};

template <int NS, bool PAIR>
__global__ void __launch_bounds__(pk_threads(PAIR), 1) k_tcp(const __grid_constant__ PackedArgs a) {
  using Ly = PLay<NS, PAIR>;
  constexpr int NSTG = Ly::NSTG, U = Ly::U;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  DevProblem* sProb = reinterpret_cast<DevProblem*>(smem + Ly::PROB);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Ly::BARS);  // this CTA's stage landed
  uint64_t* empty = full + NSTG;
  uint64_t* pfull = empty + NSTG;  // pair form, even CTA: both CTAs' stages landed
  uint64_t* acc_full = pfull + NSTG;  // [2]
  uint64_t* acc_empty = acc_full + 2;  // [2]
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + Ly::MISC);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + Ly::MISC + 4);
  constexpr int QRP = Ly::QRP;
  Item* ring = reinterpret_cast<Item*>(smem + Ly::RING);
  uint64_t* ring_full = reinterpret_cast<uint64_t*>(smem + Ly::RING + QRP * sizeof(Item));
  uint64_t* ring_empty = ring_full + QRP;
  // Tensor Memory: two accumulators and the running sums of multi-chunk
  // tiles.  One epilogue group: chunks alternate between the accumulators, so
  // that the MMAs of a chunk run while the epilogue folds the previous one,
  // and one running sum.  Two groups: each its own accumulator (all chunks of
  // its items) and its own running sum.
  constexpr uint32_t PK_COLS = 4 * BNMAX, PK_SUM = 2 * BNMAX;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < NSTG; ++s) {
      mbar_init(&full[s], 1);   // the producer's arrival, with the transaction count
      mbar_init(&empty[s], 1);  // tcgen05.commit (pair form: multicast to both CTAs)
      mbar_init(&pfull[s], 2);  // pair form: one relay arrival from each CTA
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      // pair form: the even CTA's also counts the odd CTA's epilogue threads
      mbar_init(&acc_empty[b], (PAIR ? 2 : 1) * NEPI);
    }
    mbar_init(drain, 1);
    for (int q = 0; q < QRP; ++q) {
      mbar_init(&ring_full[q], 1);
      // read by the MMA thread, the four epilogue warps and (pair form) the relay
      mbar_init(&ring_empty[q], 5 + (PAIR ? 1 : 0));
    }
    *abort = (a.gate && *a.gate == kDevBounds) ? 2 : 0;
    *sProb = a.single;
    fence_mbar_init();
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      tmem_alloc2(tmem_slot, PK_COLS);
      tmem_relinquish2();
    } else {
      tmem_alloc(tmem_slot, PK_COLS);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync();  // both CTAs' barriers exist before any remote arrival
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t crank = PAIR ? cluster_ctarank() : 0u;
  // the pair form takes work items per pair: both CTAs the same ones
  const int64_t nitems = a.nitems;
  const int64_t w0 = PAIR ? blockIdx.x / 2 : blockIdx.x, dw = PAIR ? gridDim.x / 2 : gridDim.x;
  const uint32_t a_bytes = (uint32_t)Ly::A_BYTES;
  // work item w: a tile of the single problem, or entry w of the batch's list
  // (longest first; the CTAs take them round robin)
  auto item = [&](int64_t w) {
    if (a.probs) {
      const WorkItem wi = a.items[w];
      return item_of_tile<PAIR>(a.probs + wi.prob, wi.tile, wi.split, crank);
    }
    return item_of_tile<PAIR>(sProb, w % a.tiles_single, (int)(w / a.tiles_single), crank);
  };
  // this CTA's j-th item from the ring (false at the end of its items, or on
  // a timeout); the caller releases the entry with ring_release once read
  auto ring_get = [&](int64_t j, Item& out) -> bool {
    const int q = (int)(j & (QRP - 1));
    if (!mbar_wait(&ring_full[q], (uint32_t)((j / QRP) & 1), abort)) {
      record_timeout(abort, a.err);
      return false;
    }
    out = ring[q];
    return out.d != nullptr;
  };
  auto ring_release = [&](int64_t j) { mbar_arrive(&ring_empty[j & (QRP - 1)]); };

  if (warp == 0) {
    // ---- producer: one lane streams the units of every work item ----
    if (lane == 0) {
      int64_t g = 0, g_iss = -1;
      uint32_t st_i = 0, ph = 0;  // stage and phase parity of k-tile g
      bool failed = false;
      // Items up to j + 2 are published before item j's stages are streamed:
      // an epilogue group reads one of its items ahead (to fetch its rows'
      // and columns' scatter entries) -- item j + 1 with one group, j + 2 with
      // two -- and item j's later stages reach the producer only through that
      // group's release of accumulators.  An entry with d == null ends the
      // sequence; a second one follows it, since with two groups each reads
      // every other entry.
      auto decode = [&](int64_t w) {
        Item x;
        if (w < nitems) {
          x = a.pitems ? a.pitems[w] : item(w);
        } else {
          std::memset(&x, 0, sizeof x);
        }
        return x;
      };
      // a batch's CTAs claim their items after the first from a counter
      // (items cost unevenly: their epilogues' stores differ with C's layout),
      // each claim issued one entry ahead of its use, so that its round trip
      // overlaps the streaming of the item before
      int64_t claimed = w0;
      auto next_index = [&](int64_t n) -> int64_t {
        if (!a.counter) return w0 + n * dw;
        const int64_t w = claimed;
        if (w < nitems) claimed = dw + (int64_t)atomicAdd(a.counter, 1ull);
        return w;
      };
      auto publish = [&](int64_t j, const Item& x) {
        const int q = (int)(j & (QRP - 1));
        if (!mbar_wait(&ring_empty[q], (uint32_t)(((j / QRP) & 1) ^ 1), abort)) {
          record_timeout(abort, a.err);
          return false;
        }
        ring[q] = x;
        mbar_arrive(&ring_full[q]);
        return true;
      };
      int64_t npub = 0;    // entries published
      bool ended = false;  // both end entries published
      auto publish_upto = [&](int64_t last) {
        while (!ended && npub <= last) {
          const Item x = decode(next_index(npub));
          if (!publish(npub, x)) return false;
          ++npub;
          if (x.d == nullptr) {
            if (!publish(npub, x)) return false;
            ++npub;
            ended = true;
          }
        }
        return true;
      };
      for (int64_t j = 0; !*abort && !failed; ++j) {
        if (!publish_upto(j + 2)) break;
        // item j as published (its slot is not rewritten before item j + 14)
        const Item it = ring[j & (QRP - 1)];
        if (it.d == nullptr) break;
        const DevProblem* d = it.d;
        const int64_t KT = (d->k + BK - 1) / BK;
        // pair form: B in half-tile units, this CTA's half
        const int rb = PAIR ? d->bn / 2 : d->bn;
        const uint32_t b_bytes = (uint32_t)(NS * rb * BK * 2);
        const int64_t ubi = PAIR ? (it.n0 / d->bn) * 2 + crank : it.n0 / d->bn;
        const uint8_t* ua = d->pa + ((it.m0 / BM) * KT + it.kbeg / BK) * (int64_t)a_bytes;
        const uint8_t* ub = d->pb + (ubi * KT + it.kbeg / BK) * (int64_t)b_bytes;
        for (int64_t kt = 0; kt < it.KT; kt += U, ++g) {
          const int s = (int)st_i;
          const uint32_t nu = (uint32_t)(it.KT - kt < U ? it.KT - kt : U);  // units in this stage
          if (!mbar_wait(&empty[s], ph ^ 1u, abort)) {
            record_timeout(abort, a.err);
            failed = true;
            break;
          }
          const uint32_t st = smem_u32(smem + s * Ly::STAGE);
          mbar_expect_tx(&full[s], nu * (a_bytes + b_bytes));
          bulk_load(st, ua + kt * (int64_t)a_bytes, nu * a_bytes, &full[s]);
          bulk_load(st + U * Ly::A_BYTES, ub + kt * (int64_t)b_bytes, nu * b_bytes, &full[s]);
          mbar_arrive(&full[s]);
          g_iss = g;
          if (++st_i == (uint32_t)NSTG) {
            st_i = 0;
            ph ^= 1u;
          }
        }
      }
      // no copy may outlive the CTA (matters only after an abort): only the
      // last NSTG stages can be in flight; wait for their phases (bounded)
      if (g_iss >= 0) {
        for (int64_t gi = g_iss - NSTG + 1 > 0 ? g_iss - NSTG + 1 : 0; gi <= g_iss; ++gi) {
          const long long t0 = clock64();
          while (!mbar_try_wait(&full[gi % NSTG], (uint32_t)((gi / NSTG) & 1)) &&
                 clock64() - t0 < 20000000LL) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issue: the same products, in the same order, as k_tc (pair
    // form: the even CTA issues for both; the odd one only waits, before
    // releasing Tensor Memory, for the MMAs writing it) ----
    if (lane == 0) {
      int64_t gc = 0;
      uint32_t st_i = 0, ph = 0;  // stage and phase parity of the next k-tile
      bool failed = false;
      const bool issuer = !PAIR || crank == 0;
      // matrix descriptors of stage 0; a stage's, piece's or k-slice's own
      // descriptor adds its byte offset / 16 to the start-address field
      // (shared-memory addresses stay below 256 KB: no carry out of it)
      const uint64_t descA0 = smem_desc(smem_u32(smem), (BM / 8) * 128, 128);
      if (issuer && a.fault == 1) {
        // injected failure: a bounded wait (about 10 ms) on a barrier nothing
        // arrives on yet; it expires, and the CTA unwinds through the abort path
        if (!mbar_wait(drain, 0, abort, 20000000LL)) {
          record_timeout(abort, a.err);
          failed = true;
        }
      }
      int64_t uses0 = 0, uses1 = 0;  // two groups: chunks issued into each accumulator so far
      for (int64_t j = 0; !*abort && !failed; ++j) {
        Item it;
        const bool got = ring_get(j, it);
        ring_release(j);
        if (!got) break;
        if (!issuer) continue;  // pair form, odd CTA: only keeps the ring moving
        const int bn = it.d->bn;
        const int rb = PAIR ? bn / 2 : bn;  // B rows in each CTA's stage
        const uint32_t idesc = idesc_bf16_f32(PAIR ? 2 * BM : BM, (uint32_t)bn);
        const uint32_t b_bytes = (uint32_t)(NS * rb * BK * 2);  // one unit of B
        const uint64_t descB0 =
            smem_desc(smem_u32(smem) + U * Ly::A_BYTES, (uint32_t)(rb / 8) * 128, 128);
        for (int ch = 0; ch < it.nchunks && !failed; ++ch, ++gc) {
          // one group: chunks alternate between the accumulators; two groups:
          // item j's chunks all go to accumulator j % 2, the one its group reads
          const int buf = a.dual ? (int)(j & 1) : (int)(gc & 1);
          // earlier uses of this accumulator (scalars, not an array: no local memory)
          const int64_t use = a.dual ? (buf ? uses1++ : uses0++) : gc >> 1;
          if (use > 0 &&
              !mbar_wait<PAIR>(&acc_empty[buf], (uint32_t)((use - 1) & 1), abort)) {
            record_timeout(abort, a.err);
            failed = true;
            break;
          }
          tc_fence_after();
          const uint32_t acc = tmem + (uint32_t)buf * BNMAX;
          const int64_t kt0 = (int64_t)ch * CHUNK_KT;
          const int64_t kt1 = kt0 + CHUNK_KT < it.KT ? kt0 + CHUNK_KT : it.KT;
          for (int64_t kt = kt0; kt < kt1; kt += U) {
            const int s = (int)st_i;
            const int nu = (int)(kt1 - kt < U ? kt1 - kt : U);
            if (!mbar_wait<PAIR>(PAIR ? &pfull[s] : &full[s], ph, abort)) {
              record_timeout(abort, a.err);
              failed = true;
              break;
            }
            tc_fence_after();
            const uint64_t so = (uint64_t)((s * Ly::STAGE) >> 4);
#pragma unroll
            for (int u = 0; u < U; ++u) {
              if (u >= nu) break;
#pragma unroll
            for (int ksl = 0; ksl < BK / 16; ++ksl) {
              uint64_t dA[NS], dB[NS];
#pragma unroll
              for (int i = 0; i < NS; ++i) {
                dA[i] = descA0 + so +
                        (uint64_t)((u * Ly::A_BYTES + i * BM * BK * 2 + ksl * 2 * (BM / 8) * 128) >> 4);
                dB[i] = descB0 + so +
                        (uint64_t)((u * b_bytes + i * rb * BK * 2 + ksl * 2 * (rb / 8) * 128) >> 4);
              }
              auto mma = [&](uint64_t da, uint64_t db, uint32_t accum) {
                if constexpr (PAIR) mma_bf16_ss2(acc, da, db, idesc, accum);
                else mma_bf16_ss(acc, da, db, idesc, accum);
              };
              mma(dA[0], dB[0], (kt + u > kt0 || ksl > 0) ? 1u : 0u);
#pragma unroll
              for (int ts = 1; ts < NS; ++ts)
#pragma unroll
                for (int i = 0; i <= ts; ++i) mma(dA[i], dB[ts - i], 1u);
            }
            }
            if constexpr (PAIR) mma_commit2(&empty[s], 0x3);  // both CTAs' stages
            else mma_commit(&empty[s]);
            if (++st_i == (uint32_t)NSTG) {
              st_i = 0;
              ph ^= 1u;
            }
          }
          if (failed) break;
          if (kt1 > kt0) {
            if constexpr (PAIR) mma_commit2(&acc_full[buf], 0x3);
            else mma_commit(&acc_full[buf]);
          } else if constexpr (PAIR) {  // nothing to accumulate: hand over at once
            mbar_arrive_cluster(&acc_full[buf], 0);
            mbar_arrive_cluster(&acc_full[buf], 1);
          } else {
            mbar_arrive(&acc_full[buf]);
          }
        }
      }
      // every MMA the issuer issued has completed once this commit arrives
      // (in the pair form on both CTAs' drain barriers)
      if (issuer) {
        if constexpr (PAIR) mma_commit2(drain, 0x3);
        else mma_commit(drain);
      }
      if (!mbar_wait(drain, 0, abort)) {
        const long long t0 = clock64();
        while (!mbar_try_wait(drain, 0) && clock64() - t0 < 4000000000LL) {
        }
      }
    }
  } else if (PAIR && warp == PK_RELAY_WARP) {
    // ---- relay (pair form): once this CTA's stage has landed, one arrival
    // on the even CTA's pfull for it ----
    if (lane == 0) {
      uint32_t st_i = 0, ph = 0;
      bool failed = false;
      for (int64_t j = 0; !*abort && !failed; ++j) {
        Item it;
        const bool got = ring_get(j, it);
        ring_release(j);
        if (!got) break;
        for (int64_t kt = 0; kt < it.KT; kt += U) {
          const int s = (int)st_i;
          if (!mbar_wait(&full[s], ph, abort)) {
            record_timeout(abort, a.err);
            failed = true;
            break;
          }
          mbar_arrive_cluster(&pfull[s], 0);
          if (++st_i == (uint32_t)NSTG) {
            st_i = 0;
            ph ^= 1u;
          }
        }
      }
    }
  } else if (warp < PK_EPI_W0 + 8 && (warp - PK_EPI_W0) / 4 < (a.dual ? 2 : 1)) {
    // ---- epilogue: one thread per accumulator row (as in k_tc); with two
    // groups, group g takes items g, g + 2, ... (each item one chunk, in
    // accumulator g) ----
    const int grp = (warp - PK_EPI_W0) >> 2, EG = a.dual ? 2 : 1;
    // the running sum of a multi-chunk tile: one region, or one per group
    const uint32_t psum = PK_SUM + (uint32_t)(a.dual ? grp : 0) * BNMAX;
    const int ebar = BAR_EPI + grp;
    int64_t* sRC = reinterpret_cast<int64_t*>(smem + Ly::SCAT) + grp * (BM + BNMAX);
    int64_t* sCC = sRC + BM;
    const int t = tid - (PK_EPI_W0 + 4 * grp) * 32;
    const int wq = warp & 3;
    const int row = 32 * wq + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * wq) << 16);
    constexpr int NB = BNMAX / NEPI;
    int64_t pre_r = 0, pre_c[NB];
    auto fetch_rows = [&](const Item& it) {
      pre_r = t < it.rows_a ? __ldg(it.d->sp.rC + it.m0 + t) : 0;
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        const int c = t + i * NEPI;
        pre_c[i] = c < it.rows_b ? __ldg(it.d->sp.cC + it.n0 + c) : 0;
      }
    };
    // item j from the ring, read by every lane, released once per warp
    auto get = [&](int64_t j, Item& out) {
      const bool got = ring_get(j, out);
      __syncwarp();
      if (lane == 0) ring_release(j);
      return got;
    };
    Item cur, nxt;
    bool got_cur = get(grp, cur);
    if (got_cur) fetch_rows(cur);
    int64_t gc = 0;  // chunks before this one in the CTA's sequence
    for (int64_t j = grp;; j += EG) {
      if (bar_or(ebar, NEPI, !got_cur || *abort)) break;  // uniform exit
      const Item it = cur;
      const DevProblem* d = it.d;
      sRC[t] = pre_r;
#pragma unroll
      for (int i = 0; i < NB; ++i) sCC[t + i * NEPI] = pre_c[i];
      // the next item's row and column entries are fetched one item ahead
      const bool have_next = get(j + EG, nxt);
      if (have_next) fetch_rows(nxt);
      bar_sync(ebar, NEPI);

      const bool have = it.KT > 0;
      const int bn = d->bn;
      const bool direct = d->splits == 1;
      const float al = (float)d->alpha, be = (float)d->beta;
      float* const crow = static_cast<float*>(d->c) + sRC[row];
      float* const prow = direct ? nullptr
                                 : static_cast<float*>(d->partial) +
                                       ((int64_t)it.split * d->n + it.n0) * d->m + it.m0 + row;
      const int64_t pm = d->m;
      // rows past the operand, and holes of a blocked row bundle, write nothing
      const bool mv = row < it.rows_a && sRC[row] != kHole;
      const int cols = it.rows_b;
      bool ok = true;
      auto out8 = [&](int cb, const float (&hi)[8], const float (&lo)[8]) {
        if (!mv) return;
        if (!direct) {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (cb + q < cols) prow[(int64_t)(cb + q) * pm] = __fadd_rn(hi[q], lo[q]);
        } else if (be == 0.f) {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (cb + q < cols) crow[sCC[cb + q]] = __fmaf_rn(al, hi[q], al * lo[q]);
        } else {
          float old[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) old[q] = cb + q < cols ? crow[sCC[cb + q]] : 0.f;
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (cb + q < cols)
              crow[sCC[cb + q]] = __fmaf_rn(be, old[q], __fmaf_rn(al, hi[q], al * lo[q]));
        }
      };
      for (int ch = 0; ch < it.nchunks; ++ch, ++gc) {
        const bool first = ch == 0, last = ch + 1 == it.nchunks;
        // one group: chunk gc of the CTA in accumulator gc % 2; two groups:
        // this group's gc-th chunk in accumulator grp (its own running sum too)
        const int buf = a.dual ? grp : (int)(gc & 1);
        const uint32_t use = (uint32_t)(a.dual ? gc : gc >> 1);
        if (have && !*abort) {
          if (!mbar_wait<PAIR>(&acc_full[buf], use & 1u, abort)) record_timeout(abort, a.err);
        }
        tc_fence_after();
        ok = __all_sync(0xffffffffu, !*abort);
        // a one-chunk tile is written straight from its accumulator; longer
        // ones are folded into the running sum chunk by chunk
        const bool direct_out = first && last;
        const uint32_t accc = (uint32_t)buf * BNMAX;
        if (ok && direct_out) {
          float z[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) z[q] = 0.f;
          for (int cb = 0; cb < bn; cb += 16) {
            float v[16];
            if (have) {
              tmem_ld16(lane_base + accc + (uint32_t)cb, v);
            } else {
#pragma unroll
              for (int q = 0; q < 16; ++q) v[q] = 0.f;
            }
#pragma unroll
            for (int p8 = 0; p8 < 2; ++p8) {
              float v8[8];
#pragma unroll
              for (int q = 0; q < 8; ++q) v8[q] = v[8 * p8 + q];
              out8(cb + 8 * p8, v8, z);
            }
          }
        } else if (ok) {
          for (int cb = 0; cb < bn; cb += 8) {
            float v[8], sum[8];
            if (have) {
              tmem_ld8(lane_base + accc + (uint32_t)cb, v);
            } else {
#pragma unroll
              for (int q = 0; q < 8; ++q) v[q] = 0.f;
            }
            if (first) {
#pragma unroll
              for (int q = 0; q < 8; ++q) sum[q] = v[q];
            } else {
              tmem_ld8(lane_base + psum + (uint32_t)cb, sum);
#pragma unroll
              for (int q = 0; q < 8; ++q) sum[q] = __fadd_rn(sum[q], v[q]);
            }
            tmem_st8(lane_base + psum + (uint32_t)cb, sum);
          }
          tmem_st_wait();
        }
        tc_fence_before();
        if constexpr (PAIR) mbar_arrive_cluster(&acc_empty[buf], 0);
        else mbar_arrive(&acc_empty[buf]);
        if (!ok) break;
        if (!last || direct_out) continue;
        for (int cb = 0; cb < bn; cb += 8) {
          float sum[8], z[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) z[q] = 0.f;
          tmem_ld8(lane_base + psum + (uint32_t)cb, sum);
          out8(cb, sum, z);
        }
      }
      cur = nxt;
      got_cur = have_next;
    }
  }

  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync();  // both CTAs are done with both Tensor Memories
  if (warp == 1) {
    tc_fence_after();
    if constexpr (PAIR) tmem_dealloc2(tmem, PK_COLS);
    else tmem_dealloc(tmem, PK_COLS);
  }
}

cudaError_t launch_reduce(const TcLaunch& q, cudaStream_t s);

template <int NS, bool BOX, bool PAIR>
cudaError_t launch_cfg(const TcLaunch& q, cudaStream_t s) {
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_tc<NS, BOX, PAIR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Lay<NS, BOX, PAIR>::ALLOC);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  Args a;
  a.tm[0] = q.tm[0];
  a.tm[1] = q.tm[1];
  a.single = q.single;
  a.probs = q.probs;
  a.items = q.items;
  a.err = q.err;
  a.fault = q.fault;
  a.counter = q.probs && !BOX ? q.counter : nullptr;
  a.gate = q.gate;
  // a single problem whose every work item is one accumulation chunk
  a.dbuf = !q.probs && q.single.kps <= (int64_t)CHUNK_KT * BK ? 1 : 0;
  if (q.probs) {
    a.nitems = q.nitems;
    a.tiles_single = 1;
  } else {
    const int64_t rows = PAIR ? 2 * BM : BM;  // the pair form's tiles have 256 rows
    a.tiles_single = ((q.single.m + rows - 1) / rows) * q.single.tiles_n;
    a.nitems = a.tiles_single * q.single.splits;
  }
  if (a.nitems == 0) return cudaSuccess;
  // dynamic items count from zero in every launch (a memset node under capture)
  if (a.counter && cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), s) != cudaSuccess)
    return cudaGetLastError();
  mainloop_event_before(s);
  if constexpr (PAIR) {
    // clusters of two CTAs, one pair per work item at a time
    const int64_t pairs = std::max<int64_t>(1, std::min<int64_t>(q.ctas / 2, a.nitems));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * pairs), 1, 1);
    cfg.blockDim = dim3(nthreads(BOX), 1, 1);
    cfg.dynamicSmemBytes = Lay<NS, BOX, PAIR>::ALLOC;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_tc<NS, BOX, PAIR>, a);
    if (e != cudaSuccess) return e;
  } else {
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(q.ctas, a.nitems));
    k_tc<NS, BOX, PAIR><<<(unsigned)grid, nthreads(BOX), Lay<NS, BOX, PAIR>::ALLOC, s>>>(a);
  }
  note_launch();
  const cudaError_t e = launch_reduce(q, s);
  mainloop_event_after(s);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// K4 after the mainloop: the single problem's k-splits, or every split
// problem of a batch.
cudaError_t launch_reduce(const TcLaunch& q, cudaStream_t s) {
  const bool single_split = !q.probs && q.single.splits > 1;
  if (single_split || (q.probs && q.n_split_probs > 0)) {
    const int64_t mm = single_split ? q.single.m : q.max_m_split;
    const int64_t nn = single_split ? q.single.n : q.max_n_split;
    const unsigned bx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((mm + 255) / 256, 16));
    const unsigned by = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(single_split ? nn : q.split_cols, single_split ? 8192 : 16384));
    if (q.reduce_f64)
      k_reduce_partials<true><<<dim3(bx, by), 256, 0, s>>>(q.single, q.probs, q.split_probs,
                                                           q.split_col_prefix,
                                                           single_split ? 0 : q.n_split_probs,
                                                           q.gate);
    else
      k_reduce_partials<false><<<dim3(bx, by), 256, 0, s>>>(q.single, q.probs, q.split_probs,
                                                            q.split_col_prefix,
                                                            single_split ? 0 : q.n_split_probs,
                                                            q.gate);
    note_launch();
  }
  return cudaGetLastError();
}

// A's row units: 128 rows each; the pair form pads them to whole 256-row tiles.
int64_t pack_a_units(int64_t m, bool pair) { return pair ? 2 * ((m + 2 * BM - 1) / (2 * BM)) : (m + BM - 1) / BM; }

size_t pack_a_bytes(int64_t m, int64_t k, int pieces, bool pair) {
  return align_up((size_t)pack_a_units(m, pair) * (size_t)((k + BK - 1) / BK) * pieces * BM * BK * 2,
                  256);
}

template <int NS, bool PAIR>
cudaError_t launch_packed(const TcLaunch& q, cudaStream_t s) {
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_tcp<NS, PAIR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         PLay<NS, PAIR>::ALLOC);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  PackLaunch pk;
  std::memset(&pk, 0, sizeof pk);
  pk.gate = q.gate;
  PackedArgs a;
  std::memset(&a, 0, sizeof a);
  a.single = q.single;
  if (q.probs) {
    pk.jobs = q.pack_jobs;
    pk.prefix = q.pack_prefix;
    pk.njobs = q.pack_njobs;
    pk.total = q.pack_groups;
    pk.claim = q.counter;
    a.probs = q.probs;
    a.items = q.items;
    a.nitems = q.nitems;
    a.tiles_single = 1;
  } else {
    DevProblem& d = a.single;
    const int64_t KT = (d.k + BK - 1) / BK;
    const int64_t tm = pack_a_units(d.m, PAIR), tn = d.tiles_n;
    if (KT == 0 || tm == 0 || tn == 0) return cudaSuccess;
    d.pa = static_cast<const uint8_t*>(q.pack_ws);
    d.pb = d.pa + pack_a_bytes(d.m, d.k, NS, PAIR);
    PackJob& ja = pk.local[0];
    ja.x = static_cast<const float*>(d.a);
    ja.rs = d.sp.rA;
    ja.ks = d.sp.cA;
    ja.kbs = d.sp.cbsA;
    ja.rows = d.m;
    ja.k = d.k;
    ja.R = BM;
    ja.KT = KT;
    ja.units = tm * KT;
    ja.swz = d.rows_blocked ? 16 : 0;
    ja.out = const_cast<uint8_t*>(d.pa);
    PackJob& jb = pk.local[1];
    jb = ja;
    jb.x = static_cast<const float*>(d.b);
    jb.rs = d.sp.cB;
    jb.ks = d.sp.rB;
    jb.kbs = d.sp.rbsB;
    jb.rows = d.n;
    jb.swz = 0;
    jb.R = PAIR ? d.bn / 2 : d.bn;  // pair form: half-tile units, one per CTA
    jb.units = (PAIR ? 2 : 1) * tn * KT;
    jb.out = const_cast<uint8_t*>(d.pb);
    pack_job_groups(ja);
    pack_job_groups(jb);
    pk.local_prefix[1] = ja.groups;
    pk.local_prefix[2] = pk.total = ja.groups + jb.groups;
    a.tiles_single = (PAIR ? tm / 2 : tm) * tn;
    a.nitems = a.tiles_single * d.splits;
  }
  if (a.nitems == 0) return cudaSuccess;
  a.err = q.err;
  a.gate = q.gate;
  a.fault = q.fault;
  // two epilogue groups that take the items in turn: for a batch (short
  // items, most of them one chunk), and for a single problem whose items are
  // one chunk each; a single problem of long items keeps one group, whose
  // chunks alternate between the accumulators (the MMAs of a chunk then run
  // while the previous chunk is folded)
  a.dual = q.probs ? 1 : (q.single.kps <= (int64_t)CHUNK_KT * BK ? 1 : 0);
  a.counter = q.probs && !PAIR ? q.counter + 1 : nullptr;
  a.pitems = q.probs && !PAIR ? static_cast<const Item*>(q.pack_items) : nullptr;
  mainloop_event_before(s);
  if (q.probs) {
    // the claim counters of the packing launch and of the mainloop
    if (!q.counter) return cudaErrorInvalidValue;
    const cudaError_t e = cudaMemsetAsync(q.counter, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
  }
  if (pk.total > 0) {
    // a batch: one wave, as many CTAs as the SMs hold at once, claiming
    // about 16 runs each; a single contraction: eight CTAs per SM
    static int resident = 0;
    if (resident == 0) {
      int r = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_pack<NS>, 256, 0) != cudaSuccess || r <= 0) {
        cudaGetLastError();
        r = 4;
      }
      resident = r;
    }
    int64_t grid = std::min<int64_t>(pk.total, (int64_t)q.ctas * 8);
    if (q.probs) {
      grid = std::min<int64_t>(pk.total, (int64_t)q.ctas * resident);
      pk.chunk = std::max<int64_t>(1, pk.total / (grid * 16));
    }
    k_pack<NS><<<(unsigned)grid, 256, 0, s>>>(pk);
    note_launch();
  }
  if constexpr (PAIR) {
    // clusters of two CTAs, one pair per work item at a time
    const int64_t pairs = std::max<int64_t>(1, std::min<int64_t>(q.ctas / 2, a.nitems));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * pairs), 1, 1);
    cfg.blockDim = dim3(pk_threads(true), 1, 1);
    cfg.dynamicSmemBytes = PLay<NS, true>::ALLOC;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_tcp<NS, true>, a);
    if (e != cudaSuccess) return e;
  } else {
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(q.ctas, a.nitems));
    k_tcp<NS, false><<<(unsigned)grid, pk_threads(false), PLay<NS, false>::ALLOC, s>>>(a);
  }
  note_launch();
  const cudaError_t e = launch_reduce(q, s);
  mainloop_event_after(s);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Packed batches: each work item decoded once, at plan creation (the
// producer of k_tcp then loads it instead of decoding it from the work list
// and the problem's descriptor, two dependent round trips per item).
__global__ void k_decode_items(const DevProblem* probs, const WorkItem* items, int64_t n, Item* out) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < n;
       w += (int64_t)gridDim.x * blockDim.x) {
    const WorkItem wi = items[w];
    out[w] = item_of_tile<false>(probs + wi.prob, wi.tile, wi.split);
  }
}

}  // namespace

int tc_bn_max() { return BNMAX; }
size_t tc_item_bytes() { return sizeof(Item); }
cudaError_t launch_decode_items(const DevProblem* probs, const WorkItem* items, int64_t n, void* out,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t grid = std::min<int64_t>((n + 255) / 256, 1024);
  k_decode_items<<<(unsigned)grid, 256, 0, s>>>(probs, items, n, static_cast<Item*>(out));
  note_launch();
  return cudaGetLastError();
}
size_t tc_pack_bytes(int64_t m, int64_t n, int64_t k, int bn, int pieces, bool pair) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  const size_t b = (size_t)((n + bn - 1) / bn) * (size_t)((k + BK - 1) / BK) * pieces * bn * BK * 2;
  return pack_a_bytes(m, k, pieces, pair) + align_up(b, 256);
}
int tc_max_item_ktiles() { return MAX_CHUNKS * CHUNK_KT; }

cudaError_t launch_tc(const TcLaunch& q, cudaStream_t s) {
  // boxes only when every work item has both operands as boxes (the planner
  // sets both or neither; batch plans set neither); the pair form only with
  // boxes planned for it (B boxes half the tile wide)
  if (q.probs ? q.pack_jobs != nullptr : q.pack_ws != nullptr) {
    const bool pp = !q.probs && q.single.pair;  // batches: single CTAs
    if (q.pieces == 3) return pp ? launch_packed<3, true>(q, s) : launch_packed<3, false>(q, s);
    return pp ? launch_packed<2, true>(q, s) : launch_packed<2, false>(q, s);
  }
  const bool box = !q.probs && q.single.boxA.rank > 0 && q.single.boxB.rank > 0;
  const bool pair = box && q.single.pair;
  if (q.pieces == 3)
    return pair ? launch_cfg<3, true, true>(q, s)
                : box ? launch_cfg<3, true, false>(q, s) : launch_cfg<3, false, false>(q, s);
  return pair ? launch_cfg<2, true, true>(q, s)
              : box ? launch_cfg<2, true, false>(q, s) : launch_cfg<2, false, false>(q, s);
}

}  // namespace tc
