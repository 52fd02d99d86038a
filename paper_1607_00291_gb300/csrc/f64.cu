// K2 + K5: FP64 mainloop over the block-scatter-matrix view, with the scattered
// alpha/beta epilogue fused in.
//
// The matrix product C_{IJ} = A_{IP} B_{PJ} of Section 4 is tiled into
// BM x BN output tiles (Section 6.1: partitioning a scatter-matrix is slicing
// its scatter vectors).  Each CTA gathers its A and B panels straight from the
// tensors through rscat/cscat (Section 6.1's packing kernel, here a register-
// staged global->shared gather, coalesced along each operand's own unit-stride
// index), multiplies them on the FP64 tensor pipe (DMMA, mma.sync m8n8k4 f64),
// and updates C through rscat(C) + cscat(C) (Section 6.1's scattered
// micro-tile update), reading C only when beta != 0.
//
// Scheduling: plain tiling when the tiles fill whole waves of CTAs, else a
// stream-K split of the (tile, k-tile) iteration space over one CTA per SM
// with a deterministic FP64 fix-up of the cut tiles.
//
// GB300 has no tcgen05 kind for FP64, and its FP64 rate (DMMA ~= DFMA) is low
// enough that a register-blocked warp-level DMMA tile keeps the pipe saturated;
// global traffic is far below HBM bandwidth at every tile size used here.
#include <algorithm>

#include "kernels.h"

namespace tc {
namespace {

constexpr int BK = 16;

// A BM_ x BN_ output tile computed by (BM_/32) x (BN_/32) warps of 32 x 32.
// The single-contraction kernels use 128 x 64 (one 256-thread CTA per SM);
// batches choose per problem among 64 x 64, 32 x 64 and 64 x 32 (eight warps
// per SM in every case): the problems of a batch are small, and the tile that
// pads a problem least wastes the fewest FP64 operations.  (32 x 32 would pad
// the 512-problem workload 1 % less, but a one-warp CTA spills registers.)
template <int BM_, int BN_>
struct FT {
  static constexpr int BM = BM_, BN = BN_;
  static constexpr int WN = BN / 32;                       // warps along n
  static constexpr int NT = (BM / 32) * WN * 32;           // threads
  static constexpr int LDA = BM + 8, LDB = BN + 8;  // row pitch (doubles); rows 64 B apart in banks
  static constexpr int A_PER_T = BM * BK / NT;
  static constexpr int B_PER_T = BN * BK / NT;
  static constexpr size_t SMEM = (size_t)(2 * BK * LDA + 2 * BK * LDB) * sizeof(double) +
                                 (size_t)(2 * BM + 2 * BN) * sizeof(int64_t);
  static_assert(BM % 32 == 0 && BN % 32 == 0 && (BM * BK) % NT == 0 && (BN * BK) % NT == 0,
                "tile shape");
};
using F1 = FT<128, 64>;  // single contractions
constexpr int BM = F1::BM, BN = F1::BN, NT = F1::NT;
constexpr size_t kSmem = F1::SMEM;

// Checked launches: the whole CTA skips its work when the device error word
// (`gate`) holds a bounds error from the scatter-vector check (thread 0 reads
// it once, so the CTA takes one decision).
__device__ __forceinline__ bool gate_closed(const int32_t* gate) {
  __shared__ int s_closed;
  if (threadIdx.x == 0) s_closed = *gate == kDevBounds;
  __syncthreads();
  return s_closed != 0;
}

__device__ __forceinline__ void dmma(double (&d)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d[0]), "+d"(d[1])
               : "d"(a), "d"(b));
}

// Work split (stream-K): the T = tiles * KT (tile, k-tile) iterations are cut
// into G equal contiguous ranges, one per CTA.  CTA c walks its range tile by
// tile; a tile it covers whole is finished in place (fused epilogue), a tile
// cut by a range boundary leaves FP64 partial sums in one of the CTA's two
// slots (slot 0: the segment at the start of its range, slot 1: the segment at
// its end), and k_f64_fixup adds them up in k order and applies the epilogue.
// With G = tiles every range is exactly one tile (plain data-parallel tiling).
struct SkArgs {
  int64_t tiles, tiles_n, KT;
  int64_t G;
  double* partial;  // [G][2][BM*BN], element (mm, nn) at nn*BM + mm
};

__host__ __device__ __forceinline__ int64_t sk_start(int64_t c, int64_t T, int64_t G) {
  return (int64_t)(((__int128)c * T) / G);
}

template <typename T>
struct F64Ctx {
  const T* a;
  const T* b;
  T* c;
  ScatterPtrs sp;
  int64_t M, N, K;
  double alpha, beta;
  int a_kc, b_kc;
};

struct F64Smem {
  double* As;   // [2][BK][LDA]
  double* Bs;   // [2][BK][LDB]
  int64_t *sRA, *sRC, *sCB, *sCC;
};

template <class F>
__device__ __forceinline__ F64Smem f64_smem(unsigned char* smem) {
  F64Smem S;
  S.As = reinterpret_cast<double*>(smem);
  S.Bs = S.As + 2 * BK * F::LDA;
  S.sRA = reinterpret_cast<int64_t*>(S.Bs + 2 * BK * F::LDB);
  S.sRC = S.sRA + F::BM;
  S.sCB = S.sRC + F::BM;
  S.sCC = S.sCB + F::BN;
  return S;
}

// One BM x BN output tile at (m0, n0) over k-tiles [kb, ke) (possibly empty).
// direct: apply the epilogue to C.  Otherwise store the raw FP64 sums at
// part[nn * ldp + mm] for the tile-local (mm, nn) -- only inside the operand
// when `bounded`.  All threads of the CTA call it together.
template <typename T, class F>
__device__ __forceinline__ void f64_tile(const F64Ctx<T>& P, const F64Smem& S, int64_t m0,
                                         int64_t n0, int64_t kb, int64_t ke, bool direct,
                                         double* part, int64_t ldp, bool bounded) {
  constexpr int BM = F::BM, BN = F::BN, NT = F::NT, LDA = F::LDA, LDB = F::LDB;
  constexpr int A_PER_T = F::A_PER_T, B_PER_T = F::B_PER_T;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, tig = lane & 3;
  const int wm = warp / F::WN, wn = warp % F::WN;
  const int64_t M = P.M, N = P.N, K = P.K;

  // element e of a panel -> (row, k) with consecutive threads along the
  // operand's unit-stride index
  auto a_coord = [&](int e, int& mm, int& kk) {
    if (P.a_kc) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
  };
  auto b_coord = [&](int e, int& nn, int& kk) {
    if (P.b_kc) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
  };

  __syncthreads();  // the previous tile's epilogue is done with the row tables
  for (int i = tid; i < BM; i += NT) {
    const int64_t gm = m0 + i;
    S.sRA[i] = gm < M ? P.sp.rA[gm] : 0;
    S.sRC[i] = gm < M ? P.sp.rC[gm] : 0;
  }
  for (int i = tid; i < BN; i += NT) {
    const int64_t gn = n0 + i;
    S.sCB[i] = gn < N ? P.sp.cB[gn] : 0;
    S.sCC[i] = gn < N ? P.sp.cC[gn] : 0;
  }
  __syncthreads();

  double acc[4][4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

  double ra[A_PER_T], rb[B_PER_T];
  auto load = [&](int64_t kt) {
    const int64_t k0 = kt * BK;
#pragma unroll
    for (int i = 0; i < A_PER_T; ++i) {
      int mm, kk;
      a_coord(tid + i * NT, mm, kk);
      const int64_t gm = m0 + mm, gk = k0 + kk;
      ra[i] = (gm < M && gk < K) ? (double)P.a[S.sRA[mm] + P.sp.cA[gk]] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < B_PER_T; ++i) {
      int nn, kk;
      b_coord(tid + i * NT, nn, kk);
      const int64_t gn = n0 + nn, gk = k0 + kk;
      rb[i] = (gn < N && gk < K) ? (double)P.b[P.sp.rB[gk] + S.sCB[nn]] : 0.0;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int i = 0; i < A_PER_T; ++i) {
      int mm, kk;
      a_coord(tid + i * NT, mm, kk);
      S.As[(buf * BK + kk) * LDA + mm] = ra[i];
    }
#pragma unroll
    for (int i = 0; i < B_PER_T; ++i) {
      int nn, kk;
      b_coord(tid + i * NT, nn, kk);
      S.Bs[(buf * BK + kk) * LDB + nn] = rb[i];
    }
  };

  if (kb < ke) {
    load(kb);
    store(0);
  }
  __syncthreads();
  for (int64_t kt = kb; kt < ke; ++kt) {
    const int buf = (int)((kt - kb) & 1);
    if (kt + 1 < ke) load(kt + 1);
    const double* Ab = S.As + buf * BK * LDA + wm * 32 + g;
    const double* Bb = S.Bs + buf * BK * LDB + wn * 32 + g;
#pragma unroll
    for (int kk = 0; kk < BK; kk += 4) {
      double af[4], bf[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) af[i] = Ab[(kk + tig) * LDA + i * 8];
#pragma unroll
      for (int j = 0; j < 4; ++j) bf[j] = Bb[(kk + tig) * LDB + j * 8];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) dmma(acc[i][j], af[i], bf[j]);
    }
    if (kt + 1 < ke) store(buf ^ 1);
    __syncthreads();
  }

  if (direct) {
    // K5: scattered epilogue, C[rscat + cscat] = alpha * acc + beta * C
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int mm = wm * 32 + i * 8 + g, nn = wn * 32 + j * 8 + 2 * tig + q;
          if (m0 + mm < M && n0 + nn < N) {
            T* p = P.c + S.sRC[mm] + S.sCC[nn];
            double v = P.alpha * acc[i][j][q];
            if (P.beta != 0.0) v += P.beta * (double)*p;
            *p = (T)v;
          }
        }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int mm = wm * 32 + i * 8 + g, nn = wn * 32 + j * 8 + 2 * tig + q;
          if (!bounded || (m0 + mm < M && n0 + nn < N)) part[nn * ldp + mm] = acc[i][j][q];
        }
  }
}

template <typename T>
__global__ void __launch_bounds__(NT, 1)
    k_f64(const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ c, const ScatterPtrs sp,
          const int64_t M, const int64_t N, const int64_t K, const double alpha, const double beta,
          const int a_kc, const int b_kc, const SkArgs sk, const int32_t* gate) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (gate && gate_closed(gate)) return;
  const F64Smem S = f64_smem<F1>(smem);
  F64Ctx<T> P{a, b, c, sp, M, N, K, alpha, beta, a_kc, b_kc};
  const int64_t Tt = sk.tiles * sk.KT;
  const int64_t start = sk_start(blockIdx.x, Tt, sk.G), end = sk_start(blockIdx.x + 1, Tt, sk.G);
  for (int64_t it = start; it < end;) {
    const int64_t tile = it / sk.KT;
    const int64_t kb = it - tile * sk.KT;
    const int64_t ke = (end - tile * sk.KT) < sk.KT ? (end - tile * sk.KT) : sk.KT;
    const int64_t m0 = (tile / sk.tiles_n) * BM, n0 = (tile % sk.tiles_n) * BN;
    const bool whole = kb == 0 && ke == sk.KT;
    double* slot = sk.partial + ((int64_t)blockIdx.x * 2 + (it == start ? 0 : 1)) * (BM * BN);
    f64_tile<T, F1>(P, S, m0, n0, kb, ke, whole, slot, BM, false);
    it = tile * sk.KT + ke;
  }
}

// Batched FP64 contractions: a persistent grid walks the work list (output
// tile x k-split of every problem, longest first): CTA b starts with item b
// and then claims the next unclaimed item from `counter` (zero at launch).
// Unsplit tiles finish in place; split ones leave FP64 partials in
// [split][n][m] for k_f64_batched_reduce.
template <int BM_, int BN_>
struct FBatch {
  using F = FT<BM_, BN_>;
  static constexpr int CTAS_PER_SM = 8 / (F::NT / 32);  // eight warps per SM
};

template <typename T, class FBt>
__global__ void __launch_bounds__(FBt::F::NT, FBt::CTAS_PER_SM)
    k_f64_batched(const DevProblem* __restrict__ probs, const WorkItem* __restrict__ items,
                  int64_t nitems, unsigned long long* __restrict__ counter,
                  const int32_t* gate) {
  using FB = typename FBt::F;
  constexpr int BM = FB::BM, BN = FB::BN;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int64_t next_w;
  if (gate && gate_closed(gate)) return;
  const F64Smem S = f64_smem<FB>(smem);
  for (int64_t w = blockIdx.x; w < nitems;) {
    const WorkItem wi = items[w];
    const DevProblem& d = probs[wi.prob];
    F64Ctx<T> P{static_cast<const T*>(d.a), static_cast<const T*>(d.b), static_cast<T*>(d.c),
                d.sp, d.m, d.n, d.k, d.alpha, d.beta, d.a_kc, d.b_kc};
    const int64_t m0 = (int64_t)(wi.tile / d.tiles_n) * BM, n0 = (int64_t)(wi.tile % d.tiles_n) * BN;
    const int64_t KT = (d.k + BK - 1) / BK, kpt = d.kps / BK;
    const int64_t kb = (int64_t)wi.split * kpt;
    const int64_t ke = kb + kpt < KT ? kb + kpt : KT;
    double* part = d.splits > 1 ? static_cast<double*>(d.partial) +
                                      (int64_t)wi.split * d.m * d.n + n0 * d.m + m0
                                : nullptr;
    f64_tile<T, FB>(P, S, m0, n0, kb, ke, d.splits == 1, part, d.m, true);
    __syncthreads();  // every thread has read next_w of the previous claim
    if (threadIdx.x == 0) next_w = (int64_t)gridDim.x + (int64_t)atomicAdd(counter, 1ull);
    __syncthreads();
    w = next_w;
  }
}

template <typename T>
__global__ void k_f64_batched_reduce(const DevProblem* __restrict__ probs,
                                     const int32_t* __restrict__ split_probs,
                                     const int64_t* __restrict__ col_prefix, int32_t n_split,
                                     const int32_t* __restrict__ gate) {
  if (gate && *gate == kDevBounds) return;
  const int64_t total = col_prefix[n_split];
  for (int64_t r = blockIdx.y; r < total; r += gridDim.y) {
    int lo = 0, hi = n_split;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (col_prefix[mid] <= r) lo = mid; else hi = mid;
    }
    const DevProblem& d = probs[split_probs[lo]];
    const int64_t n = r - col_prefix[lo];
    const int64_t M = d.m, plane = M * d.n;
    const double* part = static_cast<const double*>(d.partial);
    T* c = static_cast<T*>(d.c);
    const int64_t cn = d.sp.cC[n];
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
      double s = 0.0;
      for (int ks = 0; ks < d.splits; ++ks) s += part[ks * plane + n * M + m];
      T* p = c + d.sp.rC[m] + cn;
      double v = d.alpha * s;
      if (d.beta != 0.0) v += d.beta * (double)*p;
      *p = (T)v;
    }
  }
}

// CTA f handles the tile cut by the boundary between ranges f and f+1, if that
// boundary lies inside a tile and is the first boundary inside it.
template <typename T>
__global__ void __launch_bounds__(NT)
    k_f64_fixup(T* __restrict__ c, const ScatterPtrs sp, const int64_t M, const int64_t N,
                const double alpha, const double beta, const SkArgs sk, const int32_t* gate) {
  if (gate && *gate == kDevBounds) return;
  const int64_t Tt = sk.tiles * sk.KT;
  const int64_t f = blockIdx.x;
  if (f + 1 >= sk.G) return;
  const int64_t bnd = sk_start(f + 1, Tt, sk.G);
  if (bnd % sk.KT == 0) return;
  const int64_t tile = bnd / sk.KT;
  const int64_t t0 = tile * sk.KT, t1 = t0 + sk.KT;
  if (sk_start(f, Tt, sk.G) > t0) return;  // an earlier boundary inside this tile owns it
  // contributing CTAs: f (holding the start of the tile) up to the one holding t1 - 1
  int64_t clast = f + 1;
  while (clast + 1 < sk.G && sk_start(clast + 1, Tt, sk.G) < t1) ++clast;
  const int64_t m0 = (tile / sk.tiles_n) * BM, n0 = (tile % sk.tiles_n) * BN;
  for (int e = threadIdx.x; e < BM * BN; e += NT) {
    const int mm = e % BM, nn = e / BM;
    if (m0 + mm >= M || n0 + nn >= N) continue;
    double s = 0.0;
    for (int64_t cc = f; cc <= clast; ++cc) {
      const int slot = sk_start(cc, Tt, sk.G) >= t0 ? 0 : 1;
      s += sk.partial[(cc * 2 + slot) * (BM * BN) + e];
    }
    T* p = c + sp.rC[m0 + mm] + sp.cC[n0 + nn];
    double v = alpha * s;
    if (beta != 0.0) v += beta * (double)*p;
    *p = (T)v;
  }
}

template <typename T>
cudaError_t launch_t(const F64Launch& p, cudaStream_t s) {
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_f64<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmem);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const int64_t tm = (p.m + BM - 1) / BM, tn = (p.n + BN - 1) / BN;
  SkArgs sk;
  sk.tiles = tm * tn;
  sk.tiles_n = tn;
  sk.KT = (p.k + BK - 1) / BK;
  sk.partial = p.partial;
  sk.G = f64_grid(p.m, p.n, p.k, p.max_ctas, p.partial != nullptr);
  if (sk.tiles == 0 || sk.KT == 0) return cudaSuccess;
  if (sk.G > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  mainloop_event_before(s);
  k_f64<T><<<(unsigned)sk.G, NT, kSmem, s>>>((const T*)p.a, (const T*)p.b, (T*)p.c, p.sp, p.m,
                                              p.n, p.k, p.alpha, p.beta, p.a_k_contig,
                                              p.b_k_contig, sk, p.gate);
  note_launch();
  if (sk.G != sk.tiles) {
    k_f64_fixup<T><<<(unsigned)sk.G, NT, 0, s>>>((T*)p.c, p.sp, p.m, p.n, p.alpha, p.beta, sk,
                                                 p.gate);
    note_launch();
  }
  mainloop_event_after(s);
  return cudaGetLastError();
}

using FB0 = FBatch<64, 64>;
using FB1 = FBatch<32, 64>;
using FB2 = FBatch<64, 32>;

// One tile class's persistent launch over its slice of the work list.
template <typename T, class FBt>
cudaError_t launch_class(const F64BatchLaunch& q, int cls, cudaStream_t s) {
  using F = typename FBt::F;
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_f64_batched<T, FBt>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F::SMEM);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const int64_t n = q.class_off[cls + 1] - q.class_off[cls];
  if (n <= 0) return cudaSuccess;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(q.sms * FBt::CTAS_PER_SM, n));
  k_f64_batched<T, FBt><<<(unsigned)grid, F::NT, F::SMEM, s>>>(q.probs, q.items + q.class_off[cls],
                                                               n, q.counter + cls, q.gate);
  note_launch();
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_batched_t(const F64BatchLaunch& q, cudaStream_t s) {
  if (q.nitems > 0) {
    if (!q.counter) return cudaErrorInvalidValue;
    // the work counters start from zero in every launch (a memset node under capture)
    if (cudaMemsetAsync(q.counter, 0, sizeof(unsigned long long) * kF64BatchClasses, s) !=
        cudaSuccess)
      return cudaGetLastError();
    mainloop_event_before(s);
    cudaError_t e;
    if ((e = launch_class<T, FB0>(q, 0, s)) != cudaSuccess) return e;
    if ((e = launch_class<T, FB1>(q, 1, s)) != cudaSuccess) return e;
    if ((e = launch_class<T, FB2>(q, 2, s)) != cudaSuccess) return e;
    if (q.n_split_probs > 0) {
      const unsigned bx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((q.max_m_split + 255) / 256, 16));
      const unsigned by = (unsigned)std::max<int64_t>(1, std::min<int64_t>(q.split_cols, 16384));
      k_f64_batched_reduce<T><<<dim3(bx, by), 256, 0, s>>>(q.probs, q.split_probs,
                                                           q.split_col_prefix, q.n_split_probs,
                                                           q.gate);
      note_launch();
    }
    mainloop_event_after(s);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_f64_batched(const F64BatchLaunch& q, cudaStream_t s) {
  return q.dtype == TC_F64 ? launch_batched_t<double>(q, s) : launch_batched_t<float>(q, s);
}

int f64_tile_m() { return BM; }
int f64_tile_n() { return BN; }
int f64_tile_k() { return BK; }
void f64_batch_tile(int cls, int* bm, int* bn) {
  static const int t[kF64BatchClasses][2] = {
      {FB0::F::BM, FB0::F::BN}, {FB1::F::BM, FB1::F::BN}, {FB2::F::BM, FB2::F::BN}};
  *bm = t[cls][0];
  *bn = t[cls][1];
}
int f64_batch_ctas_per_sm(int cls) {
  static const int c[kF64BatchClasses] = {FB0::CTAS_PER_SM, FB1::CTAS_PER_SM,
                                          FB2::CTAS_PER_SM};
  return c[cls];
}

// CTAs for the FP64 mainloop: plain tiling (one CTA per tile) when the tiles
// fill whole waves of `max_ctas` (or no partial workspace is available),
// otherwise stream-K over max_ctas CTAs, each taking at least 4 k-tiles.
int64_t f64_grid(int64_t m, int64_t n, int64_t k, int64_t max_ctas, bool can_split) {
  const int64_t tiles = ((m + BM - 1) / BM) * ((n + BN - 1) / BN);
  const int64_t KT = (k + BK - 1) / BK;
  if (!can_split || max_ctas <= 0 || tiles == 0 || KT == 0) return tiles;
  const int64_t waves = (tiles + max_ctas - 1) / max_ctas;
  if ((double)tiles / (double)(waves * max_ctas) >= 0.99) return tiles;
  int64_t G = std::min<int64_t>(max_ctas, std::max<int64_t>(1, tiles * KT / 4));
  return std::max<int64_t>(G, 1);
}

size_t f64_partial_bytes(int64_t max_ctas) { return (size_t)max_ctas * 2 * BM * BN * sizeof(double); }

cudaError_t launch_f64(const F64Launch& p, cudaStream_t s) {
  return p.dtype == TC_F64 ? launch_t<double>(p, s) : launch_t<float>(p, s);
}

}  // namespace tc
