// K6 + K7: batches of contractions in one persistent launch, with a tile and
// split-K autotuner.
//
// A plan validates and lays out every problem (Sections 4 and 7.3), chooses
// per problem the tile shape and the split of the contracted range (from the
// autotune table when TC_AUTOTUNE=1, else from the same rules as a single
// call), builds one work list -- every output tile x k-split of every
// problem, longest first -- and copies the problem descriptors, the work list
// and the scatter-vector layouts into one device buffer it owns.  The
// persistent CTAs take the items in that order from a shared counter, so that
// a CTA that drew cheap items (short k, coalesced operands) takes more.
// tc_plan_execute then only launches work: the batched scatter builder (K1
// for every problem), a reset of the work counter, the persistent mainloop
// (FP64: DMMA tiles; FP32: tcgen05 tiles) and, for problems split along k,
// the reduction -- no host synchronisation and no allocation, so it can be
// captured in a CUDA graph.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "host_common.h"
#include "kernels.h"

using namespace tc;

namespace {

struct ProbCfg {
  int bn = 0;        // tile width (n)
  int bm = 128;      // tile height (m)
  int cls = 0;       // FP64: tile class (f64_batch_tile)
  int splits = 1;
  int64_t kps = 0;   // k per split
  int64_t tiles = 0;
};

// ---- K7: autotuner ------------------------------------------------------------------------
// Two decisions of a batch plan are timed rather than estimated.
//  (1) Per shape class -- mode, rounded log2 of m, n and k, the two access
//      flags -- the output tile: on the tensor cores the tile width (the one
//      covering n up to 128, and half of it); on the FP64 path the tile class
//      (64 x 64, 32 x 64, 64 x 32).  Each candidate runs the class's first
//      problem of the batch into a scratch copy of its output; the least
//      time wins.  In a batch the other problems keep the other SMs busy, so
//      what one problem costs in SM-time is what to minimise: the tensor-core
//      candidates run on one persistent CTA (one SM), the FP64 ones as many
//      copies of the problem's tiles as fill four waves of the whole GPU's
//      CTAs of that tile class (time per copy).
//  (2) Per batch -- a signature of its problems' shapes and layout classes --
//      the split of long contracted ranges: a problem is split along k until
//      no work item exceeds 1/D of a CTA's (FP64: a warp's) fair share of the
//      batch, and D is chosen among 2, 4, 8 and 16 by running the whole batch
//      with each into scratch outputs (CUDA events, best of two).  A split's
//      benefit is balance across the SMs, which only the whole batch shows.
// Results are kept for the process and, when TC_AUTOTUNE_CACHE names a file,
// read from it and written back (one record per line).  Tuning is on when
// TC_AUTOTUNE=1, or when TC_AUTOTUNE_CACHE is set and TC_AUTOTUNE is not 0;
// otherwise the plan uses the estimates (least padding, D = 4).  Tile timing
// within one tc_plan_create stops after about two seconds (the remaining
// classes keep the estimate and are tuned by a later plan).
struct TuneKey {
  int mode, lm, ln, lk, akc, bkc;
  bool operator<(const TuneKey& o) const {
    return std::memcmp(this, &o, sizeof o) < 0;
  }
};

std::mutex g_tune_mu;
std::map<TuneKey, int> g_tile;          // tensor cores: tile width; FP64: tile class
std::map<uint64_t, int> g_balance;      // batch signature -> D
bool g_tune_loaded = false;
std::string g_tune_path;  // the cache file the tables were read from ("" for none)
thread_local double t_tile_budget_ms = 0.0;  // tile timing left to this tc_plan_create
constexpr double kTileTuneBudgetMs = 2000.0;
constexpr int kBalanceCandidates[] = {2, 4, 8, 16};
constexpr int kBalanceDefault = 4;

int ilog2r(int64_t x) { return x <= 1 ? 0 : (int)std::lround(std::log2((double)x)); }

TuneKey tune_key(tc_mode mode, const Planned& p) {
  TuneKey k;
  std::memset(&k, 0, sizeof k);
  k.mode = (int)mode;
  k.lm = ilog2r(p.L.m);
  k.ln = ilog2r(p.L.n);
  k.lk = ilog2r(p.L.k);
  k.akc = p.info.a_k_contig;
  k.bkc = p.info.b_k_contig;
  return k;
}

// FNV-1a over the mode and, per problem, m, n, k and the access flags.
uint64_t batch_signature(tc_mode mode, const std::vector<Planned>& ps) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](int64_t v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (uint64_t)((v >> (8 * b)) & 0xff);
      h *= 1099511628211ull;
    }
  };
  mix((int64_t)mode);
  mix((int64_t)ps.size());
  for (const Planned& p : ps) {
    mix(p.L.m);
    mix(p.L.n);
    mix(p.L.k);
    mix(p.info.a_k_contig * 2 + p.info.b_k_contig);
  }
  return h;
}

bool tile_record_ok(int mode, int v) {
  if (mode == TC_MODE_F64) return v >= 0 && v < kF64BatchClasses;
  return v >= 16 && v <= tc_bn_max() && v % 16 == 0;
}

// The tables belong to one cache file: when TC_AUTOTUNE_CACHE names another
// file (or none) than the one loaded, they are emptied and read again.
void tune_load_file() {
  const char* path = std::getenv("TC_AUTOTUNE_CACHE");
  const std::string now = path ? path : "";
  if (g_tune_loaded && now == g_tune_path) return;
  g_tune_loaded = true;
  g_tune_path = now;
  g_tile.clear();
  g_balance.clear();
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[256];
  while (std::fgets(line, sizeof line, f)) {
    TuneKey k;
    std::memset(&k, 0, sizeof k);
    int v = 0;
    unsigned long long sig = 0;
    if (std::sscanf(line, "tile %d %d %d %d %d %d %d", &k.mode, &k.lm, &k.ln, &k.lk, &k.akc, &k.bkc,
                    &v) == 7) {
      if (tile_record_ok(k.mode, v)) g_tile[k] = v;  // a corrupt record is skipped
    } else if (std::sscanf(line, "balance %llx %d", &sig, &v) == 2) {
      for (int c : kBalanceCandidates)
        if (c == v) g_balance[(uint64_t)sig] = v;
    }
  }
  std::fclose(f);
}

void tune_save_file() {
  const char* path = std::getenv("TC_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "w");
  if (!f) return;
  for (const auto& kv : g_tile)
    std::fprintf(f, "tile %d %d %d %d %d %d %d\n", kv.first.mode, kv.first.lm, kv.first.ln,
                 kv.first.lk, kv.first.akc, kv.first.bkc, kv.second);
  for (const auto& kv : g_balance)
    std::fprintf(f, "balance %llx %d\n", (unsigned long long)kv.first, kv.second);
  std::fclose(f);
}

bool autotune_enabled() {
  const char* e = std::getenv("TC_AUTOTUNE");
  if (e && e[0] == '1') return true;
  if (e && e[0] == '0') return false;
  return std::getenv("TC_AUTOTUNE_CACHE") != nullptr;
}

// [lo, hi] element offsets of C's span (relative to its data pointer).
void c_span(const tc_plan_info& in, int64_t* lo, int64_t* hi) {
  int64_t cmin = 0, cmax = 0;
  for (int i = 0; i < in.nI; ++i) {
    const int64_t e = (in.I_len[i] - 1) * in.I_sC[i];
    if (e < 0) cmin += e; else cmax += e;
  }
  for (int j = 0; j < in.nJ; ++j) {
    const int64_t e = (in.J_len[j] - 1) * in.J_sC[j];
    if (e < 0) cmin += e; else cmax += e;
  }
  *lo = cmin;
  *hi = cmax;
}

// Best of two timed runs (after one untimed) of `launch` on stream st.
template <class F>
float time_best(cudaStream_t st, F launch) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return 1e30f;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return 1e30f;
  }
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0, st);
    if (!launch()) {
      best = 1e30f;
      break;
    }
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      best = 1e30f;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

// Scratch for timing one problem: its scatter vectors and a zeroed copy of
// C's span (the caller's C is never touched).
struct TuneScratch {
  int64_t* scat = nullptr;
  void* c = nullptr;
  void* partial = nullptr;
  void* dev = nullptr;  // FP64: descriptor, items, counter
  int64_t c_off = 0;    // element offset of C's data pointer inside `c`
  cudaStream_t st = nullptr;
  bool ok = false;
  ~TuneScratch() {
    if (st) cudaStreamDestroy(st);
    cudaFree(scat);
    cudaFree(c);
    cudaFree(partial);
    cudaFree(dev);
    cudaGetLastError();
  }
};

bool make_scratch(const Planned& p, size_t es, size_t partial_bytes, size_t dev_bytes,
                  TuneScratch& t) {
  const ScatterOffsets o = scatter_offsets(p.L, kBsBlock);
  int64_t lo, hi;
  c_span(p.info, &lo, &hi);
  const size_t cbytes = (size_t)(hi - lo + 1) * es;
  t.c_off = -lo;
  t.ok = cudaMalloc(&t.scat, (size_t)std::max<int64_t>(1, o.total) * 8) == cudaSuccess &&
         cudaMalloc(&t.c, cbytes) == cudaSuccess && cudaMemset(t.c, 0, cbytes) == cudaSuccess &&
         (partial_bytes == 0 || cudaMalloc(&t.partial, partial_bytes) == cudaSuccess) &&
         (dev_bytes == 0 || cudaMalloc(&t.dev, dev_bytes) == cudaSuccess) &&
         cudaStreamCreateWithFlags(&t.st, cudaStreamNonBlocking) == cudaSuccess &&
         launch_build_scatter(p.L, kBsBlock, t.scat, t.st) == cudaSuccess;
  if (!t.ok) cudaGetLastError();
  return t.ok;
}

// Tensor cores: time tile width bn for problem p on one persistent CTA.
float time_tc_width(const Planned& p, tc_mode mode, double alpha, double beta, int bn,
                    TuneScratch& t) {
  const int pieces = mode == TC_MODE_BF16X6 ? 3 : 2;
  const TcChoice c = choose_tc(p.L, pieces, 1, bn, 1);
  const ScatterOffsets o = scatter_offsets(p.L, kBsBlock);
  TcLaunch q;
  std::memset(&q, 0, sizeof q);
  DevProblem& d = q.single;
  d.a = p.a;
  d.b = p.b;
  d.c = static_cast<float*>(t.c) + t.c_off;
  d.partial = c.splits > 1 ? t.partial : nullptr;
  d.sp = scatter_ptrs(t.scat, o);
  d.m = p.L.m;
  d.n = p.L.n;
  d.k = p.L.k;
  d.alpha = alpha;
  d.beta = beta;
  d.a_kc = p.info.a_k_contig;
  d.b_kc = p.info.b_k_contig;
  d.bn = c.bn;
  d.tiles_n = (int32_t)((p.L.n + c.bn - 1) / c.bn);
  d.splits = c.splits;
  d.kps = c.kps;
  plan_access(p.L, d, q.tm, /*allow_box=*/false);  // as the batch kernel will run it
  q.pieces = pieces;
  q.ctas = 1;
  q.err = err_word();
  return time_best(t.st, [&] { return launch_tc(q, t.st) == cudaSuccess; });
}

// FP64: time tile class cls for problem p on one SM's worth of its CTAs.
float time_f64_class(const Planned& p, tc_dtype dt, double alpha, double beta, int cls,
                     TuneScratch& t) {
  int bm, bn;
  f64_batch_tile(cls, &bm, &bn);
  const int64_t tiles = ((p.L.m + bm - 1) / bm) * ((p.L.n + bn - 1) / bn);
  DevProblem d;
  std::memset(&d, 0, sizeof d);
  d.a = p.a;
  d.b = p.b;
  d.c = static_cast<char*>(t.c) + t.c_off * (int64_t)elem_size(dt);
  d.sp = scatter_ptrs(t.scat, scatter_offsets(p.L, kBsBlock));
  d.m = p.L.m;
  d.n = p.L.n;
  d.k = p.L.k;
  d.alpha = alpha;
  d.beta = beta;
  d.a_kc = p.info.a_k_contig;
  d.b_kc = p.info.b_k_contig;
  d.bn = bn;
  d.tiles_n = (int32_t)((p.L.n + bn - 1) / bn);
  d.splits = 1;
  d.kps = std::max<int64_t>(1, (p.L.k + f64_tile_k() - 1) / f64_tile_k()) * f64_tile_k();
  // the problem's tiles repeated until the whole GPU's CTAs of this class run
  // at least four waves of them: time / repetitions is then what one copy of
  // the problem costs at full occupancy, as in a batch (repeated tiles
  // rewrite the same scratch output)
  const int64_t sms = sm_count();
  const int64_t reps = std::max<int64_t>(1, (4 * sms * f64_batch_ctas_per_sm(cls) + tiles - 1) / tiles);
  std::vector<WorkItem> items((size_t)(tiles * reps));
  for (int64_t i = 0; i < tiles * reps; ++i) items[(size_t)i] = WorkItem{0, (int32_t)(i % tiles), 0, 0};
  char* base = static_cast<char*>(t.dev);
  DevProblem* dprob = reinterpret_cast<DevProblem*>(base);
  WorkItem* ditems = reinterpret_cast<WorkItem*>(base + align_up(sizeof(DevProblem), 256));
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(
      base + align_up(sizeof(DevProblem), 256) + align_up(sizeof(WorkItem) * items.size(), 256));
  if (cudaMemcpy(dprob, &d, sizeof d, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ditems, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return 1e30f;
  F64BatchLaunch q;
  q.dtype = dt;
  q.probs = dprob;
  q.items = ditems;
  q.nitems = tiles * reps;
  for (int c = 0; c <= kF64BatchClasses; ++c) q.class_off[c] = c <= cls ? 0 : tiles * reps;
  q.sms = sms;
  q.split_probs = nullptr;
  q.split_col_prefix = nullptr;
  q.split_cols = 0;
  q.n_split_probs = 0;
  q.max_m_split = q.max_n_split = 0;
  q.counter = ctr;
  return time_best(t.st, [&] { return launch_f64_batched(q, t.st) == cudaSuccess; }) / (float)reps;
}

size_t f64_tune_dev_bytes(const Planned& p) {
  int64_t most = 0;
  for (int c = 0; c < kF64BatchClasses; ++c) {
    int bm, bn;
    f64_batch_tile(c, &bm, &bn);
    const int64_t tiles = ((p.L.m + bm - 1) / bm) * ((p.L.n + bn - 1) / bn);
    const int64_t reps = std::max<int64_t>(1, (4 * sm_count() * f64_batch_ctas_per_sm(c) + tiles - 1) / tiles);
    most = std::max<int64_t>(most, tiles * reps);
  }
  return align_up(sizeof(DevProblem), 256) + align_up(sizeof(WorkItem) * (size_t)most, 256) +
         align_up(sizeof(unsigned long long) * kF64BatchClasses, 256);
}

// The timed tile choice for one problem (-1: keep the estimate).
int tune_tile(const Planned& p, tc_dtype dt, tc_mode mode, double alpha, double beta) {
  TuneScratch t;
  if (mode == TC_MODE_F64) {
    if (!make_scratch(p, elem_size(dt), 0, f64_tune_dev_bytes(p), t)) return -1;
    int best = -1;
    float tb = 1e30f;
    for (int c = 0; c < kF64BatchClasses; ++c) {
      const float ms = time_f64_class(p, dt, alpha, beta, c, t);
      if (ms < tb) {
        tb = ms;
        best = c;
      }
    }
    return best;
  }
  std::vector<int> bns;
  if (p.L.n < 128) {
    const int b0 = (int)std::max<int64_t>(16, (p.L.n + 15) / 16 * 16);
    bns.push_back(b0);
    if (b0 > 32) bns.push_back((b0 / 2 + 15) / 16 * 16);
  } else {
    bns.push_back(128);
    bns.push_back(64);
  }
  const int pieces = mode == TC_MODE_BF16X6 ? 3 : 2;
  int64_t max_split = 1;
  for (int bn : bns) max_split = std::max<int64_t>(max_split, choose_tc(p.L, pieces, 1, bn, 1).splits);
  const size_t pbytes = max_split > 1 ? (size_t)max_split * p.L.m * p.L.n * sizeof(float) : 0;
  if (!make_scratch(p, sizeof(float), pbytes, 0, t)) return -1;
  int best = -1;
  float tb = 1e30f;
  for (int bn : bns) {
    const float ms = time_tc_width(p, mode, alpha, beta, bn, t);
    if (ms < tb) {
      tb = ms;
      best = bn;
    }
  }
  return best;
}

}  // namespace

// ---- the plan ----------------------------------------------------------------------------------
struct tc_plan {
  tc_dtype dtype;
  tc_mode mode;
  int device;
  std::vector<Planned> planned;   // active problems only
  std::vector<ProbCfg> cfg;
  void* dmem = nullptr;
  Layout* d_layouts = nullptr;
  int64_t* d_offs = nullptr;
  int64_t* d_scat = nullptr;
  DevProblem* d_probs = nullptr;
  WorkItem* d_items = nullptr;
  unsigned long long* d_counter = nullptr;  // work counters of the persistent mainloop(s)
  int64_t class_off[kF64BatchClasses + 1] = {};  // FP64: the work list's tile classes
  int32_t* d_split = nullptr;
  int64_t* d_split_cols = nullptr;
  int64_t split_cols = 0;
  int64_t total_scatter = 0, nitems = 0;
  int32_t n_split = 0;
  int64_t max_m_split = 0, max_n_split = 0;
  int pieces = 2;
  int reduce_f64 = 0;  // the split-reduction setting when the plan was created
  bool checks = false;  // tc_set_checks was on when the plan was created
  int balance = kBalanceDefault;   // D of the k-split rule (see the autotuner)
  std::vector<int32_t> orig;       // the caller's index of each planned problem
  int32_t count = 0;               // problems the caller passed
  CheckBounds* d_bounds = nullptr;  // checked plans: per-problem scatter-vector ranges
  int64_t ctas = 152;
  int64_t sms = 152;
  // the packed form (tensor-core plans): every problem's A and B packed by one
  // launch from a job list, then the packed mainloop over the work list
  bool packed = false;
  PackJob* d_jobs = nullptr;
  int64_t* d_job_prefix = nullptr;
  void* d_pitems = nullptr;  // packed: the work items decoded at creation (launch_decode_items)
  int32_t njobs = 0;
  int64_t pack_groups = 0;
};

namespace {

int build_plan(tc_plan* pl, const std::vector<tc_problem>& probs, int balance) {
  const int sms = sm_count();
  pl->balance = balance;
  pl->count = (int32_t)probs.size();
  const bool f64 = pl->mode == TC_MODE_F64;
  pl->ctas = sms;
  pl->sms = sms;
  pl->reduce_f64 = split_reduction_f64() ? 1 : 0;
  pl->checks = checks_on();
  pl->pieces = pl->mode == TC_MODE_BF16X6 ? 3 : 2;
  std::vector<double> alpha, beta;
  for (size_t q = 0; q < probs.size(); ++q) {
    const tc_problem& pr = probs[q];
    Planned p;
    int rc = plan_checked(pl->dtype, &pr.A, &pr.B, &pr.C, &p);
    if (rc != TC_OK) return rc;
    if (p.L.m == 0 || p.L.n == 0) continue;  // empty output: nothing to do
    if (pr.alpha == 0.0) p.L.k = 0;          // C := beta * C, A and B not read
    pl->planned.push_back(p);
    pl->orig.push_back((int32_t)q);
    alpha.push_back(pr.alpha);
    beta.push_back(pr.beta);
  }
  // The packed form for tensor-core batches: always under TC_ACCESS_PACKED,
  // under TC_ACCESS_AUTO when the batch holds at least 2^26 multiply-adds
  // (as for single contractions).  Every operand of a batch is gathered
  // otherwise, so packing pays here even for operands read by one tile: the
  // packing launch, many small CTAs per SM, gathers them faster than the
  // mainloop's loader warps.
  if (!f64) {
    double work = 0;
    for (size_t i = 0; i < pl->planned.size(); ++i) {
      const Layout& L = pl->planned[i].L;
      work += (double)L.m * (double)L.n * (double)L.k;
    }
    const int acc = access_setting();
    pl->packed = acc == TC_ACCESS_PACKED || (acc == TC_ACCESS_AUTO && work >= 67108864.0);
  }
  // Packed batches exchange A's and B's roles for problems whose 128-row
  // tiles would pad the rows far more than the columns' tiles (16..128 wide)
  // would pad them the other way round: the packed operands and the MMA work
  // shrink with the padding; the epilogue then writes C along its columns.
  if (pl->packed) {
    auto padded = [](int64_t m, int64_t n) {
      const int64_t bn = std::min<int64_t>(128, std::max<int64_t>(16, (n + 15) / 16 * 16));
      return (double)((m + 127) / 128 * 128) * (double)((n + bn - 1) / bn * bn);
    };
    for (Planned& p : pl->planned) {
      const Layout& L = p.L;
      if (L.k > 0 && L.m < 128 && padded(L.n, L.m) < 0.75 * padded(L.m, L.n)) swap_roles(&p);
    }
  }
  // the autotuner's tile records (see K7), timed here for classes without one
  const bool tune = autotune_enabled();
  auto tuned_tile = [&](int i) -> int {
    if (!tune || pl->planned[i].L.k == 0) return -1;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_file();
    const TuneKey key = tune_key(pl->mode, pl->planned[i]);
    auto it = g_tile.find(key);
    if (it != g_tile.end()) return it->second;
    if (t_tile_budget_ms <= 0.0) return -1;
    const Layout& L = pl->planned[i].L;
    // one SM runs the whole problem: skip those too large to time that way
    const double flops = 2.0 * (double)L.m * (double)L.n * (double)L.k;
    if (flops > (f64 ? 0x1p27 : 0x1p34)) return -1;
    const auto t0 = std::chrono::steady_clock::now();
    const int v = tune_tile(pl->planned[i], pl->dtype, pl->mode, alpha[i], beta[i]);
    t_tile_budget_ms -= std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (v >= 0) {
      g_tile[key] = v;
      tune_save_file();
    }
    return v;
  };
  const int np = (int)pl->planned.size();
  pl->cfg.resize(np);

  // per-problem tiles and k-splits
  const int tk_f = f64_tile_k();
  double total_cost = 0;
  std::vector<double> cost(np);
  for (int i = 0; i < np; ++i) {
    const Layout& L = pl->planned[i].L;
    ProbCfg& c = pl->cfg[i];
    if (f64) {
      // the timed tile class, else the one that pads the problem least (ties:
      // the larger tile)
      double best = 0;
      for (int cl = 0; cl < kF64BatchClasses; ++cl) {
        int bm, bn;
        f64_batch_tile(cl, &bm, &bn);
        const double padded = (double)((L.m + bm - 1) / bm * bm) * (double)((L.n + bn - 1) / bn * bn);
        if (cl == 0 || padded < best) {
          best = padded;
          c.cls = cl;
          c.bm = bm;
          c.bn = bn;
        }
      }
      const int tv = tuned_tile(i);
      if (tv >= 0) {
        c.cls = tv;
        f64_batch_tile(tv, &c.bm, &c.bn);
      }
      c.tiles = ((L.m + c.bm - 1) / c.bm) * ((L.n + c.bn - 1) / c.bn);
      // in warp x k-tile units (a warp computes 32 x 32)
      cost[i] = (double)c.tiles * (c.bm / 32) * (c.bn / 32) *
                std::max<int64_t>(1, (L.k + tk_f - 1) / tk_f);
    } else {
      const int tv = tuned_tile(i);
      // in a batch the other problems keep the SMs busy: no parallelism split
      // here (long items are split below, for balance)
      const TcChoice ch = choose_tc(L, pl->pieces, 1, tv > 0 ? tv : 0, 1);
      c.bn = ch.bn;
      c.splits = ch.splits;
      c.kps = ch.kps;
      c.tiles = ((L.m + 127) / 128) * ((L.n + c.bn - 1) / c.bn);
      cost[i] = (double)c.tiles * std::max<int64_t>(1, (L.k + 31) / 32 / c.splits) * c.splits;
    }
    total_cost += cost[i];
  }
  // Split long-k problems so that no item exceeds 1/D of a CTA's fair share
  // of the batch (in k-tiles: 16 on the FP64 path, 32 on the tensor cores;
  // D = `balance`, 4 unless the autotuner chose another).
  const double D = (double)balance;
  if (!f64) {
    const double fair = total_cost / (double)sms;
    for (int i = 0; i < np; ++i) {
      const Layout& L = pl->planned[i].L;
      ProbCfg& c = pl->cfg[i];
      const int64_t KT = (L.k + 31) / 32;
      if (KT == 0) continue;
      const double item = (double)KT / c.splits;
      if (item <= std::max(8.0, fair / D)) continue;
      int64_t s = (int64_t)std::ceil((double)KT / std::max(8.0, fair / D));
      s = std::max<int64_t>(c.splits, std::min<int64_t>(s, KT));
      const int64_t ktps = (KT + s - 1) / s;
      c.kps = ktps * 32;
      c.splits = (int)((KT + ktps - 1) / ktps);
    }
  }
  if (f64) {
    // a warp's fair share of the batch in k-tiles (eight warps per SM)
    const double fair = total_cost / (8.0 * (double)sms);
    for (int i = 0; i < np; ++i) {
      const Layout& L = pl->planned[i].L;
      ProbCfg& c = pl->cfg[i];
      const int64_t KT = (L.k + tk_f - 1) / tk_f;
      int64_t s = 1;
      if (KT > 0 && fair > 0) {
        const double item = (double)KT;  // k-tiles per tile
        s = (int64_t)std::ceil(item / std::max(1.0, fair / D));
        s = std::max<int64_t>(1, std::min<int64_t>(s, KT));
      }
      const int64_t ktps = KT > 0 ? (KT + s - 1) / s : 0;
      c.kps = std::max<int64_t>(1, ktps) * tk_f;
      c.splits = KT > 0 ? (int)((KT + ktps - 1) / ktps) : 1;
    }
  }

  std::vector<size_t> pack_a(np, 0), pack_b(np, 0);
  size_t pack_total = 0;
  if (pl->packed) {
    for (int i = 0; i < np; ++i) {
      const Layout& L = pl->planned[i].L;
      const ProbCfg& c = pl->cfg[i];
      if (L.k == 0) continue;
      const int64_t KT = (L.k + 31) / 32;
      pack_a[i] = pack_total;
      pack_total += align_up((size_t)((L.m + 127) / 128) * KT * pl->pieces * 128 * 32 * 2, 256);
      pack_b[i] = pack_total;
      pack_total += align_up((size_t)((L.n + c.bn - 1) / c.bn) * KT * pl->pieces * c.bn * 32 * 2, 256);
    }
  }

  // device buffer: layouts | offsets | scatter | problems | items | split list | partials
  std::vector<int64_t> offs(np + 1, 0);
  for (int i = 0; i < np; ++i) offs[i + 1] = offs[i] + scatter_offsets(pl->planned[i].L, kBsBlock).total;
  pl->total_scatter = offs[np];
  std::vector<WorkItem> items;
  std::vector<int32_t> splitp;
  std::vector<int64_t> part_off(np, -1);
  int64_t part_elems = 0;
  for (int i = 0; i < np; ++i) {
    const ProbCfg& c = pl->cfg[i];
    for (int s = 0; s < c.splits; ++s)
      for (int64_t t = 0; t < c.tiles; ++t) items.push_back(WorkItem{i, (int32_t)t, s, 0});
    if (c.splits > 1) {
      splitp.push_back(i);
      part_off[i] = part_elems;
      part_elems += (int64_t)c.splits * pl->planned[i].L.m * pl->planned[i].L.n;
      pl->max_m_split = std::max(pl->max_m_split, pl->planned[i].L.m);
      pl->max_n_split = std::max(pl->max_n_split, pl->planned[i].L.n);
    }
  }
  // longest items first (k-tiles of the item), stable for locality; FP64:
  // grouped by tile class first, one persistent launch per class
  auto item_cost = [&](const WorkItem& w) {
    const ProbCfg& c = pl->cfg[w.prob];
    const Layout& L = pl->planned[w.prob].L;
    const int64_t kb = (int64_t)w.split * c.kps, ke = std::min<int64_t>(L.k, kb + c.kps);
    return (double)std::max<int64_t>(0, ke - kb) * (f64 ? 1.0 : c.bn / 128.0);
  };
  std::stable_sort(items.begin(), items.end(), [&](const WorkItem& x, const WorkItem& y) {
    if (f64 && pl->cfg[x.prob].cls != pl->cfg[y.prob].cls)
      return pl->cfg[x.prob].cls < pl->cfg[y.prob].cls;
    return item_cost(x) > item_cost(y);
  });
  for (int cl = 0; cl <= kF64BatchClasses; ++cl) pl->class_off[cl] = 0;
  if (f64) {
    for (const WorkItem& w : items) pl->class_off[pl->cfg[w.prob].cls + 1]++;
    for (int cl = 0; cl < kF64BatchClasses; ++cl) pl->class_off[cl + 1] += pl->class_off[cl];
  }
  pl->nitems = (int64_t)items.size();
  pl->n_split = (int32_t)splitp.size();
  if (log_enabled()) {
    std::map<std::pair<int, int>, int> tiles;
    double ksteps = 0;
    for (const WorkItem& w : items) ksteps += item_cost(w);
    for (int i = 0; i < np; ++i) tiles[{pl->cfg[i].bm, pl->cfg[i].bn}]++;
    std::fprintf(stderr, "[libtc] batch plan: %d problems, %lld work items, %d split, "
                 "%.3g k-index-units of work%s; tiles (m x n: problems):", np,
                 (long long)pl->nitems, pl->n_split, ksteps, pl->packed ? ", packed" : "");
    for (const auto& kv : tiles)
      std::fprintf(stderr, " %dx%d: %d", kv.first.first, kv.first.second, kv.second);
    std::fprintf(stderr, "\n");
  }

  const size_t es = f64 ? sizeof(double) : sizeof(float);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  const size_t o_lay = take(sizeof(Layout) * std::max(np, 1));
  const size_t o_offs = take(sizeof(int64_t) * (np + 1));
  const size_t o_scat = take(sizeof(int64_t) * std::max<int64_t>(1, pl->total_scatter));
  const size_t o_prob = take(sizeof(DevProblem) * std::max(np, 1));
  const size_t o_item = take(sizeof(WorkItem) * std::max<int64_t>(1, pl->nitems));
  const size_t o_split = take(sizeof(int32_t) * std::max<int32_t>(1, pl->n_split));
  const size_t o_scols = take(sizeof(int64_t) * (pl->n_split + 1));
  const size_t o_part = take(es * std::max<int64_t>(1, part_elems));
  const size_t o_tmap = take(sizeof(CUtensorMap) * 2 * std::max(np, 1));
  const size_t o_ctr = take(sizeof(unsigned long long) * kF64BatchClasses);
  const size_t o_cb = take(pl->checks ? sizeof(CheckBounds) * std::max(np, 1) : 0);
  const size_t o_jobs = take(pl->packed ? sizeof(PackJob) * 2 * std::max(np, 1) : 0);
  const size_t o_jpre = take(pl->packed ? sizeof(int64_t) * (2 * np + 1) : 0);
  const size_t o_pack = take(pack_total);
  const size_t o_pit = take(pl->packed ? tc_item_bytes() * (size_t)std::max<int64_t>(1, pl->nitems) : 0);
  if (cudaMalloc(&pl->dmem, off) != cudaSuccess) {
    cudaGetLastError();
    pl->dmem = nullptr;
    return TC_ERR_CUDA;
  }
  char* base = static_cast<char*>(pl->dmem);
  pl->d_layouts = reinterpret_cast<Layout*>(base + o_lay);
  pl->d_offs = reinterpret_cast<int64_t*>(base + o_offs);
  pl->d_scat = reinterpret_cast<int64_t*>(base + o_scat);
  pl->d_probs = reinterpret_cast<DevProblem*>(base + o_prob);
  pl->d_items = reinterpret_cast<WorkItem*>(base + o_item);
  pl->d_counter = reinterpret_cast<unsigned long long*>(base + o_ctr);
  pl->d_split = reinterpret_cast<int32_t*>(base + o_split);
  pl->d_split_cols = reinterpret_cast<int64_t*>(base + o_scols);
  if (pl->checks) pl->d_bounds = reinterpret_cast<CheckBounds*>(base + o_cb);
  if (pl->packed) {
    pl->d_jobs = reinterpret_cast<PackJob*>(base + o_jobs);
    pl->d_job_prefix = reinterpret_cast<int64_t*>(base + o_jpre);
  }
  uint8_t* packbuf = reinterpret_cast<uint8_t*>(base + o_pack);
  std::vector<PackJob> jobs;
  std::vector<int64_t> jpre(1, 0);
  std::vector<int64_t> scols(pl->n_split + 1, 0);
  for (int i = 0; i < pl->n_split; ++i) scols[i + 1] = scols[i] + pl->planned[splitp[i]].L.n;
  pl->split_cols = scols[pl->n_split];
  char* partial = base + o_part;

  std::vector<Layout> lay(np);
  std::vector<DevProblem> dp(np);
  std::vector<CUtensorMap> maps(2 * (size_t)np);
  const CUtensorMap* d_maps = reinterpret_cast<const CUtensorMap*>(base + o_tmap);
  for (int i = 0; i < np; ++i) {
    const Planned& p = pl->planned[i];
    const ProbCfg& c = pl->cfg[i];
    lay[i] = p.L;
    DevProblem& d = dp[i];
    std::memset(&d, 0, sizeof d);
    d.a = p.a;
    d.b = p.b;
    d.c = p.c;
    d.partial = part_off[i] >= 0 ? partial + part_off[i] * es : nullptr;
    d.sp = scatter_ptrs(pl->d_scat + offs[i], scatter_offsets(p.L, kBsBlock));
    d.m = p.L.m;
    d.n = p.L.n;
    d.k = p.L.k;
    d.alpha = alpha[i];
    d.beta = beta[i];
    d.a_kc = p.info.a_k_contig;
    d.b_kc = p.info.b_k_contig;
    d.bn = c.bn;
    d.tiles_n = (int32_t)((p.L.n + c.bn - 1) / c.bn);
    d.splits = c.splits;
    d.kps = c.kps;
    if (!f64) {
      // batch plans gather every operand: their kernel form with boxes faulted
      // the GPU on the 512-problem workload, cause not yet found
      plan_access(p.L, d, &maps[2 * (size_t)i], /*allow_box=*/false);
      d.tmaps = d_maps + 2 * (size_t)i;
    }
    if (pl->packed && p.L.k > 0) {
      const int64_t KT = (p.L.k + 31) / 32;
      d.pa = packbuf + pack_a[i];
      d.pb = packbuf + pack_b[i];
      PackJob ja;
      std::memset(&ja, 0, sizeof ja);
      ja.x = static_cast<const float*>(d.a);
      ja.rs = d.sp.rA;
      ja.ks = d.sp.cA;
      ja.kbs = d.sp.cbsA;
      ja.rows = d.m;
      ja.k = d.k;
      ja.KT = KT;
      ja.R = 128;
      ja.units = ((d.m + 127) / 128) * KT;
      ja.out = packbuf + pack_a[i];
      PackJob jb = ja;
      jb.x = static_cast<const float*>(d.b);
      jb.rs = d.sp.cB;
      jb.ks = d.sp.rB;
      jb.kbs = d.sp.rbsB;
      jb.rows = d.n;
      jb.R = c.bn;
      jb.units = (int64_t)d.tiles_n * KT;
      jb.out = packbuf + pack_b[i];
      pack_job_groups(ja);
      pack_job_groups(jb);
      for (const PackJob& j : {ja, jb}) {
        jobs.push_back(j);
        jpre.push_back(jpre.back() + j.groups);
      }
    }
  }
  pl->njobs = (int32_t)jobs.size();
  pl->pack_groups = jpre.back();
  auto up = [](void* dst, const void* src, size_t bytes) {
    return bytes == 0 || cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  if (!up(pl->d_layouts, lay.data(), sizeof(Layout) * np) ||
      !up(pl->d_offs, offs.data(), sizeof(int64_t) * (np + 1)) ||
      !up(pl->d_probs, dp.data(), sizeof(DevProblem) * np) ||
      !up(pl->d_items, items.data(), sizeof(WorkItem) * items.size()) ||
      !up(pl->d_split, splitp.data(), sizeof(int32_t) * splitp.size()) ||
      !up(pl->d_split_cols, scols.data(), sizeof(int64_t) * scols.size()) ||
      !up(base + o_tmap, maps.data(), sizeof(CUtensorMap) * maps.size()) ||
      (pl->packed && (!up(pl->d_jobs, jobs.data(), sizeof(PackJob) * jobs.size()) ||
                      !up(pl->d_job_prefix, jpre.data(), sizeof(int64_t) * jpre.size()))))
    return TC_ERR_CUDA;
  if (pl->checks) {
    std::vector<CheckBounds> cb(np);
    for (int i = 0; i < np; ++i) cb[i] = check_bounds(lay[i]);
    if (!up(pl->d_bounds, cb.data(), sizeof(CheckBounds) * np)) return TC_ERR_CUDA;
  }
  // K1 once per plan: the scatter vectors depend on the layouts alone, so
  // every execution reads the ones built here (the call returns once they
  // are built)
  if (np > 0 && (launch_build_scatter_batched(pl->d_layouts, pl->d_offs, np, pl->total_scatter,
                                               kBsBlock, pl->d_scat, 0) != cudaSuccess ||
                 cudaStreamSynchronize(0) != cudaSuccess))
    return TC_ERR_CUDA;
  // packed: the work items decoded once, here
  if (pl->packed) {
    pl->d_pitems = base + o_pit;
    if (launch_decode_items(pl->d_probs, pl->d_items, pl->nitems, pl->d_pitems, 0) != cudaSuccess ||
        cudaStreamSynchronize(0) != cudaSuccess)
      return TC_ERR_CUDA;
  }
  return TC_OK;
}

// K7 (2): the balance divisor D for this batch, from whole-batch timings of
// plans whose outputs are scratch copies (the caller's C is never touched).
int tune_balance(tc_dtype dtype, tc_mode mode, const std::vector<tc_problem>& list) {
  const size_t es = elem_size(dtype);
  std::vector<tc_problem> tmp = list;
  std::vector<size_t> off(list.size());
  size_t total = 0;
  for (size_t i = 0; i < list.size(); ++i) {
    const tc_tensor& C = list[i].C;
    int64_t lo = 0, hi = 0;
    bool empty = false;
    for (int d = 0; d < C.rank; ++d) {
      if (C.len[d] == 0) empty = true;
      const int64_t e = (C.len[d] - 1) * C.stride[d];
      if (e < 0) lo += e; else hi += e;
    }
    off[i] = total;
    if (!empty) total = align_up(total + (size_t)(hi - lo + 1) * es, 256);
    tmp[i].C.data = reinterpret_cast<void*>(-lo * (int64_t)es);  // relative; rebased below
  }
  void* scratch = nullptr;
  if (cudaMalloc(&scratch, std::max<size_t>(total, 256)) != cudaSuccess ||
      cudaMemset(scratch, 0, std::max<size_t>(total, 256)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(scratch);
    return kBalanceDefault;
  }
  for (size_t i = 0; i < tmp.size(); ++i)
    tmp[i].C.data = static_cast<char*>(scratch) + off[i] + reinterpret_cast<intptr_t>(tmp[i].C.data);
  cudaStream_t st = nullptr;
  int best = kBalanceDefault;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess) {
    float tb = 1e30f;
    for (int D : kBalanceCandidates) {
      tc_plan* pl = new tc_plan;
      pl->dtype = dtype;
      pl->mode = mode;
      cudaGetDevice(&pl->device);
      float ms = 1e30f;
      if (build_plan(pl, tmp, D) == TC_OK)
        ms = time_best(st, [&] { return tc_plan_execute(pl, nullptr, 0, st) == TC_OK; });
      tc_plan_destroy(pl);
      if (ms < tb) {
        tb = ms;
        best = D;
      }
    }
    cudaStreamDestroy(st);
  }
  cudaFree(scratch);
  cudaGetLastError();
  return best;
}

}  // namespace

extern "C" {

int tc_plan_create(tc_dtype dtype, tc_mode mode, int32_t count, const tc_problem* probs,
                   tc_plan** out) {
  NvtxRange range("tc_plan_create");
  if (!out || count < 0 || (count > 0 && !probs)) return TC_ERR_ARG;
  int rc = check_modes(dtype, mode);
  if (rc != TC_OK) return rc;
  const std::vector<tc_problem> list(probs, probs + count);
  int balance = kBalanceDefault;
  t_tile_budget_ms = kTileTuneBudgetMs;  // shared by the balance trials and the plan
  if (autotune_enabled()) {
    std::vector<Planned> ps;
    for (const tc_problem& pr : list) {
      Planned p;
      if ((rc = plan_checked(dtype, &pr.A, &pr.B, &pr.C, &p)) != TC_OK) return rc;
      if (p.L.m > 0 && p.L.n > 0) ps.push_back(p);
    }
    const uint64_t sig = batch_signature(mode, ps);
    bool have = false;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      tune_load_file();
      auto it = g_balance.find(sig);
      if (it != g_balance.end()) {
        balance = it->second;
        have = true;
      }
    }
    if (!have && !ps.empty()) {
      balance = tune_balance(dtype, mode, list);
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_balance[sig] = balance;
      tune_save_file();
    }
  }
  tc_plan* pl = new tc_plan;
  pl->dtype = dtype;
  pl->mode = mode;
  cudaGetDevice(&pl->device);
  rc = build_plan(pl, list, balance);
  if (rc != TC_OK) {
    tc_plan_destroy(pl);
    return rc;
  }
  *out = pl;
  return TC_OK;
}

int tc_plan_config(const tc_plan* plan, int32_t index, int32_t* out) {
  if (!plan || !out || index < 0 || index >= plan->count) return TC_ERR_ARG;
  out[0] = out[1] = out[2] = 0;
  out[3] = plan->balance;
  for (size_t i = 0; i < plan->orig.size(); ++i)
    if (plan->orig[i] == index) {
      out[0] = plan->cfg[i].bm;
      out[1] = plan->cfg[i].bn;
      out[2] = plan->cfg[i].splits;
    }
  return TC_OK;
}

int tc_plan_form(const tc_plan* plan, int32_t* form) {
  if (!plan || !form) return TC_ERR_ARG;
  if (plan->mode == TC_MODE_F64) return TC_ERR_UNSUPPORTED;
  *form = plan->packed ? TC_FORM_PACKED : TC_FORM_GATHER;
  return TC_OK;
}

int tc_plan_workspace_size(const tc_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return TC_ERR_ARG;
  *bytes = 0;  // the plan owns its scatter vectors and partials
  return TC_OK;
}

int tc_plan_execute(tc_plan* plan, void* workspace, size_t ws_bytes, void* stream) {
  NvtxRange range("tc_plan_execute");
  (void)workspace;
  (void)ws_bytes;
  if (!plan) return TC_ERR_ARG;
  const int np = (int)plan->planned.size();
  if (np == 0) return TC_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int32_t* gate = nullptr;
  if (plan->checks) {
    int32_t* ew = err_word();
    if (!ew || launch_check_scatter_batched(plan->d_layouts, plan->d_offs, plan->d_bounds, np,
                                            plan->total_scatter, kBsBlock, plan->d_scat, ew,
                                            s) != cudaSuccess)
      return TC_ERR_CUDA;
    gate = ew;
  }
  cudaError_t e;
  if (plan->mode == TC_MODE_F64) {
    F64BatchLaunch q;
    q.dtype = plan->dtype;
    q.probs = plan->d_probs;
    q.items = plan->d_items;
    q.nitems = plan->nitems;
    for (int cl = 0; cl <= kF64BatchClasses; ++cl) q.class_off[cl] = plan->class_off[cl];
    q.sms = plan->sms;
    q.split_probs = plan->d_split;
    q.split_col_prefix = plan->d_split_cols;
    q.split_cols = plan->split_cols;
    q.n_split_probs = plan->n_split;
    q.max_m_split = plan->max_m_split;
    q.max_n_split = plan->max_n_split;
    q.counter = plan->d_counter;
    q.gate = gate;
    e = launch_f64_batched(q, s);
  } else {
    TcLaunch q;
    std::memset(&q, 0, sizeof q);
    q.probs = plan->d_probs;
    q.items = plan->d_items;
    q.nitems = plan->nitems;
    q.nprobs = np;
    q.pieces = plan->pieces;
    q.reduce_f64 = plan->reduce_f64;
    q.ctas = plan->ctas;
    q.split_probs = plan->d_split;
    q.split_col_prefix = plan->d_split_cols;
    q.split_cols = plan->split_cols;
    q.n_split_probs = plan->n_split;
    q.max_m_split = plan->max_m_split;
    q.max_n_split = plan->max_n_split;
    q.counter = plan->d_counter;
    q.err = err_word();
    q.gate = gate;
    if (plan->packed) {
      q.pack_items = plan->d_pitems;
      q.pack_jobs = plan->d_jobs;
      q.pack_prefix = plan->d_job_prefix;
      q.pack_njobs = plan->njobs;
      q.pack_groups = plan->pack_groups;
    }
    e = launch_tc(q, s);
  }
  return e == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

void tc_plan_destroy(tc_plan* plan) {
  if (!plan) return;
  if (plan->dmem) cudaFree(plan->dmem);
  delete plan;
}

int tc_batched_workspace_size(tc_dtype dtype, tc_mode mode, int32_t count,
                              const tc_problem* probs, size_t* bytes) {
  if (!bytes || count < 0 || (count > 0 && !probs)) return TC_ERR_ARG;
  int rc = check_modes(dtype, mode);
  if (rc != TC_OK) return rc;
  for (int32_t i = 0; i < count; ++i) {
    Planned p;
    if ((rc = plan_checked(dtype, &probs[i].A, &probs[i].B, &probs[i].C, &p)) != TC_OK) return rc;
  }
  *bytes = 0;
  return TC_OK;
}

int tc_contract_batched(tc_dtype dtype, tc_mode mode, int32_t count, const tc_problem* probs,
                        void* workspace, size_t ws_bytes, void* stream) {
  tc_plan* pl = nullptr;
  int rc = tc_plan_create(dtype, mode, count, probs, &pl);
  if (rc != TC_OK) return rc;
  rc = tc_plan_execute(pl, workspace, ws_bytes, stream);
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess && rc == TC_OK)
    rc = TC_ERR_CUDA;
  tc_plan_destroy(pl);
  return rc;
}

}  // extern "C"
