// libtc C ABI: argument checks, planning, workspace carving and launches.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "host_common.h"
#include "kernels.h"

namespace tc {
int aliases(const tc_tensor* A, const tc_tensor* B, const tc_tensor* C, size_t es);

std::atomic<uint64_t> g_launches{0};
thread_local cudaEvent_t t_ev_before = nullptr, t_ev_after = nullptr;

void note_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
void mainloop_event_before(cudaStream_t s) {
  if (t_ev_before) cudaEventRecord(t_ev_before, s);
}
void mainloop_event_after(cudaStream_t s) {
  if (t_ev_after) cudaEventRecord(t_ev_after, s);
  t_ev_before = t_ev_after = nullptr;
}
}  // namespace tc

namespace {
__device__ int32_t g_tc_error;  // device error word (kDevTimeout / kDevBounds), 0 = none
std::mutex g_mu;
int32_t* g_err_ptr[64] = {};
}  // namespace

namespace tc {

// Address of the device error word on the current device (set up once per device).
int32_t* err_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_err_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tc_error) != cudaSuccess) return nullptr;
    g_err_ptr[dev] = static_cast<int32_t*>(p);
  }
  return g_err_ptr[dev];
}

size_t elem_size(tc_dtype dt) { return dt == TC_F64 ? 8 : 4; }

bool log_enabled() {
  const char* e = std::getenv("TC_LOG");
  return e && e[0] == '1';
}

int check_modes(tc_dtype dt, tc_mode mode) {
  if (dt != TC_F64 && dt != TC_F32) return TC_ERR_ARG;
  if (mode != TC_MODE_F64 && mode != TC_MODE_BF16X3 && mode != TC_MODE_BF16X6) return TC_ERR_ARG;
  if (mode != TC_MODE_F64 && dt != TC_F32) return TC_ERR_UNSUPPORTED;
  return TC_OK;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return 152;
  }
  return n;
}

// Tile shape and split of the contracted range for the tensor-core mainloop:
//  * tile width bn: the next multiple of 16 above n, at most 128;
//  * split count S: when the output alone has fewer tiles than SMs, split the
//    contracted range so the grid covers the SMs, keeping at least 8 k-tiles
//    of 32 per split; and at least as many splits as keep every split within
//    tc_max_item_ktiles() k-tiles (the kernel bounds every FP32 accumulation
//    chain to 1024 terms and folds at most 16 such chunks per item).
TcChoice choose_tc(const Layout& L, int pieces, int sms, int bn_force, int split_mult) {
  (void)pieces;
  TcChoice c;
  const int64_t tm = (L.m + 127) / 128;
  const int bmax = tc_bn_max();
  c.bn = bn_force > 0 ? std::min(bn_force, bmax)
                      : (int)std::min<int64_t>(bmax, std::max<int64_t>(16, (L.n + 15) / 16 * 16));
  const int64_t tiles = tm * ((L.n + c.bn - 1) / c.bn);
  const int64_t kt = (L.k + 31) / 32;
  int64_t s = 1;
  if (tiles < sms) s = std::min<int64_t>(sms / std::max<int64_t>(tiles, 1), std::max<int64_t>(1, kt / 8));
  s = std::max<int64_t>(1, s) * std::max(1, split_mult);
  s = std::max<int64_t>(s, (kt + tc_max_item_ktiles() - 1) / tc_max_item_ktiles());
  s = std::min<int64_t>(s, std::max<int64_t>(kt, 1));
  const int64_t ktps = (kt + s - 1) / s;
  c.kps = std::max<int64_t>(1, ktps) * 32;
  c.splits = (int)std::max<int64_t>(1, (L.k + c.kps - 1) / c.kps);
  return c;
}

// The pair form of the tensor-core box kernel (cta_group::2: each CTA pair
// computes 256-row tiles, each CTA loading its own 128 rows of A and half of
// the tile's columns of B, which cuts every SM's intake of operand bytes per
// k-tile by a quarter) is taken when both operands are boxes for it and the
// problem has at least two waves of pair tiles.  TC_PAIR=0 turns it off,
// TC_PAIR=1 takes it whenever the boxes allow (tests, experiments).
int pair_setting() {
  const char* e = std::getenv("TC_PAIR");
  if (e && e[0] == '0') return 0;
  if (e && e[0] == '1') return 2;
  return 1;
}

// Access plan of a single tensor-core contraction: the pair form where it
// applies, else boxes or gathers (plan_access).
void plan_single_access(const Layout& L, DevProblem& d, CUtensorMap* maps, int sms) {
  const int ps = pair_setting();
  const int64_t pair_items = ((L.m + 255) / 256) * d.tiles_n * d.splits;
  if (ps > 0 && L.m > 128 && (ps == 2 || pair_items >= sms)) {
    plan_access(L, d, maps, true, true);
    if (d.pair) return;
  }
  plan_access(L, d, maps);
}

struct WsLayout {
  size_t scatter_off, scatter_bytes;
  size_t partial_off, partial_bytes;
  size_t pack_off, pack_bytes;  // packed form: the packed units of A and B
  bool pack_pair;               // packed form on CTA pairs
  size_t total;
  TcChoice tcc;
  Layout L;       // the layout the kernels run on: the planned one, or its
  bool blocked;   // blocked row bundle (packed form, block_row_bundle)
};

// The packed form on CTA pairs only under TC_PAIR=1: the pairs cut each SM's
// operand bytes per k-tile by a quarter, but the packed mainloop is bound by
// its MMA issue rather than by those bytes, and the relay of the odd CTA's
// stages to the even CTA's issuer made it slower (4096^3: 0.392 against 0.383
// ms; Section 9's square random contractions: 1.18 against 1.11 ms).
bool packed_pair(const Layout& L, const TcChoice& c, int sms) {
  (void)c;
  (void)sms;
  return pair_setting() == 2 && L.m > 128;
}

// A problem's descriptor fields that the access plan reads.
DevProblem access_problem(const Planned& p, const TcChoice& c) {
  DevProblem d;
  std::memset(&d, 0, sizeof d);
  d.a = p.a;
  d.b = p.b;
  d.a_kc = p.info.a_k_contig;
  d.b_kc = p.info.b_k_contig;
  d.bn = c.bn;
  d.tiles_n = (int32_t)((p.L.n + c.bn - 1) / c.bn);
  d.splits = c.splits;
  return d;
}

// The packed form of the tensor-core mainloop: always under TC_ACCESS_PACKED;
// under TC_ACCESS_AUTO for contractions of at least 2^26 multiply-adds, unless
// both operands are boxes and one of them has a single row (column) of output
// tiles across from it.  Packing an operand costs one read of it through its
// scatter vectors and one write and one read of its packed units; it pays
// wherever the operand is re-read by several tiles or would be gathered (the
// packing kernel, with many small CTAs per SM, gathers faster than the
// mainloop's loader warps do), and also spares the mainloop its converters.
// Measured on GB300: the 4096^3 contraction 0.53 -> 0.46 ms (boxes before),
// Section 9's square and rank-k random contractions 6.0 -> 1.3 and 7.0 -> 1.8
// ms (gathers before); the two gradient contractions whose 268 MB operand
// is a box read by one column of tiles 0.09 -> 0.17 and 0.10 -> 0.35 ms,
// hence the exception.
bool packed_form(const Planned& p, const TcChoice& c) {
  const Layout& L = p.L;
  if (L.m <= 0 || L.n <= 0 || L.k <= 0) return false;
  const int acc = access_setting();
  if (acc == TC_ACCESS_PACKED) return true;
  if (acc != TC_ACCESS_AUTO) return false;
  if ((double)L.m * (double)L.n * (double)L.k < 67108864.0) return false;
  const int64_t tm = (L.m + 127) / 128, tn = (L.n + c.bn - 1) / c.bn;
  if (tm > 1 && tn > 1) return true;
  DevProblem d = access_problem(p, c);
  plan_single_access(L, d, nullptr, sm_count());
  return !(d.boxA.rank > 0 && d.boxB.rank > 0);
}

WsLayout ws_layout(const Planned& p, tc_mode mode) {
  WsLayout w;
  w.L = p.L;
  w.blocked = false;
  w.partial_bytes = 0;
  w.pack_bytes = 0;
  w.pack_pair = false;
  w.tcc = TcChoice{128, 1, 0};
  if (mode != TC_MODE_F64 && p.L.k > 0) {
    // TC_FORCE_BN (16..128, step 16) pins the tile width, for tests and
    // tuning experiments
    int force = 0;
    if (const char* e = std::getenv("TC_FORCE_BN")) {
      const int v = std::atoi(e);
      if (v >= 16 && v % 16 == 0 && v <= tc_bn_max()) force = v;
    }
    const int pieces = mode == TC_MODE_BF16X6 ? 3 : 2;
    w.tcc = choose_tc(p.L, pieces, sm_count(), force);
    if (packed_form(p, w.tcc)) {
      w.pack_pair = packed_pair(p.L, w.tcc, sm_count());
      // single-CTA packed tiles: rows blocked 16 x 8 where A's and C's
      // unit strides lie in different row dims (the packing then reads A in
      // runs of eight, the epilogue writes C in runs of sixteen)
      Layout lb;
      if (!w.pack_pair && block_row_bundle(p.L, p.info.a_k_contig != 0, &lb)) {
        w.L = lb;
        w.blocked = true;
        w.tcc = choose_tc(w.L, pieces, sm_count(), force);
      }
      w.pack_bytes = tc_pack_bytes(w.L.m, w.L.n, w.L.k, w.tcc.bn, pieces, w.pack_pair);
    }
    if (w.tcc.splits > 1)
      w.partial_bytes = align_up((size_t)w.tcc.splits * w.L.m * w.L.n * sizeof(float), 256);
  }
  const ScatterOffsets o = scatter_offsets(w.L, kBsBlock);
  w.scatter_off = 0;
  w.scatter_bytes = align_up((size_t)o.total * sizeof(int64_t), 256);
  w.partial_off = w.scatter_bytes;
  if (mode == TC_MODE_F64 && p.L.k > 0) {
    const int sms = sm_count();
    if (f64_grid(p.L.m, p.L.n, p.L.k, sms, true) != f64_grid(p.L.m, p.L.n, p.L.k, 0, false))
      w.partial_bytes = align_up(f64_partial_bytes(sms), 256);
  }
  w.pack_off = w.scatter_bytes + w.partial_bytes;
  w.total = w.pack_off + w.pack_bytes;
  return w;
}

int plan_checked(tc_dtype dt, const tc_tensor* A, const tc_tensor* B, const tc_tensor* C,
                 Planned* p) {
  int rc = plan_problem(A, B, C, p);
  if (rc != TC_OK) return rc;
  if (tc::aliases(A, B, C, elem_size(dt))) return TC_ERR_OVERLAP;
  return TC_OK;
}

int run_planned(tc_dtype dt, tc_mode mode, double alpha, double beta, const Planned& p,
                void* ws, size_t ws_bytes, cudaStream_t s) {
  if (p.L.m == 0 || p.L.n == 0) return TC_OK;
  const WsLayout w = ws_layout(p, mode);
  const Layout& L = w.L;  // the planned layout, or its blocked row bundle
  if (ws_bytes < w.total || (w.total > 0 && ws == nullptr) ||
      (reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
    return TC_ERR_WORKSPACE;
  int64_t* scat = reinterpret_cast<int64_t*>(static_cast<char*>(ws) + w.scatter_off);
  const ScatterOffsets o = scatter_offsets(L, kBsBlock);
  if (launch_build_scatter(L, kBsBlock, scat, s) != cudaSuccess) return TC_ERR_CUDA;
  // checks on: validate the vectors, and let every later kernel skip its work
  // once the error word holds a bounds error
  const int32_t* gate = nullptr;
  if (checks_on()) {
    int32_t* e = err_word();
    // the ranges come from the planned layout (a blocked bundle's dims reach
    // past the operand only at its holes)
    if (!e || launch_check_scatter(L, kBsBlock, scat, check_bounds(p.L), e, s) != cudaSuccess)
      return TC_ERR_CUDA;
    gate = e;
  }
  const ScatterPtrs sp = scatter_ptrs(scat, o);
  if (L.k == 0 || alpha == 0.0)
    return launch_scale_c(dt, p.c, sp, L.m, L.n, beta, s, gate) == cudaSuccess ? TC_OK : TC_ERR_CUDA;
  if (mode != TC_MODE_F64) {
    TcLaunch q;
    std::memset(&q, 0, sizeof q);
    DevProblem& d = q.single;
    d.a = p.a;
    d.b = p.b;
    d.c = p.c;
    d.partial = w.tcc.splits > 1 ? static_cast<char*>(ws) + w.partial_off : nullptr;
    d.sp = sp;
    d.m = L.m;
    d.n = L.n;
    d.k = L.k;
    d.alpha = alpha;
    d.beta = beta;
    d.a_kc = p.info.a_k_contig;
    d.b_kc = p.info.b_k_contig;
    d.bn = w.tcc.bn;
    d.tiles_n = (int32_t)((L.n + d.bn - 1) / d.bn);
    d.splits = w.tcc.splits;
    d.kps = w.tcc.kps;
    plan_single_access(L, d, q.tm, sm_count());
    q.pieces = mode == TC_MODE_BF16X6 ? 3 : 2;
    q.reduce_f64 = split_reduction_f64() ? 1 : 0;
    q.pack_ws = w.pack_bytes > 0 ? static_cast<char*>(ws) + w.pack_off : nullptr;
    if (q.pack_ws) d.pair = w.pack_pair ? 1 : 0;
    d.rows_blocked = w.blocked ? 1 : 0;
    q.ctas = sm_count();
    q.err = err_word();
    q.gate = gate;
    if (log_enabled())
      std::fprintf(stderr,
                   "[libtc] contract: %s data, %s, m=%lld n=%lld k=%lld, tile %dx%d, %d k-split(s), "
                   "access %s%s%s%s\n",
                   dt == TC_F64 ? "f64" : "f32", mode == TC_MODE_BF16X6 ? "bf16x6" : "bf16x3",
                   (long long)L.m, (long long)L.n, (long long)L.k, d.pair ? 256 : 128, d.bn,
                   d.splits, q.pack_ws ? "packed units" : d.boxA.rank > 0 ? "TMA boxes"
                                        : d.elem_gather ? "element gathers" : "block gathers",
                   d.pair ? " on CTA pairs" : "", w.blocked ? ", rows blocked 16 x 8" : "",
                   gate ? ", checked" : "");
    // TC_FAULT=timeout: test hook that makes the kernel's first wait expire
    if (const char* f = std::getenv("TC_FAULT")) q.fault = std::strcmp(f, "timeout") == 0 ? 1 : 0;
    return launch_tc(q, s) == cudaSuccess ? TC_OK : TC_ERR_CUDA;
  }
  F64Launch f;
  f.dtype = dt;
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
  f.partial = w.partial_bytes ? reinterpret_cast<double*>(static_cast<char*>(ws) + w.partial_off)
                              : nullptr;
  f.max_ctas = sm_count();
  f.err = err_word();
  f.gate = gate;
  if (log_enabled())
    std::fprintf(stderr, "[libtc] contract: %s data, f64, m=%lld n=%lld k=%lld, %s%s\n",
                 dt == TC_F64 ? "f64" : "f32", (long long)L.m, (long long)L.n, (long long)L.k,
                 f64_grid(L.m, L.n, L.k, f.max_ctas, f.partial != nullptr) ==
                         f64_grid(L.m, L.n, L.k, 0, false)
                     ? "plain tiling"
                     : "stream-K over one CTA per SM",
                 gate ? ", checked" : "");
  return launch_f64(f, s) == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

}  // namespace tc

using namespace tc;


extern "C" {

int tc_version(void) { return 100; }

const char* tc_status_string(int status) {
  switch (status) {
    case TC_OK: return "ok";
    case TC_ERR_ARG: return "invalid argument";
    case TC_ERR_LABEL: return "invalid labels (each label must appear in exactly two tensors)";
    case TC_ERR_EXTENT: return "mismatched extents for a shared label";
    case TC_ERR_OVERLAP: return "C overlaps itself or aliases A/B";
    case TC_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case TC_ERR_CUDA: return "CUDA runtime error";
    case TC_ERR_DEVICE_TIMEOUT: return "device-side bounded wait expired";
    case TC_ERR_UNSUPPORTED: return "unsupported dtype/mode combination";
    case TC_ERR_DEVICE_BOUNDS: return "device-side offset outside an operand";
    case TC_ERR_SCRATCH_LIMIT: return "problem exceeds the fixed scratch of tc_contract_noalloc";
    default: return "unknown status";
  }
}

int tc_plan_describe(const tc_tensor* A, const tc_tensor* B, const tc_tensor* C,
                     tc_plan_info* info) {
  if (!info) return TC_ERR_ARG;
  Planned p;
  int rc = plan_problem(A, B, C, &p);
  if (rc != TC_OK) return rc;
  *info = p.info;
  return TC_OK;
}

int tc_workspace_size(tc_dtype dtype, tc_mode mode, const tc_tensor* A, const tc_tensor* B,
                      const tc_tensor* C, size_t* bytes) {
  if (!bytes) return TC_ERR_ARG;
  int rc = check_modes(dtype, mode);
  if (rc != TC_OK) return rc;
  Planned p;
  if ((rc = plan_problem(A, B, C, &p)) != TC_OK) return rc;
  *bytes = (p.L.m == 0 || p.L.n == 0) ? 0 : ws_layout(p, mode).total;
  return TC_OK;
}

int tc_contract(tc_dtype dtype, tc_mode mode, double alpha, const tc_tensor* A,
                const tc_tensor* B, double beta, const tc_tensor* C, void* workspace,
                size_t ws_bytes, void* stream) {
  NvtxRange range("tc_contract");
  int rc = check_modes(dtype, mode);
  if (rc != TC_OK) return rc;
  Planned p;
  if ((rc = plan_checked(dtype, A, B, C, &p)) != TC_OK) return rc;
  return run_planned(dtype, mode, alpha, beta, p, workspace, ws_bytes,
                     static_cast<cudaStream_t>(stream));
}

int tc_box_access(tc_dtype dtype, tc_mode mode, const tc_tensor* A, const tc_tensor* B,
                  const tc_tensor* C, int32_t* a_box, int32_t* b_box) {
  if (!a_box || !b_box) return TC_ERR_ARG;
  int rc = check_modes(dtype, mode);
  if (rc != TC_OK) return rc;
  if (mode == TC_MODE_F64) return TC_ERR_UNSUPPORTED;
  Planned p;
  if ((rc = plan_problem(A, B, C, &p)) != TC_OK) return rc;
  const WsLayout w = ws_layout(p, mode);
  DevProblem d = access_problem(p, w.tcc);
  CUtensorMap maps[2];
  if (w.pack_bytes == 0)  // the packed form reads no boxes
    plan_single_access(p.L, d, box_encoder_available() ? maps : nullptr, sm_count());
  *a_box = d.boxA.rank > 0;
  *b_box = d.boxB.rank > 0;
  return TC_OK;
}

int tc_operand_form(tc_dtype dtype, tc_mode mode, const tc_tensor* A, const tc_tensor* B,
                    const tc_tensor* C, int32_t* form) {
  if (!form) return TC_ERR_ARG;
  int rc = check_modes(dtype, mode);
  if (rc != TC_OK) return rc;
  if (mode == TC_MODE_F64) return TC_ERR_UNSUPPORTED;
  Planned p;
  if ((rc = plan_problem(A, B, C, &p)) != TC_OK) return rc;
  const WsLayout w = ws_layout(p, mode);
  if (w.pack_bytes > 0) {
    *form = TC_FORM_PACKED;
    return TC_OK;
  }
  DevProblem d = access_problem(p, w.tcc);
  CUtensorMap maps[2];
  plan_single_access(p.L, d, box_encoder_available() ? maps : nullptr, sm_count());
  *form = d.boxA.rank > 0 && d.boxB.rank > 0 ? (d.pair ? TC_FORM_PAIR : TC_FORM_BOX)
                                             : TC_FORM_GATHER;
  return TC_OK;
}

int tc_scatter_count(const tc_tensor* A, const tc_tensor* B, const tc_tensor* C, int32_t b,
                     int64_t* count) {
  if (!count || b <= 0) return TC_ERR_ARG;
  Planned p;
  int rc = plan_problem(A, B, C, &p);
  if (rc != TC_OK) return rc;
  *count = scatter_offsets(p.L, b).total;
  return TC_OK;
}

int tc_build_scatter(const tc_tensor* A, const tc_tensor* B, const tc_tensor* C, int32_t b,
                     int64_t* out, int64_t count, void* stream) {
  if (b <= 0) return TC_ERR_ARG;
  Planned p;
  int rc = plan_problem(A, B, C, &p);
  if (rc != TC_OK) return rc;
  const ScatterOffsets o = scatter_offsets(p.L, b);
  if (count < o.total || (o.total > 0 && !out)) return TC_ERR_WORKSPACE;
  return launch_build_scatter(p.L, b, out, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? TC_OK
             : TC_ERR_CUDA;
}

int tc_set_mainloop_events(void* before, void* after) {
  tc::t_ev_before = static_cast<cudaEvent_t>(before);
  tc::t_ev_after = static_cast<cudaEvent_t>(after);
  return TC_OK;
}

uint64_t tc_launch_count(void) { return tc::g_launches.load(); }

int tc_get_device_error(void* stream, int32_t* code) {
  if (!code) return TC_ERR_ARG;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return TC_ERR_CUDA;
  int32_t* w = err_word();
  if (!w) return TC_ERR_CUDA;
  int32_t v = 0;
  if (cudaMemcpy(&v, w, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return TC_ERR_CUDA;
  const int32_t zero = 0;
  if (cudaMemcpy(w, &zero, sizeof zero, cudaMemcpyHostToDevice) != cudaSuccess) return TC_ERR_CUDA;
  // a bounds error outranks a timeout (the check kernels raise the word to it)
  *code = v == kDevOk        ? TC_OK
          : v == kDevTimeout ? TC_ERR_DEVICE_TIMEOUT
          : v == kDevBounds  ? TC_ERR_DEVICE_BOUNDS
                             : TC_ERR_CUDA;
  return TC_OK;
}

}  // extern "C"
