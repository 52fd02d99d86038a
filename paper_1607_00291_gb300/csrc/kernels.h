// Launch wrappers of the device kernels (one translation unit each).
#pragma once

#include <cuda.h>  // CUtensorMap (the type only; the encoder is looked up at run time)
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
// `gate`: see CheckBounds (null when the checks are off).
cudaError_t launch_scale_c(tc_dtype dt, void* c, const ScatterPtrs& sp, int64_t m, int64_t n,
                           double beta, cudaStream_t s, const int32_t* gate = nullptr);

// ---- device-side checks (tc_set_checks) ----------------------------------------------
// Every global address the mainloops and the epilogue compute from the scatter
// vectors is rscat[i] + cscat[j] (Section 6.1); a 16-byte copy at a block the
// block-scatter vector marks as unit stride reads the four entries of that
// block (Section 6.2).  With checks on, a check kernel after K1 verifies that
// every scatter entry lies in its vector's range [lo, hi] -- the least and
// largest offset its bundle's dims can reach, computed on the host from the
// operand's own lengths and strides, so that every rscat + cscat stays inside
// the operand -- and that every block-scatter entry s > 0 is the common
// difference of its block's entries.  A failure sets kDevBounds in the device
// error word (never a trap); every later kernel of a checked launch reads that
// word (its `gate`) first and does nothing when it holds kDevBounds, so no
// access outside an operand is made.
struct CheckBounds {
  int64_t lo[6], hi[6];  // per scatter vector, in the order rA cA rB cB rC cC
};
bool checks_on();      // the process-wide setting of tc_set_checks
CheckBounds check_bounds(const Layout& L);  // also applies the TC_CHECK_SHRINK test hook
cudaError_t launch_check_scatter(const Layout& L, int32_t b, const int64_t* scat,
                                 const CheckBounds& cb, int32_t* err, cudaStream_t s);
// A batch: problem p's bounds in cbs[p] (device).
cudaError_t launch_check_scatter_batched(const Layout* layouts, const int64_t* offsets,
                                         const CheckBounds* cbs, int32_t count, int64_t total,
                                         int32_t b, const int64_t* scat, int32_t* err,
                                         cudaStream_t s);

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
  const int32_t* gate = nullptr;  // checked launch: skip all work if *gate == kDevBounds
};
cudaError_t launch_f64(const F64Launch& p, cudaStream_t s);
int64_t f64_grid(int64_t m, int64_t n, int64_t k, int64_t max_ctas, bool can_split);
size_t f64_partial_bytes(int64_t max_ctas);
int f64_tile_m();
int f64_tile_n();
int f64_tile_k();
// tiles and resident CTAs per SM of the batched FP64 kernel
// FP64 batch tile classes: class c computes f64_batch_tile(c) = bm x bn tiles
// in its own persistent launch of f64_batch_ctas_per_sm(c) CTAs per SM.
constexpr int kF64BatchClasses = 3;
void f64_batch_tile(int cls, int* bm, int* bn);
int f64_batch_ctas_per_sm(int cls);

// Access plan of one operand of the tensor-core mainloop (Section 7.3's
// preference for unit-stride access, in the GPU's terms).  When the rows of a
// tile and a k-tile of the operand form a box in the operand's own dims -- its
// unit-stride dim leads one bundle, every bundle dim before the one the tile
// ends in is covered whole, and that dim's tile extent divides its length (the
// bundle's last dim may run past its end: the box reads zeros there) -- the
// tile is one TMA box load: like a regular block of Section 6.2, but in
// several dims at once, every address follows from the box's corner and the
// operand's own strides, so no scatter entry is read.  Otherwise (rank == 0)
// the loaders gather it through its scatter vectors.
struct BoxAccess {
  int32_t rank;     // dims of the tensor map, 2..5 (0: gather)
  int32_t nfirst;   // dims of the bundle that leads the map (the one holding the unit stride)
  int32_t kfirst;   // that bundle is the k bundle (else the row bundle)
  int32_t bytes;    // bytes one box delivers
  int32_t len[5];   // extents in map order: each bundle fastest dim first
  int32_t klast;    // map index of the k bundle's last dim
  int32_t kstep_dim, kstep;  // the next k-tile's box: coordinate kstep_dim + kstep,
                             // then carries (the dims before it are covered whole)
};
// Fill d.boxA / d.boxB / d.elem_gather for the tensor-core mainloop from the
// process-wide access setting (tc_set_access) and the problem's layout,
// operands, access flags and tile width, and encode the tensor maps of the
// operands that take boxes into maps[0] (A) and maps[1] (B); with maps ==
// null only the eligibility is decided; allow_box = false keeps every operand
// gathered; pair = true plans B's boxes bn / 2 columns wide (the pair form)
// and sets d.pair when both operands take boxes.  Defined in access.cu.
struct DevProblem;
void plan_access(const Layout& L, DevProblem& d, CUtensorMap* maps, bool allow_box = true,
                 bool pair = false);
bool box_encoder_available();  // the driver's tensor-map encoder could be found
int access_setting();           // the process-wide tc_set_access value
// The process-wide split-reduction setting (tc_set_split_reduction): true for FP64.
bool split_reduction_f64();

// One planned contraction as the persistent kernels see it: a kernel
// parameter for a single call, an array in device memory for a batch.
struct DevProblem {
  const void* a;
  const void* b;
  void* c;
  void* partial;    // split partial sums, [splits][n][m] (FP32 on the tensor-core
                    // path, FP64 on the FP64 path); null when splits == 1
  ScatterPtrs sp;
  int64_t m, n, k;
  double alpha, beta;
  int32_t a_kc, b_kc;
  int32_t tiles_n;  // output tiles along n
  int32_t bn;       // n-width of an output tile (tensor-core path: 16..256, step 16)
  int32_t splits;   // pieces of the contracted range
  int32_t elem_gather;  // tensor-core path: gather element by element, ignoring the
                        // block-scatter vectors (the plain scatter-matrix form)
  int32_t pair;     // tensor-core box form on CTA pairs (cta_group::2): 256-row tiles,
                    // each CTA of the pair loading its 128 rows of A and half of B's
                    // columns (boxB then covers bn / 2 columns)
  int64_t kps;      // contracted indices per split (a multiple of the k-tile)
  int32_t rows_blocked;  // packed form: the row bundle is blocked 16 x 8 (block_row_bundle);
                         // its scatter entries may be kHole
  int32_t pad_;
  BoxAccess boxA, boxB;       // tensor-core path: TMA boxes or gathers per operand
  const CUtensorMap* tmaps;   // batch: the two tensor maps in device memory (a single
                              // call passes them as kernel parameters instead)
  const uint8_t* pa;          // packed form: A's units [ceil(m/128)][ceil(k/32)] and
  const uint8_t* pb;          // B's [tiles_n][ceil(k/32)], each all pieces of 128 (bn)
                              // rows x 32 k in the tensor core's K-major layout
};

// One operand of one problem to pack (the packed form): `units` units of R
// rows x 32 k, row tile by row tile, k-tile by k-tile, from x through its row
// scatter vector rs and its scatter vector along the contracted range ks
// (kbs: its block-scatter vector, blocks of four).  The packing launch hands
// out groups of G consecutive units (G units of R rows make a multiple of 256
// tasks of eight values, at least 512: pack_job_groups), `groups` of them.
struct PackJob {
  const float* x;
  const int64_t* rs;  // may hold kHole entries (a blocked row bundle): zeros
  const int64_t* ks;
  const int64_t* kbs;
  int64_t rows, k, KT, units, groups;
  int32_t R, G;
  int32_t swz;  // blocked rows (R = 128 = 16 x 8): walk each unit's rows with
                // the eight of one 16-row column consecutive (0: in order)
  int32_t pad;
  uint8_t* out;
};
// Units per group: the fewest whose tasks (R * 4 per unit, one 8-value chunk
// each) fill the packing launch's 256 threads evenly, at least twice over.
inline void pack_job_groups(PackJob& j) {
  const int t = j.R * 4;  // R is a multiple of 8: G <= 16
  int G = 1;
  while ((G * t) % 256 != 0 || G * t < 512) ++G;
  j.G = G;
  j.groups = (j.units + j.G - 1) / j.G;
}

// One unit of work of a batch: an output tile of a problem over one k-split.
struct WorkItem {
  int32_t prob, tile, split, pad;
};

// K3 + K5 (tc_mma.cu): tcgen05 mainloop over bf16 pieces (2 -> BF16x3,
// 3 -> BF16x6), persistent over work items, chunked FP32 accumulation summed
// in float-float; K4 reduces the partials of k-splits (two-sum FP32).
struct TcLaunch {
  CUtensorMap tm[2];          // tensor maps of the single problem's box operands
  DevProblem single;          // the problem of a single call (probs == null)
  const DevProblem* probs;    // batch descriptors (device), or null
  const WorkItem* items;      // batch work list (device), or null
  int64_t nitems;             // work items in the list (batch)
  int32_t nprobs;             // problems in the batch
  int pieces;                 // 2 or 3
  int64_t ctas;               // persistent grid size
  const int32_t* split_probs; // batch: indices of problems with splits > 1 (device)
  const int64_t* split_col_prefix;  // batch: prefix sums of their n (device, n_split + 1)
  int64_t split_cols;         // batch: total columns of the split problems
  int32_t n_split_probs;
  int64_t max_m_split, max_n_split;  // batch: largest m and n among split problems
  int32_t reduce_f64;         // sum the k-split partials in FP64 (else compensated FP32)
  unsigned long long* counter;  // batch: device work counter for dynamic items, or null
  int32_t* err;
  int fault;  // fault injection for tests: 1 makes the MMA warp's first wait
              // expire (bounded), exercising the timeout and unwind path
  const int32_t* gate;  // checked launch: skip all work if *gate == kDevBounds (or null)
  void* pack_ws;  // single problem, packed form: tc_pack_bytes() bytes for the packed
                  // units of A and B (null: the gather or box form)
  const void* pack_items;      // batch, packed form: the work items decoded (launch_decode_items)
  const PackJob* pack_jobs;    // batch, packed form: two jobs per problem (device), or null
  const int64_t* pack_prefix;  // their prefix sums of unit groups (device, pack_njobs + 1)
  int32_t pack_njobs;
  int64_t pack_groups;
};
cudaError_t launch_tc(const TcLaunch& q, cudaStream_t s);
// Workspace of the packed form: A's units (128 rows x 32 k, all pieces; the
// pair form pads them to whole 256-row tiles) then B's (bn rows x 32 k; the
// pair form: two half-tile units of bn / 2 rows, the same bytes), each part
// 256-byte aligned.
size_t tc_pack_bytes(int64_t m, int64_t n, int64_t k, int bn, int pieces, bool pair);
// Packed batches: every work item decoded once, at plan creation, into the
// form the mainloop's roles read (tc_item_bytes() bytes each, 16-byte aligned).
size_t tc_item_bytes();
cudaError_t launch_decode_items(const DevProblem* probs, const WorkItem* items, int64_t n, void* out,
                                cudaStream_t s);

// K6 on the FP64 path (f64.cu): persistent batched mainloop + FP64 reduction
// of split problems.
struct F64BatchLaunch {
  tc_dtype dtype;
  const DevProblem* probs;
  const WorkItem* items;      // the work list, tile class by tile class
  int64_t nitems;
  int64_t class_off[kF64BatchClasses + 1];  // class c: items [class_off[c], class_off[c + 1])
  int64_t sms;
  const int32_t* split_probs;
  const int64_t* split_col_prefix;
  int64_t split_cols;
  int32_t n_split_probs;
  int64_t max_m_split, max_n_split;
  unsigned long long* counter;  // device work counters, one per tile class
  const int32_t* gate = nullptr;  // checked launch: skip all work if *gate == kDevBounds
};
cudaError_t launch_f64_batched(const F64BatchLaunch& q, cudaStream_t s);

// K1 for a batch (scatter.cu): every problem's vectors in one launch.
// layouts[count], offsets[count + 1] (prefix sums of scatter_offsets().total).
cudaError_t launch_build_scatter_batched(const Layout* layouts, const int64_t* offsets,
                                         int32_t count, int64_t total, int32_t b, int64_t* out,
                                         cudaStream_t s);
int tc_bn_max();  // widest output tile of the tensor-core mainloop (columns)
// Most k-tiles (of 32) one work item of the tensor-core mainloop may take:
// its running chunk sum is plain FP32, accurate for that many chunks.
int tc_max_item_ktiles();

}  // namespace tc
