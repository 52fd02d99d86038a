/*
 * tc.h -- C ABI of the transposition-free tensor contraction library (libtc).
 *
 * The operation (Section 4, eq. (gen-contraction); alpha/beta as in Section 3):
 *
 *   C[pi_C(I J)] := alpha * sum_P A[pi_A(I P)] * B[pi_B(P J)] + beta * C[pi_C(I J)]
 *
 * The I bundle holds the labels shared by A and C, J those shared by B and C,
 * P those shared by A and B (Section 4).  The contraction runs as a matrix
 * multiplication C_{IJ} = A_{IP} B_{PJ} directly on the tensors' own layouts
 * through scatter and block-scatter vectors (Sections 6.1-6.2); no operand is
 * transposed or copied.
 *
 * Conventions for every entry point:
 *  - Strides and lengths are in ELEMENTS.  A data pointer addresses the element
 *    whose indices are all zero.  A and B may have any int64 strides (negative
 *    or zero included); C must not overlap itself.
 *  - Labels are single bytes, one per dimension, unique within a tensor; every
 *    label must appear in exactly two of A, B, C, with one extent.
 *  - All data pointers are DEVICE pointers owned by the caller.  The library
 *    keeps no pointer after a call returns, except that a tc_plan keeps copies
 *    of its problem descriptors (and a device buffer of its own, see below).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued asynchronously; a return of TC_OK means the launches were issued.
 *  - Errors are returned as negative codes (never thrown, never aborting);
 *    device-side faults detected by the kernels (bounded waits that expired,
 *    offsets outside an operand) are reported by tc_get_device_error.
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TC_API __attribute__((visibility("default")))
#else
#define TC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define TC_MAX_RANK 16

/* Element type of A, B and C (all three share it). */
typedef enum { TC_F64 = 0, TC_F32 = 1 } tc_dtype;

/* Arithmetic:
 *  TC_MODE_F64    -- products and sums in FP64 (F32 data is widened on load);
 *  TC_MODE_BF16X3 -- F32 data only: each operand split as x = hi + lo with
 *                    hi = RN_bf16(x), lo = RN_bf16(x - hi); hi*hi + hi*lo + lo*hi
 *                    on the tensor cores with FP32 accumulation, split-K
 *                    partials summed with compensated (two-sum) FP32
 *                    arithmetic.  Two bf16 pieces hold 16 of
 *                    FP32's 24 significand bits: a single product can be off
 *                    by up to about 3 * 2^-16 of |a||b|.
 *  TC_MODE_BF16X6 -- as BF16X3 with three pieces x = b0 + b1 + b2 (exact for
 *                    normal FP32 values) and the six products b_i*b_j with
 *                    i + j <= 2: per-product error about 2^-22, at twice the
 *                    tensor-core work. */
typedef enum { TC_MODE_F64 = 0, TC_MODE_BF16X3 = 1, TC_MODE_BF16X6 = 2 } tc_mode;

enum {
  TC_OK = 0,
  TC_ERR_ARG = -1,            /* null pointer, rank > TC_MAX_RANK, negative length, bad enum */
  TC_ERR_LABEL = -2,          /* label repeated in a tensor, or not in exactly two tensors */
  TC_ERR_EXTENT = -3,         /* one label with two different lengths */
  TC_ERR_OVERLAP = -4,        /* C overlaps itself */
  TC_ERR_WORKSPACE = -5,      /* workspace missing, too small or misaligned */
  TC_ERR_CUDA = -6,           /* a CUDA runtime call failed */
  TC_ERR_DEVICE_TIMEOUT = -7, /* a kernel's bounded wait expired (device error word) */
  TC_ERR_UNSUPPORTED = -8,    /* combination not provided (e.g. BF16X3 on F64 data) */
  TC_ERR_DEVICE_BOUNDS = -9,  /* checked launch: a scatter vector reached outside its operand */
  TC_ERR_SCRATCH_LIMIT = -10  /* tc_contract_noalloc: problem needs more than its fixed scratch */
};

/* One tensor operand: `rank` dimensions with lengths `len[d]` >= 0, strides
 * `stride[d]` (elements) and labels `labels[d]` (rank nonzero bytes, distinct
 * within the tensor, not necessarily NUL-terminated; TC_ERR_LABEL otherwise).
 * rank 0 is a scalar.  All arrays are host memory, read only
 * during the call. */
typedef struct {
  int32_t rank;
  const int64_t* len;
  const int64_t* stride;
  const char* labels;
  void* data;
} tc_tensor;

/* One contraction of a batch. */
typedef struct {
  double alpha, beta;
  tc_tensor A, B, C;
} tc_problem;

/* Host-side description of how a contraction is laid out as a matrix
 * multiplication (Section 7.3: length-one dims dropped, sequentially contiguous
 * dims folded, I and J sorted by stride in C, A<->B swapped when C's unit
 * stride is in J, P sorted by stride in A).  After a swap, "A" and "B" below
 * name the operands in their matrix roles (A is the caller's B). */
typedef struct {
  int32_t swapped;                 /* 1 if the caller's A and B were exchanged */
  int32_t nI, nJ, nP;              /* folded dimensions per bundle */
  int64_t m, n, k;                 /* products of the bundle lengths */
  int64_t I_len[TC_MAX_RANK], I_sA[TC_MAX_RANK], I_sC[TC_MAX_RANK];
  int64_t J_len[TC_MAX_RANK], J_sB[TC_MAX_RANK], J_sC[TC_MAX_RANK];
  int64_t P_len[TC_MAX_RANK], P_sA[TC_MAX_RANK], P_sB[TC_MAX_RANK];
  /* For each folded dim, the caller's labels it covers (NUL-terminated). */
  char I_labels[TC_MAX_RANK][TC_MAX_RANK + 1];
  char J_labels[TC_MAX_RANK][TC_MAX_RANK + 1];
  char P_labels[TC_MAX_RANK][TC_MAX_RANK + 1];
  /* Access plan (Section 7.3, stride-1 preference): 1 if the operand's
   * smallest |stride| lies along K (A, B) or along M (C). */
  int32_t a_k_contig, b_k_contig, c_m_contig;
} tc_plan_info;

/* Opaque batched plan. */
typedef struct tc_plan tc_plan;

/* ---- planning (host only, no GPU needed) -------------------------------- */

/* Validate and lay out a contraction (Sections 4 and 7.3) without launching
 * anything.  Returns TC_OK and fills *info, or an error code. */
TC_API int tc_plan_describe(const tc_tensor* A, const tc_tensor* B, const tc_tensor* C,
                     tc_plan_info* info);

/* Device workspace in bytes that tc_contract needs for this problem: the
 * scatter and block-scatter vectors, O(m + n + k) (Sections 6.1-6.3), plus
 * split-K or stream-K partial tiles where the tile scheduler uses them.  Never
 * an operand-sized copy.  Alignment: 256 bytes. */
TC_API int tc_workspace_size(tc_dtype dtype, tc_mode mode, const tc_tensor* A, const tc_tensor* B,
                      const tc_tensor* C, size_t* bytes);

/* ---- the contraction -------------------------------------------------------- */

/* C := alpha * A.B + beta * C, in place on the caller's layouts (Section 4,
 * Section 6.2's block-scatter-matrix algorithm mapped onto GPU tiles).
 * beta == 0: C is only written (NaN in C does not propagate); alpha == 0 or an
 * empty contracted range: C := beta * C.  `workspace` must hold at least
 * tc_workspace_size bytes, 256-byte aligned (may be NULL if that size is 0).
 * Asynchronous on `stream`. */
TC_API int tc_contract(tc_dtype dtype, tc_mode mode, double alpha, const tc_tensor* A,
                const tc_tensor* B, double beta, const tc_tensor* C, void* workspace,
                size_t ws_bytes, void* stream);

/* ---- batches ------------------------------------------------------------------ */

/* Workspace for tc_contract_batched over the same problems. */
TC_API int tc_batched_workspace_size(tc_dtype dtype, tc_mode mode, int32_t count,
                              const tc_problem* probs, size_t* bytes);

/* Run `count` independent contractions of possibly different ranks, extents,
 * strides and labels in one persistent launch per tile shape (one on the
 * tensor cores; on the FP64 path one for each of the 64 x 64, 32 x 64 and
 * 64 x 32 tiles the problems are given), plus one launch building all scatter
 * vectors and one reduction launch for problems split along k.  The
 * persistent CTAs claim work items (output tile x k-split, longest first)
 * from a device counter reset before each launch.  Equivalent to calling
 * tc_contract on each problem.  Problems must not write overlapping
 * C elements.  Creates and destroys a temporary plan (allocates and frees a
 * small device descriptor buffer; synchronises `stream` before freeing it). */
TC_API int tc_contract_batched(tc_dtype dtype, tc_mode mode, int32_t count, const tc_problem* probs,
                        void* workspace, size_t ws_bytes, void* stream);

/* Plan form for repeated batches: tc_plan_create validates and plans every
 * problem, chooses tiles and k-splits, and copies the descriptors into a
 * device buffer that the plan owns (cudaMalloc at create, cudaFree at
 * destroy).  Autotuning (on with TC_AUTOTUNE=1, or whenever the environment
 * names a cache file in TC_AUTOTUNE_CACHE, unless TC_AUTOTUNE=0): per shape
 * class (rounded log2 of m, n, k and the access flags) the output tile is
 * chosen by timing the candidates on one SM's worth of CTAs, and per batch the
 * balance divisor D of the k-split rule by timing the whole batch with each of
 * 2, 4, 8 and 16; the timed runs write scratch copies of the outputs (the
 * caller's C is not touched) and their results are kept for the process and
 * in the cache file.  Untuned: least-padding FP64 tiles, tensor-core tiles
 * covering n, D = 4.  The plan's scatter vectors (K1) depend on the layouts
 * alone: tc_plan_create builds them on the device, on the legacy default
 * stream (a packed plan also decodes its work items there, once), and
 * returns once they are built.  tc_plan_execute only enqueues
 * work -- the device-side checks if they were on at creation, the packing,
 * mainloop and reduction kernels and the memset of the work counters -- with
 * no host synchronisation and no allocation, so it can be captured in a CUDA
 * graph. */
TC_API int tc_plan_create(tc_dtype dtype, tc_mode mode, int32_t count, const tc_problem* probs,
                   tc_plan** out);
TC_API int tc_plan_workspace_size(const tc_plan* plan, size_t* bytes);
/* What the plan chose for the caller's problem `index` (0-based, as passed to
 * tc_plan_create): out[0] = tile rows, out[1] = tile columns, out[2] = pieces
 * of its contracted range (k-splits), out[3] = the balance divisor D of the
 * batch (a problem is split along k until no work item exceeds 1/D of a CTA's
 * fair share).  A problem with an empty output gets zeros in out[0..2].
 * Host only.  TC_ERR_ARG for a null pointer or an index out of range. */
TC_API int tc_plan_config(const tc_plan* plan, int32_t index, int32_t* out);
/* Mainloop forms of the tensor-core path (tc_operand_form, tc_plan_form). */
typedef enum { TC_FORM_GATHER = 0, TC_FORM_BOX = 1, TC_FORM_PAIR = 2, TC_FORM_PACKED = 3 } tc_form;
/* The mainloop form of a tensor-core plan (tc_form): TC_FORM_PACKED when the
 * plan packs every problem's A and B before its mainloop (tc_set_access), else
 * TC_FORM_GATHER (batch plans take no boxes).  Host only.
 * TC_ERR_UNSUPPORTED for an FP64 plan, TC_ERR_ARG for a null pointer. */
TC_API int tc_plan_form(const tc_plan* plan, int32_t* form);
TC_API int tc_plan_execute(tc_plan* plan, void* workspace, size_t ws_bytes, void* stream);
TC_API void tc_plan_destroy(tc_plan* plan);

/* ---- operand access of the tensor-core mainloop ------------------------------- */

/* How the tensor-core mainloop (BF16X3 / BF16X6 modes) reads A and B into
 * shared memory.  Results are identical, bit for bit, in every setting; only
 * the speed differs.
 * TC_ACCESS_AUTO (default): the packed form (below) for single contractions
 * of at least 2^26 multiply-adds (m n k) unless both operands are boxes and
 * one of them is read by a single row or column of output tiles (packing
 * would add a write and a read of it and save nothing: a box reads it at
 * full speed), and for batch plans of at least 2^26 multiply-adds in all;
 * otherwise as TC_ACCESS_BOX.  tc_operand_form and tc_plan_form report the
 * choice.
 * TC_ACCESS_BOX: when, for both A and B, the tile rows and a k-tile
 * form one box in the operand's own dims -- its unit-stride dim leads the row
 * or the k bundle, the bundle dims before the one a tile ends in are covered
 * whole, and that dim's tile extent divides its length (the last dim of a
 * bundle may run past its end), no box extent exceeds its dim's length, at
 * most 5 dims, FP32 strides that are multiples of 4 elements, 16-byte aligned
 * data -- both are loaded with one TMA box per tile (a regular block in the
 * sense of Section 6.2, in several dims at once, read along the unit stride
 * as Section 7.3 prefers, with no scatter entry); otherwise, and for batches
 * (tc_plan_*, tc_contract_batched), as in TC_ACCESS_BLOCK.
 * TC_ACCESS_BLOCK: gathers through the scatter vectors (Section 6.1), 16
 * bytes at a time wherever the block-scatter vectors (Section 6.2) show four
 * consecutive elements at unit stride: the paper's block-scatter form.
 * TC_ACCESS_SCATTER: the same gathers one element at a time, ignoring the
 * block-scatter vectors: the paper's plain scatter-matrix form, kept for
 * comparison.
 * TC_ACCESS_PACKED: single contractions first pack A and B, once each,
 * through their scatter vectors into bf16 pieces laid out as the tensor core
 * reads them (the packing of BLIS that Sections 5-6 build on: every element
 * gathered once instead of once per output tile across from it); the
 * mainloop then streams the packed units with bulk copies.  The workspace
 * grows by about the bytes of A and B (tc_workspace_size reports it); a
 * batch plan packs every problem in one launch into its own buffer.
 * The FP64 mode always uses the BLOCK form.  The setting is process-wide and
 * read when a contraction is issued or a plan is created; it is not tied to
 * any thread or stream, so a host thread that changes it while another issues
 * contractions races with that thread (either setting may apply to a call
 * issued meanwhile): set it once at start-up, or serialise.  Returns the
 * previous setting, or TC_ERR_ARG for an unknown value. */
typedef enum {
  TC_ACCESS_BOX = 0,
  TC_ACCESS_BLOCK = 1,
  TC_ACCESS_SCATTER = 2,
  TC_ACCESS_PACKED = 3,
  TC_ACCESS_AUTO = 4
} tc_access;
TC_API int tc_set_access(int access);

/* How the tensor-core path sums the FP32 partial results of a contracted
 * range split across CTAs (for parallelism on few output tiles, or for
 * balance in a batch), before alpha/beta and the final FP32 rounding.
 * TC_REDUCE_COMPENSATED (default): error-free transformations on the FP32
 * pipes (Knuth's two-sum, the errors collected once): for up to 64 partials
 * as accurate as an FP64 sum, and faster on GB300, whose FP64 rate is low.
 * TC_REDUCE_F64: each partial widened to FP64, summed and scaled in FP64.
 * Within one tile the tensor core's own FP32 accumulation is summed in
 * float-float chunks of at most 1024 terms in either setting.  Process-wide,
 * read when a contraction is issued or a plan is created, with the same
 * caveat as tc_set_access for host threads that change it concurrently.
 * Returns the previous setting, or TC_ERR_ARG for an unknown value. */
typedef enum { TC_REDUCE_COMPENSATED = 0, TC_REDUCE_F64 = 1 } tc_reduce;
TC_API int tc_set_split_reduction(int reduce);

/* Report how tc_contract would read A and B (matrix roles, as in
 * tc_plan_describe) in tensor-core mode `mode` with the current setting:
 * *a_box, *b_box = 1 for a TMA box per tile, 0 for the scatter gather (both
 * or neither).  Host only; without a CUDA driver it reports the eligibility
 * rules alone (the driver may still refuse a tensor map, and both operands
 * are then gathered).  TC_ERR_UNSUPPORTED for the FP64 mode or F64 data. */
TC_API int tc_box_access(tc_dtype dtype, tc_mode mode, const tc_tensor* A, const tc_tensor* B,
                         const tc_tensor* C, int32_t* a_box, int32_t* b_box);

/* The form the tensor-core mainloop will take for this contraction under the
 * current settings (tc_set_access, TC_PAIR): *form = TC_FORM_GATHER (both
 * operands gathered through their scatter vectors), TC_FORM_BOX (both TMA
 * boxes, one CTA per tile), TC_FORM_PAIR (boxes on CTA pairs) or
 * TC_FORM_PACKED (both packed before the mainloop).  Host only.
 * TC_ERR_UNSUPPORTED for the FP64 mode or F64 data. */
TC_API int tc_operand_form(tc_dtype dtype, tc_mode mode, const tc_tensor* A, const tc_tensor* B,
                           const tc_tensor* C, int32_t* form);

/* ---- scatter vectors (K1 on its own; used by the tests) ------------------------ */

/* Number of int64 entries tc_build_scatter writes for this problem and block
 * size b: 2(m + n + k) scatter entries followed by the six block-scatter
 * vectors. */
TC_API int tc_scatter_count(const tc_tensor* A, const tc_tensor* B, const tc_tensor* C, int32_t b,
                     int64_t* count);

/* Build on the device, into `out` (device, count int64), the scatter vectors of
 * Section 6.1 for the planned bundles and the block-scatter vectors of
 * Section 6.2 with blocking parameter b, in this order:
 *   rscat(A)[m] cscat(A)[k] rscat(B)[k] cscat(B)[n] rscat(C)[m] cscat(C)[n]
 *   rbs(A)[ceil(m/b)] cbs(A)[ceil(k/b)] rbs(B)[ceil(k/b)] cbs(B)[ceil(n/b)]
 *   rbs(C)[ceil(m/b)] cbs(C)[ceil(n/b)]
 * where A and B are the matrix-role operands of tc_plan_describe.  A block
 * entry is its constant stride s > 0, or 0 when the block's stride varies; a
 * one-element block has stride 1. */
TC_API int tc_build_scatter(const tc_tensor* A, const tc_tensor* B, const tc_tensor* C, int32_t b,
                     int64_t* out, int64_t count, void* stream);

/* ---- contraction without any device allocation ------------------------------------ */

/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory at all -- code running while another part of
 * the program captures a CUDA graph, real-time or embedded hosts whose device
 * memory is divided up once at start-up, plug-ins whose host application owns
 * every allocation.
 *
 * Same operation and argument rules as tc_contract in FP64 mode (F64 data, or
 * F32 data widened to FP64), but it takes no workspace and allocates nothing:
 * the scatter and block-scatter vectors live in one fixed array of
 * TC_NOALLOC_SCRATCH_BYTES compiled into the library, which every GPU that
 * loads the library holds until the process exits.  A problem whose vectors
 * need more -- 2(m + n + k) + 2(ceil(m/4) + ceil(n/4) + ceil(k/4)) int64
 * entries after the planner's folding, i.e. m + n + k up to about 104,000 --
 * is rejected with TC_ERR_SCRATCH_LIMIT before anything is launched.
 *
 * The first call on each device looks up the array's device address (with
 * that device current) and caches it; make that first call before any stream
 * capture.  All calls share the one array: calls whose kernels overlap on the
 * GPU (different streams, or different host threads, without ordering between
 * them) race on it and must be serialised by the caller.  Nothing in the array
 * needs to start at zero: each call writes every entry it reads.  The cached
 * address belongs to the device's current context: after a cudaDeviceReset of
 * that device the process must not call this entry point on it again (the
 * library keeps other per-device state the same way).  Device-side faults are
 * reported through tc_get_device_error like every other call. */
#define TC_NOALLOC_SCRATCH_BYTES (2u << 20)
TC_API int tc_contract_noalloc(tc_dtype dtype, double alpha, const tc_tensor* A,
                               const tc_tensor* B, double beta, const tc_tensor* C, void* stream);

/* ---- diagnostics ------------------------------------------------------------------ */

/* Device-side checks, a debugging mode (the paper has none; it stands in for a
 * bounds-checking sanitizer).  With on = 1, every contraction issued and every
 * plan created afterwards (tc_contract, tc_contract_noalloc, tc_plan_create,
 * tc_contract_batched) adds one launch after the scatter-vector builder that
 * verifies what every later address rests on: each entry of each scatter
 * vector (Section 6.1) lies between the least and the largest offset its
 * bundle's dims reach in the operand (computed on the host from the operand's
 * own lengths and strides, so rscat + cscat stays inside the operand), and
 * each block-scatter entry s > 0 (Section 6.2) is the common difference of its
 * block.  A failure raises the device error word to TC_ERR_DEVICE_BOUNDS
 * (tc_get_device_error) without a trap; the mainloop, epilogue and reduction
 * launches of checked work read that word first and do nothing while it holds
 * the bounds error, so no access outside an operand is made and C is left
 * untouched.  The word stays set until tc_get_device_error reads and clears
 * it: until then every checked contraction skips its work.  Process-wide, with
 * the caveat of tc_set_access; a plan keeps the setting it was created with.
 * Results are bit-identical with and without checks.  Returns the previous
 * setting, or TC_ERR_ARG for a value other than 0 or 1. */
TC_API int tc_set_checks(int on);

/* Synchronise `stream`, read and clear the library's device error word.
 * *code is TC_OK, TC_ERR_DEVICE_TIMEOUT or TC_ERR_DEVICE_BOUNDS. */
TC_API int tc_get_device_error(void* stream, int32_t* code);

/* Instrumentation: record the caller's CUDA events `before` and `after`
 * (cudaEvent_t handles, or NULL to stop) on the launching stream immediately
 * before and after the mainloop kernel of the next contraction issued from
 * this host thread (tc_contract or tc_plan_execute); the pair is used once and
 * then cleared.  Lets a caller time the dominant kernel alone. */
TC_API int tc_set_mainloop_events(void* before, void* after);

/* Number of kernels libtc has launched in this process so far. */
TC_API uint64_t tc_launch_count(void);

/* Static string for a status code. */
TC_API const char* tc_status_string(int status);

/* Library version (major*10000 + minor*100 + patch). */
TC_API int tc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TC_H */
