/*
 * ttsketch.h - C ABI of the GB300 (sm_103a) streaming two-sided TT sketch.
 *
 * The operation is PSTT2 / PSTT2-onepass of Shi, Ruth & Townsend, "Parallel
 * algorithms for computing the tensor-train decomposition", Sec. 3.2:
 * given a d-way tensor X (n_1 x ... x n_d), target TT ranks r or a tolerance
 * eps, and an oversampling p, return TT cores G_1..G_d whose contraction X~
 * approximates X with ||X - X~||_F <= eps ||X||_F (eq. (1.1), the problem
 * statement of the paper; with ranks known, Sec. 4.1).
 *
 * Conventions used throughout:
 *  - X is column-major with i_1 fastest (Sec. 2.1); the k-th unfolding X_k is
 *    the same buffer seen as N_k x M_k, N_k = n_1..n_k, M_k = n_{k+1}..n_d.
 *  - d* = ceil(d/2).  Column sketches S_k = X_k Omega_k (k < d*, plus k = d*
 *    in one-pass mode), row sketches R_k = X_k^T Psi_k (k = d*..d-1).
 *  - Omega_k / Psi_k are i.i.d. N(0,1) test matrices regenerated on the fly
 *    from a Philox4x32-10 counter stream keyed by `seed`: never kept across
 *    calls (rows that many tiles read are staged in the workspace for the
 *    duration of one accumulate).
 *  - Cores are FP64, written into ONE caller buffer: core k (1-based) lives
 *    at element offset core_off[k] with the padded shape
 *    rpad[k-1] x n_k x rpad[k], entry (a, i, c) at a + rpad[k-1] (i + n_k c);
 *    entries outside the actual ranks are zero, so the padded cores
 *    represent exactly the same tensor.  Actual ranks go to a device int
 *    array of d+1 entries.  Nothing has to come back to the host, which keeps
 *    every call asynchronous.
 *
 * Pointer kinds: "device" pointers are CUDA device (or managed) memory of the
 * current device; "host" pointers are ordinary host memory.  All calls are
 * asynchronous on `stream` unless stated otherwise; argument errors are
 * returned synchronously; conditions found on the device (a singular
 * least-squares matrix, a rank cap reached) are written to a status word in
 * the workspace and reported by tt_query_status.  The library never traps or
 * aborts the process.
 *
 * Ownership: the caller owns X, the workspace, the core buffer, the rank
 * array and any gradient buffer.  A plan is a host object; it owns no device
 * memory.  No call allocates device memory.  The workspace holds all state
 * between the calls of one decomposition (sketches, bases, factorisations)
 * and stays valid until the next tt_pstt2* call on the same workspace.
 *
 * Sharing a workspace: the workspace also holds a copy of the plan's device
 * tables (shapes and offsets the kernels read).  The library remembers, per
 * workspace address, which plan's tables it holds and re-sends them (a small
 * host-synchronous copy) whenever a plan uses a workspace that last held
 * another plan's, so several plans may take turns on one workspace.  Each
 * such switch ends the saved state of the previous plan there: a streaming
 * decomposition whose workspace another plan used after tt_pstt2_begin, or a
 * backward whose forward state was replaced, is refused with TT_ERR_STATE.
 * Memory freed and allocated again at the same address is a new workspace to
 * the caller but not to the library: call tt_workspace_release(ws) before
 * freeing a workspace (tt_plan_destroy releases every workspace of its plan).
 */
#ifndef TTSKETCH_H
#define TTSKETCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TT_MAXD 16   /* largest supported order d                        */
#define TT_MAXL 64   /* largest supported sketch width l = r + p          */

typedef struct tt_plan_s* tt_plan_t;
typedef void* tt_stream_t; /* a cudaStream_t; NULL means the legacy default stream */

typedef enum {
  TT_OK = 0,
  TT_ERR_INVALID_ARG = 1,     /* bad shape, rank, width, pointer or state      */
  TT_ERR_UNSUPPORTED = 2,     /* valid request this build cannot serve          */
  TT_ERR_CUDA = 3,            /* a CUDA runtime call failed                     */
  TT_ERR_STATE = 4,           /* calls out of order (e.g. slab twice)           */
  TT_ERR_RANK_DEFICIENT = 5,  /* device: B = P^T Omega (one-pass) is singular   */
  TT_ERR_TIMEOUT = 6,         /* device: a bounded wait gave up                 */
  TT_WARN_RANK_CAP = 7,       /* device: eps not met at rmax; cores still valid */
  TT_ERR_NO_DEVICE = 8,       /* no usable CUDA device                          */
  TT_ERR_NONFINITE = 9        /* device: an FP16 plan's sketch holds an inf or  */
                              /* NaN (X non-finite, or |X| 2^s past FP16 range) */
} tt_status;

typedef enum { TT_F32 = 0, TT_F64 = 1 } tt_dtype;

/* Arithmetic of the sketch (the hot loop).  The small solves (QR, least
 * squares, core products) are always FP64.
 *  FP64: FP64 FMA everywhere (the correctness path).
 *  TF32 / BF16 / FP16: tensor cores with FP32 accumulation, flushed into FP64
 *    sketch accumulators.  The test-matrix entries are rounded once to the
 *    MMA type; X is split into a high and a low part of the MMA type (two
 *    products), which keeps the error of the sketch near 2^-22 (TF32) /
 *    2^-17 (BF16) / 2^-22 (FP16) relative instead of 2^-11 / 2^-9 / 2^-11.
 *  FP16 has BF16's cost (16-bit operands, the same MMA rate) and TF32's
 *    resolution, but a narrow range: the split is of X 2^s, s =
 *    x_scale_log2 (a power of two, so the scaling is exact), and the FP64
 *    sketches are scaled back by 2^-s before the bases are formed.  Full
 *    resolution needs 2^-3 <= |X| 2^s < 65520 for the entries that matter:
 *    below 2^-3 the low part is subnormal and the split's error is at most
 *    2^-25 2^-s absolute; at 65520 and above the high part overflows and the
 *    finalize reports TT_ERR_NONFINITE (tt_x_scale_log2 picks s from the
 *    largest |X|).  Of the tensor-core kernels, the sketch adjoint of
 *    tt_pstt2_backward is BF16 / TF32 only: FP16 plans take the SIMT
 *    adjoint (same result, slower). */
typedef enum { TT_PREC_FP64 = 0, TT_PREC_TF32 = 1, TT_PREC_BF16 = 2, TT_PREC_FP16 = 3 } tt_prec;

typedef struct {
  int d;                     /* order, 2 <= d <= TT_MAXD                         */
  int64_t n[TT_MAXD];        /* mode sizes n_1..n_d (n[0..d-1]), each >= 1       */
  double eps;                /* > 0: tolerance mode; == 0: fixed-rank mode       */
  int ranks[TT_MAXD + 1];    /* fixed-rank mode: r_0..r_d, r_0 = r_d = 1         */
  int rmax;                  /* tolerance mode: rank cap (sketch width rmax + p) */
  int p;                     /* oversampling, >= 2 (Theorem 3.3 needs p >= 2)    */
  uint64_t seed;             /* Philox key of the test matrices                  */
  int passes;                /* 1 = PSTT2-onepass (hot path); 2 = PSTT2          */
  tt_dtype x_dtype;          /* storage type of X                                */
  tt_prec prec;              /* arithmetic of the sketch                         */
  int flags;                 /* TT_FLAG_* bits                                   */
  int x_scale_log2;          /* FP16 plans: s, X is split as X 2^s (-100..100);  */
                             /* other precisions ignore it                       */
} tt_problem;

/* Reserve the workspace that tt_reconstruct_backward needs (all left and
 * right interfaces of the train, about 2 r prod(n) / n bytes x 8). */
#define TT_FLAG_DIFF 1
/* One-sided PSTT-onepass instead of the two-sided PSTT2-onepass (Algorithm
 * 2 and the single-pass last core of the paragraph after Theorem 3.3): every
 * unfolding is sketched from the right, S_k = X_k Omega_k (k = 1..d-1, the
 * bases Q_k), plus T_{d-1} = Psi_{d-1}^T X_{d-1}; the cores are eq. (3.1) and
 * G_d = (Psi_{d-1}^T Q_{d-1})^+ T_{d-1}.  With passes = 2 it is Algorithm 2
 * itself: no T_{d-1}, and G_d = Q_{d-1}^T X_{d-1} from a second pass over X
 * (tt_pstt2 only, as for the two-sided two-pass core).  Sketch storage grows
 * to O(l n^{d-1}) (the two-sided form needs O(l n^{ceil(d/2)})).  Requires a
 * single-problem plan; not with TT_FLAG_DIFF (TT_ERR_UNSUPPORTED otherwise). */
#define TT_FLAG_ONESIDED 2
/* Khatri-Rao test matrices (Sec. 3.2, the paragraph after Theorem 3.3,
 * eq. (sketch_orig)) instead of dense i.i.d. Gaussian ones: the test matrix of
 * each sketch is the row-wise Khatri-Rao product of small i.i.d. N(0,1)
 * factors, one n_m x l factor per mode m its rows run over (Omega_k: modes
 * k+1..d; Psi_k: modes 1..k).  Row i of the factor of mode m (1-based) is row
 * i + (2^31 + m) 2^32 of the sketch's Philox stream, so it never coincides
 * with a dense row.  The entry at the column-major multi-index of the modes is
 * the product of the factor entries: for Omega_k multiplied in increasing
 * mode order, for Psi_k in decreasing mode order (in FP64 on the FP64 path;
 * in FP32 from the FP32 generator, then rounded once to the MMA type, on the
 * TF32 / BF16 paths).  One exception on the TF32 / BF16 paths: Psi_{d-1} with
 * d - 1 >= 2 is taken mode by mode, each entry round(F_1) x round(F_{d-1} ..
 * F_2) (the rounded mode-1 factor times the rounded product of the others),
 * so that R_{d-1} = (X^T round(F_1)) scaled per plane -- the form the sketch
 * kernels use.  The factors (sum of n_m l entries per sketch) are staged in
 * the workspace by tt_pstt2 and tt_pstt2_begin.  Single-problem plans only
 * (TT_ERR_UNSUPPORTED in batched plans). */
#define TT_FLAG_KR 4
/* Tensor-core plans (TF32 / BF16 / FP16) on the tcgen05 kernels: flush the
 * FP32 tensor-memory accumulators of the column sketches every 32
 * accumulating MMAs instead of every 256.  Each accumulating MMA adds about
 * 2e-8 relative error (measured on GB300); in the one-pass middle sketch
 * S_{d*} that error enters the cores directly.  On the 256^4 Hilbert-type
 * tensor at eps = 1e-6 (FP16, Khatri-Rao, 1 GiB slabs) it brings ||X - X~||
 * / ||X|| from 2.5e-6 to 8.8e-7 for about 6 % more sketch time (dense test
 * matrices and whole-last-mode launches: 9-14 % more, and the FP64 path's
 * ranks where the default chains take one or two more on the first bond).
 * Other kernels ignore it. */
#define TT_FLAG_SHORT_CHAINS 8

/* ---------------------------------------------------------------- plans */

/* Build a host plan for one problem (Sec. 3.2: split d*, widths l_k = r_k + p
 * or rmax + p, the sketch list, the workspace layout).  Host only; touches no
 * device.  Fixed ranks are clamped to min(N_k, M_k).  On error *out = NULL. */
tt_status tt_sketch_plan(const tt_problem* prob, tt_plan_t* out);

/* Plan for `count` independent problems processed together by the batched
 * calls (one persistent sketch launch over all of them).  Each problem gets
 * its own slice of the workspace, core buffer and rank array. */
tt_status tt_sketch_plan_batched(const tt_problem* probs, int count, tt_plan_t* out);

/* Destroy a plan and forget every workspace it used (tt_workspace_release). */
void tt_plan_destroy(tt_plan_t plan);

/* Forget which plan's tables and state the workspace at `ws` holds (host
 * only; touches no device).  Call it before freeing a workspace that a plan
 * of a live plan object used, so that memory allocated later at the same
 * address is treated as new: the next call on it sends its plan's tables.
 * Unknown addresses and NULL are ignored. */
void tt_workspace_release(const void* ws);

/* Sizes the caller must allocate: workspace bytes (device, 256-byte aligned
 * base) and the number of FP64 entries of the core buffer (all items of a
 * batched plan together).  Any pointer may be NULL. */
tt_status tt_plan_sizes(tt_plan_t plan, size_t* workspace_bytes, int64_t* core_entries,
                        int* rank_entries);

/* Core layout of item `item` (0 for a single plan): core_off[k] for
 * k = 1..d (index 0 unused; offsets are into the whole core buffer) and the
 * padded ranks rpad[0..d].  Host arrays of TT_MAXD + 1 entries. */
tt_status tt_plan_core_layout(tt_plan_t plan, int item, int64_t* core_off, int* rpad);

/* Where sketch number `index` (0-based, in plan order: column sketches
 * k = 1..d*-1, the one-pass middle sketch S_{d*}, then row sketches
 * k = d*..d-1) of item `item` lives in the workspace: FP64, column-major,
 * rows x width at byte offset *byte_off.  type: 0 = column sketch S_k = X_k
 * Omega_k, 1 = row sketch R_k = X_k^T Psi_k.  For tests and inspection; the
 * contents are valid after an accumulate and before the next finalize (the
 * finalize factorises basis sketches in place).  TT_ERR_INVALID_ARG past
 * the last sketch.  During a stream, call tt_pstt2_sync first: the slab
 * kernel stages part of S_{d*}'s partial sums in FP32 and adds them in
 * batches of a few launches. */
tt_status tt_plan_sketch_info(tt_plan_t plan, int item, int index, int* type, int* k, int64_t* rows,
                              int* width, int64_t* byte_off);

/* Which sketch kernel an accumulate of `count_last` last-mode slices runs for
 * item 0: 0 = FP64 SIMT kernel, 1 = generic tensor-core kernel (mma.sync,
 * any shape; in single-problem plans the test-matrix rows that several
 * tiles read are staged once per call, up to 256 MB a sketch), 2 = a tcgen05
 * kernel: the plane kernel (n_1 and count_last in {128, 256}, d in {3, 4},
 * dense Gaussian test matrices, equal widths with 16 <= l * #sketches per
 * side <= 32) or the slab kernel (d = 4, n_1 in {128, 256}, l in {8, 16},
 * count_last = 16, 32 or 64 -- a 1 GiB slab of the 256^4 FP32 tensor is 16 --
 * or, with Khatri-Rao test matrices, any multiple of 64, taken 64 slices a
 * launch), both BF16 or FP16 and two-sided; 3 = small-plane kernel (BF16,
 * FP16 or TF32,
 * n_1 and count_last <= 32, widths l_k <= 32, padded to the widest; mma.sync
 * with test-matrix rows shared by many planes staged once per call).  Host
 * only. */
int tt_sketch_kernel_kind(tt_plan_t plan, int64_t count_last);

/* Problem of item `item` as stored by the plan (ranks clamped). */
tt_status tt_plan_problem(tt_plan_t plan, int item, tt_problem* out);

/* ------------------------------------------------------------ forward */

/* One-shot PSTT2 of X (device, x_dtype, prod(n) entries): zero the sketches,
 * sketch every unfolding in one pass over X (a second pass in two-pass mode),
 * then form the cores (= tt_pstt2_begin + one accumulate of the whole tensor
 * + tt_pstt2_finalize). */
tt_status tt_pstt2(tt_plan_t plan, const void* X, void* ws, double* cores, int* ranks,
                   tt_stream_t stream);

/* Streaming form (one-pass plans only).  begin zeroes the sketches; each
 * accumulate adds the contribution of one slab, a contiguous range
 * [first_last, first_last + count_last) of the LAST mode (device pointer to
 * count_last * N_{d-1} entries), in any order, each index exactly once;
 * finalize forms the cores.  The host checks the slab bookkeeping (a repeated
 * or out-of-range index is TT_ERR_STATE / TT_ERR_INVALID_ARG).  The tensor-
 * core kernels stage test-matrix rows in the workspace during an accumulate,
 * so accumulates on one workspace must not overlap: issue them on one stream
 * (or order them with events). */
tt_status tt_pstt2_begin(tt_plan_t plan, void* ws, tt_stream_t stream);
tt_status tt_pstt2_accumulate(tt_plan_t plan, const void* slab, int64_t first_last,
                              int64_t count_last, void* ws, tt_stream_t stream);
tt_status tt_pstt2_finalize(tt_plan_t plan, void* ws, double* cores, int* ranks,
                            tt_stream_t stream);

/* Checkpoint / resume of a stream (no counterpart in the paper, whose
 * streaming is restartable by construction: the sketch accumulators and the
 * set of slabs already added are the entire state of PSTT2-onepass between
 * slabs, Sec. 4.2).  Single-problem one-pass plans only (TT_ERR_UNSUPPORTED
 * otherwise).
 *   tt_pstt2_state_size: bytes of the state (a header with the problem, the
 *     slab bitmap, every sketch in FP64).
 *   tt_pstt2_export_state: SYNCHRONOUS (waits for `stream`); copies the state
 *     of the stream begun on ws (after tt_pstt2_begin and any accumulates,
 *     before tt_pstt2_finalize) into `host` (host memory, `bytes` >= the
 *     state size).  TT_ERR_STATE when no stream of this plan is open on ws.
 *   tt_pstt2_import_state: SYNCHRONOUS; opens a stream on ws from an exported
 *     state instead of tt_pstt2_begin (any plan object and workspace of the
 *     same problem: every field of the problem must match, else
 *     TT_ERR_INVALID_ARG); then accumulate the remaining slabs and finalize.
 *     The result equals the uninterrupted stream's up to summation order. */
tt_status tt_pstt2_state_size(tt_plan_t plan, size_t* bytes);
/* Complete the sketches of the stream in progress on ws (asynchronous on
 * `stream`): partial sums still staged by the slab kernel are added into
 * the FP64 sketches.  Needed only to read sketches between accumulates
 * (tt_plan_sketch_info); finalize and export do it themselves.  TT_OK
 * without work when no stream of this plan is open on ws. */
tt_status tt_pstt2_sync(tt_plan_t plan, void* ws, tt_stream_t stream);
tt_status tt_pstt2_export_state(tt_plan_t plan, const void* ws, void* host, size_t bytes, tt_stream_t stream);
tt_status tt_pstt2_import_state(tt_plan_t plan, void* ws, const void* host, size_t bytes, tt_stream_t stream);

/* tt_pstt2 without a caller workspace (the paper has no counterpart; this is
 * a library convenience).  For callers that cannot allocate device memory
 * where they call: the workspace is a fixed 32 MiB array inside this library,
 * one per device, so the call allocates nothing.  A plan whose workspace
 * (tt_plan_sizes) exceeds 32 MiB is refused with TT_ERR_UNSUPPORTED before
 * anything runs.  X, cores and ranks are as for tt_pstt2; status_dev, if not
 * NULL, is a device int that receives the device status bits of the call:
 * 1 = rank cap reached (TT_WARN_RANK_CAP), 2 = singular least-squares matrix
 * (TT_ERR_RANK_DEFICIENT), 4 = a bounded wait gave up (TT_ERR_TIMEOUT),
 * 8 = a non-finite sketch entry (TT_ERR_NONFINITE); 0 = no condition.  Nothing has to be zeroed by the
 * caller: the call clears the sketches and the status word itself.
 * The first call on a device sets the array up (it looks up its address) and
 * the first call with a plan sends that plan's tables into it with a
 * host-synchronous copy; make those first calls before any stream capture.
 * The array is shared by every call on the device: calls that can overlap
 * (on different streams or host threads without ordering) race on it and give
 * wrong results; order them.  The saved state stays in the array only until
 * the next call, so tt_pstt2_backward is not available after this call. */
tt_status tt_pstt2_noalloc(tt_plan_t plan, const void* X, double* cores, int* ranks, int* status_dev,
                           tt_stream_t stream);

/* Batched one-pass PSTT2 of many independent tensors (one plan from
 * tt_sketch_plan_batched; not in the paper).  X_ptrs is a HOST array of
 * `count` device pointers, one tensor per item (at most 2048 items, all of one
 * precision; TF32 / BF16 items need FP32 tensors).  The sketches of all items
 * come from ONE persistent launch: CTAs take tiles of every tensor from a work
 * counter in the workspace, the largest tensors first, with the launch shape
 * of the plan (tt_plan_batch_config / tt_plan_autotune).  The bases and cores
 * of all items are formed by launches that each cover every item.  The first
 * call on a workspace sends the plan tables (host-synchronous); after that
 * nothing synchronises with the host, so the call can be captured in a CUDA
 * graph and replayed (the pointers in X_ptrs are fixed at capture). */
tt_status tt_pstt2_batched(tt_plan_t plan, const void* const* X_ptrs, void* ws, double* cores,
                           int* ranks, tt_stream_t stream);

/* Launch shape of the batched sketch: ta = tile rows along i_1 (32 or 64;
 * used by FP64 plans, TF32 / BF16 tiles are 64 rows); for a TF32 / BF16 batch
 * whose items all fit the small-plane kernel (n_1, n_d <= 32) ta is instead
 * the largest number of kR values in a 16-plane block (1, 2, 4 or 8; other
 * values mean 4); chunk = tiles (blocks) a CTA takes from the work counter at
 * a time (>= 1), ctas_per_sm = persistent CTAs per SM (1..32; the small-plane
 * kernel always runs one).  Host only. */
tt_status tt_plan_batch_config(tt_plan_t plan, int ta, int chunk, int ctas_per_sm);

/* Autotuner of the batched sketch (not in the paper): runs the batched
 * decomposition of X_ptrs once, times the batched sketch launch for every
 * candidate shape (ta in {32, 64} for FP64 plans, chunk in {1, 4, 16},
 * ctas_per_sm in {2, 4, 8}; small-plane batches: ta in {1, 2, 4, 8}, chunk
 * in {1, 4, 8}; CUDA events on `stream`, the second of two runs
 * each) and keeps the fastest in the plan, then runs the decomposition once
 * more with it so that cores and ranks hold a valid result.  Synchronises;
 * refused during stream capture (TT_ERR_STATE).  best_out (host, 3 ints, may
 * be NULL) receives the chosen ta, chunk and ctas_per_sm.  With the
 * environment variable TT_TUNE_CACHE naming a text file, a batch whose key
 * (device, and every item's precision, shape and sketch widths) is in the
 * file takes the stored shape without timing, and a tuned batch appends
 * its line "key ta chunk ctas_per_sm".  (TT_LOG=1 in the environment prints
 * plan layouts, the kernel of every accumulate and the tuner's choice on
 * stderr.) */
tt_status tt_plan_autotune(tt_plan_t plan, const void* const* X_ptrs, void* ws, double* cores, int* ranks,
                           tt_stream_t stream, int* best_out);

/* ----------------------------------------------------------- backward */

/* Adjoint of the one-pass map X -> cores with the pivots and ranks of the
 * last forward call frozen (the map is then smooth): given dL/dcores (device,
 * same padded layout as the cores), write dL/dX (device, x_dtype, prod(n)
 * entries; overwritten).  X enters only through the sketches, so
 * dX = sum_k Sbar_k Omega_k^T + sum_k Psi_k Rbar_k^T, with the test matrices
 * regenerated from Philox.  Uses the state saved in ws by the forward call:
 * ws must be the workspace of this plan's last completed forward call
 * (tt_pstt2, tt_pstt2_finalize), and no other plan may have used it since;
 * otherwise TT_ERR_STATE (also after tt_pstt2_noalloc, whose state is not in
 * any caller workspace). */
tt_status tt_pstt2_backward(tt_plan_t plan, void* ws, const double* dcores, void* dX,
                            tt_stream_t stream);

/* ------------------------------------------------------ reconstruction */

/* Dense X~ = G_1(:, i_1, :) ... G_d(:, i_d, :) (Sec. 2.2) from padded cores
 * (device) into Xt (device, dtype, prod(n) entries).  Uses ws for the left
 * and right interfaces. */
tt_status tt_reconstruct(tt_plan_t plan, const double* cores, void* Xt, tt_dtype dtype, void* ws,
                         tt_stream_t stream);

/* Fused error: out2 (device, 2 doubles, overwritten) = [||X - X~||_F^2,
 * ||X||_F^2] without materialising X~ (eq. (1.1)). */
tt_status tt_reconstruct_error(tt_plan_t plan, const double* cores, const void* X, double* out2,
                               void* ws, tt_stream_t stream);

/* Adjoint of tt_reconstruct: dcores (device, padded layout, overwritten) from
 * dL/dX~ (device, dtype), for the cores `cores` (device).  Every padded entry
 * gets its gradient too (the padded cores are a valid TT).  Needs a plan made
 * with TT_FLAG_DIFF (else TT_ERR_STATE). */
tt_status tt_reconstruct_backward(tt_plan_t plan, const double* cores, const void* dXt,
                                  tt_dtype dtype, double* dcores, void* ws, tt_stream_t stream);

/* -------------------------------------------------------------- status */

/* SYNCHRONOUS: waits for `stream`, then reads the workspace status word and
 * the rank array.  status_host (may be NULL) receives TT_OK,
 * TT_WARN_RANK_CAP, TT_ERR_RANK_DEFICIENT, TT_ERR_TIMEOUT or TT_ERR_NONFINITE
 * (the worst seen over all items); ranks_host (may be NULL) receives
 * rank_entries ints. */
tt_status tt_query_status(tt_plan_t plan, const void* ws, const int* ranks, int* status_host,
                          int* ranks_host, tt_stream_t stream);

const char* tt_status_string(tt_status s);

/* SYNCHRONOUS helper for FP16 plans (not in the paper): the scale exponent s
 * = 15 - e, where 2^(e-1) <= max |X| < 2^e, so that every |X| 2^s < 2^15
 * (the FP16 range ends at 65504) and the low parts of the split stay normal
 * down to |X| = 2^-18 max |X|.  X: device, dtype, count entries; reads X once
 * with one reduction kernel on `stream` and waits for it.  *s_out = 0 when X
 * is all zero or count = 0.  Errors: TT_ERR_INVALID_ARG (null pointer, count
 * < 0), TT_ERR_NONFINITE (X holds an inf or NaN; *s_out unchanged),
 * TT_ERR_CUDA. */
tt_status tt_x_scale_log2(const void* X, tt_dtype dtype, int64_t count, int* s_out, tt_stream_t stream);

/* -------------------------------------------------------- test helpers */

/* Test matrix entries (the Gaussian stream of the library) for rows
 * [row0, row0 + nrows) and columns [0, ncols) of stream `stream_id`, written
 * column-major to out (device, FP64, nrows x ncols) exactly as the sketch of
 * precision `prec` uses them (FP64 values, or the FP32 generator rounded to
 * TF32 / BF16 / FP16).  Errors: TT_ERR_INVALID_ARG (null out, negative sizes or
 * row0, ncols > TT_MAXL, unknown prec), TT_ERR_CUDA; empty ranges are TT_OK. */
tt_status tt_test_matrix(uint64_t seed, int stream_id, int64_t row0, int64_t nrows, int ncols,
                         tt_prec prec, double* out, tt_stream_t stream);

/* Raw Philox4x32-10 on `count` counters (device uint32 arrays of 4*count,
 * key = (key0, key1)); out gets 4*count words.  Errors: TT_ERR_INVALID_ARG
 * (null pointer, count < 0), TT_ERR_CUDA; count = 0 is TT_OK. */
tt_status tt_philox4x32_10(const uint32_t* ctr, uint32_t key0, uint32_t key1, uint32_t* out,
                           int64_t count, tt_stream_t stream);

/* Synthetic input: the Hilbert-type tensor 1/(x_{i_1} + ... + x_{i_d}),
 * x_i = 1 + i/(n-1), for the slab [first_last, first_last + count_last) of
 * the last mode, written to out (device, dtype).  The sum is formed in FP64
 * from i_1 upwards, then rounded to dtype.  Errors: TT_ERR_INVALID_ARG for
 * bad sizes or a slab outside n[d-1], TT_ERR_CUDA. */
tt_status tt_generate_hilbert_type(int d, const int64_t* n, int64_t first_last,
                                   int64_t count_last, void* out, tt_dtype dtype,
                                   tt_stream_t stream);

/* Synthetic input: the paper's Hilbert tensor 1/(1 - d + i_1 + ... + i_d)
 * with 1-based indices (Sec. 4.3, the tensor of its memory and timing
 * experiments, Table 1), for the slab [first_last, first_last + count_last)
 * of the last mode, written to out (device, dtype): the integer sum is exact,
 * then one FP64 division, rounded to dtype.  Errors: TT_ERR_INVALID_ARG for
 * bad sizes or a slab outside n[d-1]. */
tt_status tt_generate_hilbert(int d, const int64_t* n, int64_t first_last, int64_t count_last,
                              void* out, tt_dtype dtype, tt_stream_t stream);

/* Synthetic input: the Gaussian-bumps tensor of Sec. 4.4,
 *   X(i) = sum_{j < nbumps} exp(-gamma sum_k (x_k - c_{j,k})^2),
 *   x_k = 2 i_k / n_k - 1 (0-based i_k),
 * evaluated in FP64 as sum_j prod_k exp(-gamma (x_k - c_{j,k})^2) (products
 * over k in increasing order, sum over j in increasing order) and rounded to
 * dtype, for the slab [first_last, first_last + count_last) of the last mode.
 * centres: HOST array of nbumps x d doubles, row j = (c_{j,1} .. c_{j,d}),
 * copied before the call returns.  Uses stream-ordered scratch for the
 * per-mode factor tables (sum_k n_k nbumps doubles) and synchronizes the
 * stream before returning.  Errors: TT_ERR_INVALID_ARG, TT_ERR_CUDA (also when
 * the scratch cannot be allocated). */
tt_status tt_generate_gaussian_bumps(int d, const int64_t* n, int nbumps, double gamma,
                                     const double* centres, int64_t first_last, int64_t count_last,
                                     void* out, tt_dtype dtype, tt_stream_t stream);

/* Tucker2TT (Algorithm 3), second step: T = H x_2 A for one TT core.  H: the
 * core (r0 x s x r1, column-major, device FP64), e.g. a core of the train that
 * tt_pstt2 computed for a Tucker core tensor; A: the Tucker factor of that mode
 * (n x s, column-major, device FP64); T: output r0 x n x r1 (column-major,
 * device FP64), T(a, i, c) = sum_k A(i, k) H(a, k, c).  Zero rows of padded
 * ranks stay zero.  Asynchronous on stream.  Errors: TT_ERR_INVALID_ARG for
 * null pointers or sizes < 1, TT_ERR_CUDA. */
tt_status tt_core_mode2(const double* H, int r0, int64_t s, int r1, const double* A, int64_t n,
                        double* T, tt_stream_t stream);

/* TT2Tucker (Algorithm 4) layout step: out(j, i, k) = in(i, j, k) for a
 * column-major in of n0 x n1 x n2 doubles (device; out is n1 x n0 x n2 and
 * must not overlap in).  With (n0, n1, n2) = (r_{k-1}, n_k, r_k) it gives the
 * mode-2 matricization (T_k)_(2) (n_k x r_{k-1} r_k); with (t_k, r_{k-1},
 * r_k) it folds t_k x r_{k-1} r_k back into a core.  Asynchronous on stream.
 * Errors: TT_ERR_INVALID_ARG (null, sizes < 1, in == out), TT_ERR_CUDA. */
tt_status tt_swap12(const double* in, int64_t n0, int64_t n1, int64_t n2, double* out,
                    tt_stream_t stream);

/* Self-test of failure detection (no counterpart in the paper): launches one
 * CTA whose thread waits, with the bounded wait every kernel of this library
 * uses, on an mbarrier that nothing arrives at; after limit_cycles SM clock
 * cycles (1 .. 4e9) the wait gives up and ORs 4 (the timeout bit, reported as
 * TT_ERR_TIMEOUT by tt_query_status) into the device int *status_dev, and the
 * kernel returns normally; the context stays usable.  Asynchronous on stream. */
tt_status tt_selftest_wait_timeout(int64_t limit_cycles, int* status_dev, tt_stream_t stream);

/* Number of CUDA kernels this library has launched in this process so far
 * (host-side counter, incremented at every launch; for benchmarks that
 * report how many of the library's kernels ran inside a timed region). */
int64_t tt_kernel_launches(void);

/* Library version string (build id). */
const char* tt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TTSKETCH_H */
