/*
 * sdft.h - C ABI of the GB300 generalized radix-2 transform for signals whose
 * DFT is supported on a known homogeneous set (arxiv 2211.15299, "Fast DFT
 * Computation for Signals with Structured Support").
 *
 * Problem (Section II, Definitions 1 and 3): N = 2^log2N, a support J of k
 * distinct frequencies, and a signal f whose DFT F f (F(m,n) = exp(-2 pi i m n/N))
 * vanishes off J. Given J and k samples of f, return (F f)_J.
 *
 * Method (Sections VI-VIII): J must be homogeneous (Definition 9: its congruence
 * tree has exactly log2 k split levels, the pivots r_1 < ... < r_s, k = 2^s).
 * The samples are read at the pivoted sampling pattern I_r (Definition
 * "r_sampling_pattern") and combined by s butterfly levels (Lemma
 * "rec-hom-tree-split", Corollary "block-structure", Algorithm 1). The result is
 * (N/k) times the height-0 Hi-DFT (eq. "hom-implies-spectral" with the 1/N of
 * F^{-1} kept), exactly, up to floating-point rounding.
 *
 * Orders used by every call:
 *   sample t (0 <= t < k) is f(I[t]) with I[t] = sum_q bit_q(t) 2^(log2N-1-r_{q+1});
 *   coefficient t is (F f)(Jc[t]) with Jc[t] the element of J whose bit r_{q+1}
 *   equals bit_q(t) for every q (the canonical order; Corollary "block-structure").
 * sdft_plan_sample_indices and sdft_plan_support_order return I and Jc.
 *
 * Data layout: complex values are interleaved (re, im); complex64 = 2 x float,
 * complex128 = 2 x double. Device buffers are owned by the caller, must be
 * 16-byte aligned, and hold k values per instance, instances packed back to back.
 *
 * Errors: every call returns an sdft_status; nothing is thrown across the ABI.
 * Execute calls are asynchronous on the given stream; a CUDA error raised by a
 * launch is returned as SDFT_ERR_CUDA (call sdft_last_cuda_error for the code).
 * Kernel-side bounded waits that expire set a device status word read by
 * sdft_plan_device_status / sdft_batch_device_status (SDFT_ERR_TIMEOUT).
 *
 * Streams are passed as `void*` holding a cudaStream_t (NULL = legacy default).
 */
#ifndef SDFT_H
#define SDFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdft_plan_s* sdft_plan;
typedef struct sdft_batch_s* sdft_batch;

typedef enum {
  SDFT_OK = 0,
  SDFT_ERR_ARG = 1,             /* null pointer, bad size, misaligned buffer      */
  SDFT_ERR_NOT_POW2 = 2,        /* k is not a power of two                       */
  SDFT_ERR_RANGE = 3,           /* an element of J is >= N, or log2N too large   */
  SDFT_ERR_DUPLICATE = 4,       /* J has a repeated element                      */
  SDFT_ERR_NOT_HOMOGENEOUS = 5, /* number of pivots differs from log2 k          */
  SDFT_ERR_NOMEM = 6,           /* host or device allocation failed              */
  SDFT_ERR_BUDGET = 7,          /* request exceeds a caller-set memory budget    */
  SDFT_ERR_CUDA = 8,            /* a CUDA runtime/driver call failed             */
  SDFT_ERR_TIMEOUT = 9,         /* a bounded device-side wait expired            */
  SDFT_ERR_UNSUPPORTED = 10,    /* size or mode outside what the library supports */
  SDFT_ERR_NO_DEVICE = 11,      /* plan was created host-only / no CUDA device   */
  SDFT_ERR_PRECISION = 12       /* plans of different precision mixed in a batch */
} sdft_status;

typedef enum { SDFT_C64 = 0, SDFT_C128 = 1 } sdft_prec;

/* Plan flags. */
#define SDFT_PLAN_HOST_ONLY 0x1u    /* build the host tables only; no device upload */
#define SDFT_PLAN_FP64_DF 0x8u      /* complex128 plans: strided transforms and synthesis run
                                       their level kernels in double-float arithmetic (pairs of
                                       FP32 values, 48-bit significand, FP32 exponent range) on
                                       the FP32 pipes instead of the FP64 pipe (small batches of
                                       k <= 2^10 and k <= 16 stay FP64); the caller's buffers stay
                                       complex128; relative L2 error about 1e-14 for values of
                                       magnitude 1e-30 .. 1e30. Batches and servers run such
                                       plans in FP64. */
#define SDFT_PLAN_DEFER_DEVICE 0x2u /* build the device tables in host memory but do not upload:
                                       the plan can only be used through a server
                                       (sdft_server_submit), which uploads them into its arena
                                       per request, so creating it allocates no device memory */
#define SDFT_PLAN_USER_ORDER 0x10u  /* also keep, on the device, the canonical position of every
                                       J[u] as passed (4 bytes per frequency), for
                                       sdft_plan_to_user_order */

/* Largest log2N and log2 k the library accepts. */
#define SDFT_MAX_LOG2N 62u
#define SDFT_MAX_LOG2K 28u

/*
 * sdft_plan_create - validate J, find its pivots, order it, build I_r and the
 * twiddles, and upload the tables to the current CUDA device.
 *   log2N  : M, with N = 2^M, 0 <= M <= SDFT_MAX_LOG2N.
 *   J      : host array of k distinct frequencies in [0, N), any order; read only
 *            during the call.
 *   k      : |J|, a power of two, k <= 2^SDFT_MAX_LOG2K.
 *   prec   : arithmetic of the device path (complex64 or complex128 buffers).
 *   flags  : 0, or SDFT_PLAN_HOST_ONLY or SDFT_PLAN_DEFER_DEVICE (not both), with
 *            SDFT_PLAN_FP64_DF (complex128 only) and SDFT_PLAN_USER_ORDER as needed.
 *   out    : receives the plan; the caller owns it (sdft_plan_destroy).
 * Pivots: the levels l at which the congruence tree T(J) splits (Definition 8),
 * found as the 2-adic valuations of differences of neighbours in bit-reversed
 * order (Remark "tree-2-adic", Remark "pivot-as-gcd").
 * Homogeneity: exactly log2 k pivots (Definition 9, Proposition "hom-tree-prop").
 * Twiddles: stage m (1..s) and u < 2^(m-1) use
 *   exp(-2 pi i (Jc[u] mod 2^(r_m)) / 2^(r_m+1)),
 * i.e. omega_{r_m+1}^{Jc[u]} of Lemma "rec-hom-tree-split", evaluated in FP64 and
 * rounded once to the plan's precision.
 * Errors: SDFT_ERR_ARG, _NOT_POW2, _RANGE, _DUPLICATE, _NOT_HOMOGENEOUS, _NOMEM,
 * _CUDA, _UNSUPPORTED; *out is left NULL on error.
 */
sdft_status sdft_plan_create(uint32_t log2N, const uint64_t* J, uint64_t k, sdft_prec prec,
                             uint32_t flags, sdft_plan* out);

/* log2N, s = log2 k and precision of a plan. Any output pointer may be NULL. */
sdft_status sdft_plan_info(sdft_plan plan, uint32_t* log2N, uint32_t* log2k, sdft_prec* prec);

/* The s pivots r_1 < ... < r_s (Definition 8), written to host array `pivots`. */
sdft_status sdft_plan_pivots(sdft_plan plan, uint32_t* pivots);

/* I_r in sample order t = 0..k-1 (Definition "r_sampling_pattern"), host array of k. */
sdft_status sdft_plan_sample_indices(sdft_plan plan, uint64_t* I);

/* J in coefficient order t = 0..k-1 (canonical order), host array of k. */
sdft_status sdft_plan_support_order(sdft_plan plan, uint64_t* Jc);

/* The FP64 twiddles before rounding, stage-major: for m = 1..s and u < 2^(m-1),
 * (re, im) at tw[2 * (2^(m-1) - 1 + u)]; 2 * (k - 1) doubles. Unscaled. */
sdft_status sdft_plan_twiddles(sdft_plan plan, double* tw);

/* Device bytes the plan allocated when it was created: its tables (with the
 * double-float copy and the user-order positions when their flags are set) and
 * its status word. Work queues cached later by the queue strategy are not
 * counted. */
sdft_status sdft_plan_device_bytes(sdft_plan plan, uint64_t* bytes);

/*
 * sdft_execute - one instance: d_coeffs[t] = (F f)(Jc[t]) from d_samples[t] = f(I[t]).
 * d_samples, d_coeffs: device buffers of k complex values of the plan's
 * precision, 16-byte aligned; either the same buffer (in place) or disjoint.
 * Asynchronous on `stream`; allocates nothing; may run concurrently on one plan.
 */
sdft_status sdft_execute(sdft_plan plan, const void* d_samples, void* d_coeffs, void* stream);

/*
 * sdft_execute_strided - `batch` instances of one plan; instance b reads
 * d_samples + b*k and writes d_coeffs + b*k (complex elements). Same rules as
 * sdft_execute. One persistent launch per butterfly level (one launch when
 * k <= 2^12 for complex64, 2^11 for complex128).
 */
sdft_status sdft_execute_strided(sdft_plan plan, uint64_t batch, const void* d_samples,
                                 void* d_coeffs, void* stream);

/*
 * sdft_execute_strided_host - sdft_execute_strided on samples and coefficients
 * in host memory: h_samples (batch x k values, sample order) is copied to the
 * device buffer d_samples, transformed into d_coeffs and copied back into
 * h_coeffs, in chunks of `chunk` instances (0: about 16 MiB; rounded up so
 * that every chunk is a multiple of 16 bytes) so that a chunk's copy-in, the
 * previous chunk's transform and an earlier chunk's copy-out overlap. Host
 * buffers should be page-locked (cudaHostAlloc / cudaHostRegister) for the
 * copies to be asynchronous; they may be identical or must be disjoint. Device
 * buffers as for sdft_execute_strided (caller-owned, 16-byte aligned, identical
 * or disjoint), each of batch x k values. The copies run on two streams of the
 * plan (created with three events on the first call; no device memory is
 * allocated) that start after the work already queued on `stream`; `stream`
 * itself runs the transforms and, when the call returns, has been made to wait
 * for the last copy-out, so synchronising `stream` (or an event recorded on it
 * afterwards) covers the whole call. Calls on one plan are serialised while
 * they enqueue; graph capture of `stream` captures the fork and join. All
 * arguments, host and device, are checked before anything is enqueued. Errors:
 * SDFT_ERR_ARG, SDFT_ERR_NO_DEVICE, SDFT_ERR_CUDA, and those of
 * sdft_execute_strided.
 */
sdft_status sdft_execute_strided_host(sdft_plan plan, uint64_t batch, const void* h_samples, void* h_coeffs,
                                      void* d_samples, void* d_coeffs, uint64_t chunk, void* stream);

/*
 * sdft_plan_to_user_order - the optional reordering of the coefficients into the
 * caller's order of J: for `batch` instances, d_user[b k + u] = d_canonical[b k +
 * t(u)], where t(u) is the canonical position of J[u] (J as passed to
 * sdft_plan_create; the canonical order is the one sdft_execute returns and
 * sdft_plan_support_order lists). One gather kernel, out of place (the buffers
 * must not overlap), asynchronous on `stream`. Needs a plan created with
 * SDFT_PLAN_USER_ORDER (SDFT_ERR_ARG otherwise); SDFT_ERR_NO_DEVICE for
 * host-only plans.
 */
sdft_status sdft_plan_to_user_order(sdft_plan plan, uint64_t batch, const void* d_canonical, void* d_user,
                                    void* stream);

/*
 * sdft_execute_batched - n instances, instance i with its own plan plans[i]
 * (repeats allowed, one precision, all on the current device), packed at the
 * caller's offsets: instance i's samples are d_samples[d_offsets[i] ..
 * d_offsets[i+1]) (sample order, d_offsets[i+1] - d_offsets[i] = k of plans[i])
 * and its coefficients go to the same range of d_coeffs. d_offsets is a device
 * array of n + 1 value offsets (read on the device, so the call is
 * graph-capturable). It runs the uneven-batch work queue (sdft_batch_*) between
 * a gather into the batch's own packing and a scatter back; the first call for a
 * given list of plans builds that batch and its staging buffers (2 x total
 * values) and caches them (allocates and may synchronise the device: make that
 * call before capturing a graph). The 8 most recently built unpinned lists are
 * kept: building a ninth frees the oldest unpinned one, and a CUDA graph
 * captured on a freed list would replay on freed memory, so pin every list a
 * graph is captured on (sdft_execute_batched_pin). sdft_plan_destroy of any
 * plan in a list frees that list, pinned or not. Calls with the same list must
 * not overlap on the GPU. sdft_batch_execute on the batch's own layout saves
 * the two copies.
 * Offsets that do not match the plans' k are reported as 0x104 in the status
 * word of plans[0] (sdft_plan_device_status) and those instances are skipped;
 * offsets must lie inside the caller's buffers. Buffers 16-byte aligned,
 * identical or disjoint. Errors: SDFT_ERR_ARG, SDFT_ERR_NO_DEVICE,
 * SDFT_ERR_PRECISION, SDFT_ERR_NOMEM, SDFT_ERR_CUDA, and those of
 * sdft_batch_create. The paper computes one instance at a time (Algorithm 1).
 */
sdft_status sdft_execute_batched(const sdft_plan* plans, uint64_t n, const void* d_samples,
                                 const uint64_t* d_offsets, void* d_coeffs, void* stream);

/*
 * sdft_execute_batched_pin - pin != 0: build (if not cached yet; allocates and
 * may synchronise the device) and pin the cached list of these plans, so that
 * building other lists never frees it; pin == 0: unpin it (it becomes the
 * candidate for eviction it would have been by age; nothing is built). Pinned
 * lists do not count toward the 8 kept unpinned lists. Plans as for
 * sdft_execute_batched. Errors: SDFT_ERR_ARG, SDFT_ERR_NO_DEVICE,
 * SDFT_ERR_PRECISION, SDFT_ERR_NOMEM, SDFT_ERR_CUDA.
 * sdft_execute_batched_cache_info - whether the list of these plans is cached
 * and pinned (0 or 1; plans may be NULL with n = 0), and the number of cached
 * lists (any output may be NULL). Host-only, no device work.
 * The paper has no counterpart: these manage the library's own cache.
 */
sdft_status sdft_execute_batched_pin(const sdft_plan* plans, uint64_t n, int pin);
sdft_status sdft_execute_batched_cache_info(const sdft_plan* plans, uint64_t n, int* cached, int* pinned,
                                            uint64_t* n_lists);

/* The same for synthesis (sdft_synthesize_strided): h_coeffs in, h_samples out,
 * through the device buffers d_coeffs and d_samples. */
sdft_status sdft_synthesize_strided_host(sdft_plan plan, uint64_t batch, const void* h_coeffs, void* h_samples,
                                         void* d_coeffs, void* d_samples, uint64_t chunk, void* stream);

/*
 * sdft_synthesize / sdft_synthesize_strided - the inverse map: samples
 * f_I = F^{-1}(I_r, J) c = (1/N) F(J, I_r)^H c from coefficients c (Section II,
 * eq. "submatrix-method"; F(J, I_r)^H F(J, I_r) = k Id, so this inverts
 * sdft_execute). It runs the adjoint of the execute network (Cor.
 * "block-structure"): the same stages in reverse order with conjugated
 * twiddles, the N/k folded into the last stage undone exactly and 1/N applied
 * at stage 1. Layouts, buffers, in-place use and errors as for sdft_execute /
 * sdft_execute_strided with the roles swapped: coefficients in canonical order
 * in, samples in sample order out.
 */
sdft_status sdft_synthesize(sdft_plan plan, const void* d_coeffs, void* d_samples, void* stream);
sdft_status sdft_synthesize_strided(sdft_plan plan, uint64_t batch, const void* d_coeffs, void* d_samples,
                                    void* stream);

/* Execution strategy of a multi-level plan (k > 2^12 for complex64, 2^11 for
 * complex128) in sdft_execute / sdft_execute_strided:
 *   SDFT_STRATEGY_LEVELS: one persistent launch per butterfly level (default);
 *   SDFT_STRATEGY_QUEUE : one persistent launch over a work queue whose
 *     later-level tiles follow their instance's previous level, so the
 *     intermediate is read back from L2; the first call with a given batch size
 *     builds and caches the queue (allocates: make that call before capturing
 *     a CUDA graph). A plan keeps the queues of its 4 most recent batch sizes:
 *     a fifth size synchronises the device and frees the oldest, and a CUDA
 *     graph captured on a freed queue must not be replayed. The cached
 *     queue's dependency counters are shared, so with this strategy calls on
 *     one plan with the same batch size must not overlap on the GPU (the
 *     default strategy has no such state). Single-level plans ignore the
 *     strategy. */
typedef enum { SDFT_STRATEGY_LEVELS = 1, SDFT_STRATEGY_QUEUE = 2 } sdft_strategy;
sdft_status sdft_plan_set_strategy(sdft_plan plan, sdft_strategy strategy);

/*
 * sdft_plan_autotune - time every strategy x stages-per-pass choice on `batch`
 * instances in the given buffers (each run `reps` times after one warm-up,
 * CUDA events on `stream`), keep the fastest for the plan (strategy, and
 * stages per pass: sdft_plan_get_stages_per_pass) and report each strategy's
 * best mean time in milliseconds (any output pointer may be NULL). The choice
 * is also stored in the library's tuning cache under (precision, log2 k,
 * floor(log2 batch)) (see sdft_autotune_cache_save). Synchronises `stream`.
 * The buffers are overwritten. Single-level plans report
 * SDFT_STRATEGY_LEVELS and time it only.
 */
sdft_status sdft_plan_autotune(sdft_plan plan, uint64_t batch, const void* d_samples, void* d_coeffs,
                               void* stream, int reps, sdft_strategy* chosen, float* ms_levels,
                               float* ms_queue);

/* Apply the tuning cache's choice for this plan at this batch size (same key
 * as sdft_plan_autotune), without timing: *found = 1 if there was one (else
 * the plan is left as it is and *found = 0). Errors: SDFT_ERR_ARG (also for a
 * cached entry this plan cannot take). */
sdft_status sdft_plan_apply_tuning(sdft_plan plan, uint64_t batch, int* found);

/*
 * Stages per pass of a plan's butterfly kernels: every tile holds 2^12
 * (complex64) or 2^11 (complex128) values in shared memory, and each thread
 * runs `stages_per_pass` consecutive stages of Algorithm 1's network on
 * 2^stages_per_pass of them in registers per pass over the tile. 4 (the
 * default; 16 values per thread, 256 threads per complex64 tile) or, for
 * complex64 plans, 3 (8 values per thread, 512 threads, one pass more per
 * 12 stages). Every choice gives the same bits. sdft_plan_autotune chooses it
 * with the strategy. A change synchronises the device if the plan holds
 * cached work queues (they are rebuilt on next use). Like
 * sdft_plan_set_strategy, sdft_plan_autotune and sdft_plan_apply_tuning, it
 * changes the plan: call it while no other thread is calling an execute or
 * synthesis entry point on the same plan. The paper has no counterpart
 * (Algorithm 1 is stated as a recursion). Errors: SDFT_ERR_ARG.
 */
sdft_status sdft_plan_set_stages_per_pass(sdft_plan plan, uint32_t stages_per_pass);
sdft_status sdft_plan_get_stages_per_pass(sdft_plan plan, uint32_t* stages_per_pass);

/* Device status word of a plan: SDFT_OK, SDFT_ERR_TIMEOUT, or a launch
 * self-check code above 0xff (0x101: dynamic shared memory smaller than the
 * kernel's layout; 0x102: tensor-map parameter not 64-byte aligned; 0x103:
 * twiddle table, or a batch's item list, not 16-byte aligned; the kernel did
 * no work; 0x104: sdft_execute_batched offsets that do not match the plans). Synchronises the
 * device; clears the word when `clear` is non-zero. */
sdft_status sdft_plan_device_status(sdft_plan plan, int clear);

/* Release a plan: its tables, status word, cached work queues and host-copy
 * streams, and every cached sdft_execute_batched list that names it. The caller
 * must first synchronise any work using it; a batch (sdft_batch_*) built on it
 * must not run afterwards. */
sdft_status sdft_plan_destroy(sdft_plan plan);

/* ------------------------------------------------------------------------ */
/* Uneven batches: many instances, each with its own plan, in one launch.    */
/* ------------------------------------------------------------------------ */

/*
 * sdft_batch_create - build a device work queue for instances i = 0..n-1 with
 * plans[i] (repeats allowed; all of one precision, all on the current device).
 * The library chooses the packed layout: instances sit by decreasing k, so each
 * instance's element offset is a multiple of its k; sdft_batch_info returns the
 * offset of every instance (in the caller's order) and the total. Work items:
 * level-0 tiles (several same-size instances per 32 KiB tile), later-level tiles
 * placed at least 4 x grid items after their instance's previous level, and
 * ranges of instances with k <= 16. The plans must outlive the batch (the queue
 * points at their device twiddle tables). Allocates the queue, the dependency
 * counters and a status word on the device.
 */
sdft_status sdft_batch_create(const sdft_plan* plans, uint64_t n, sdft_batch* out);

/* Total coefficients, and (if `offsets` is not NULL) n+1 values: offsets[i] is the
 * element offset of instance i in the packed buffers, offsets[n] the total. */
sdft_status sdft_batch_info(sdft_batch batch, uint64_t* total, uint64_t* offsets);

/*
 * sdft_batch_execute - run every instance of the batch: one persistent kernel
 * over the work queue. Buffers as described at sdft_batch_create, 16-byte
 * aligned, identical (in place) or disjoint. Asynchronous, allocates nothing,
 * and may be captured into a CUDA graph. A launch uses the batch's dependency
 * counters: launches of one batch must not overlap on the GPU (one stream, or
 * one batch per stream). The launch is cooperative: CTA c takes items c,
 * c + G, ... and later-level items wait for tiles of other CTAs, so it relies
 * on all G CTAs being resident. By default G is every co-resident CTA of the
 * device; to run several batch launches at once on other streams, give them
 * disjoint shares (sdft_batch_set_schedule's grid), else waits may run out
 * (SDFT_ERR_TIMEOUT in the status word).
 */
sdft_status sdft_batch_execute(sdft_batch batch, const void* d_samples, void* d_coeffs,
                               void* stream);

/*
 * sdft_batch_execute_noalloc - the same work as sdft_batch_execute, for callers
 * that must not allocate device memory while they run: for example code that
 * works under a fixed device-memory budget handed out once at start-up, or a
 * serving loop where a cudaMalloc could stall every stream on the device. The
 * paper has no counterpart; this is a property of the library only.
 * The call itself allocates nothing: the batch (created earlier) supplies its
 * queue, and the dependency counters come from one fixed array of 65536
 * 32-bit counters (256 KiB) built into the library, present on every device
 * that loads it until the process exits. Batches needing more counters (more
 * than 65536 multi-level instance levels) are rejected with
 * SDFT_ERR_UNSUPPORTED. sdft_batch_create looks up that array's device address
 * on the batch's device (with that device current) and keeps it in the batch,
 * so this call does no lookup either. All calls share the array and it keeps the last call's
 * counts, so each call clears the part it uses first; calls whose work
 * overlaps on the GPU (other streams, other threads) race on it and must be
 * serialised by the caller. Buffers as for sdft_batch_execute.
 */
sdft_status sdft_batch_execute_noalloc(sdft_batch batch, const void* d_samples, void* d_coeffs,
                                       void* stream);

/* Stages per pass of a batch's queue kernel (as for plans: 4, or 3 for
 * complex64; the same bits either way). Rebuilds the batch's item list (its
 * grid follows the kernel's occupancy): synchronise work using the batch
 * first, re-capture graphs, and call it (like every setter of a batch) while
 * no other thread is launching the batch. */
sdft_status sdft_batch_set_stages_per_pass(sdft_batch batch, uint32_t stages_per_pass);
sdft_status sdft_batch_get_stages_per_pass(sdft_batch batch, uint32_t* stages_per_pass);

/* Where a batch's queue kernel keeps each item's twiddle table: 0 (default)
 * registers and L1 for the last pass, shared-memory copies of the small first
 * and middle regions, two CTAs per SM; 1 (complex64 only) the whole table
 * (2^12 entries, 32 KiB) copied into shared memory with each tile, so no pass
 * waits on a global load, one CTA per SM. The same bits either way. Rebuilds the
 * item list as for sdft_batch_set_stages_per_pass. sdft_batch_autotune chooses
 * it with the other settings. Errors: SDFT_ERR_ARG. */
sdft_status sdft_batch_set_table_staging(sdft_batch batch, int staged);
sdft_status sdft_batch_get_table_staging(sdft_batch batch, int* staged);

/* Dependency distance of the batch's item list (an implementation setting of
 * the work queue, not part of the paper's method): an item of a later level of
 * an instance is placed at least `lag` x grid list places after the last item
 * of the level before it (4 <= lag <= 64; default 6). 4 is the least for
 * which every dependency wait of the persistent launch ends; a larger lag
 * means fewer waits but an intermediate that stays longer in L2. Rebuilds the
 * item list as for sdft_batch_set_stages_per_pass; sdft_batch_autotune chooses
 * it (4, 6 or 8) with the other settings. Errors: SDFT_ERR_ARG. */
sdft_status sdft_batch_set_lag(sdft_batch batch, uint32_t lag);
sdft_status sdft_batch_get_lag(sdft_batch batch, uint32_t* lag);

/* Apply the tuning cache's choice for this batch (key: precision,
 * floor(log2 n), floor(log2 total values)) without timing; *found as for
 * sdft_plan_apply_tuning. Rebuilds the item list when the choice differs. */
sdft_status sdft_batch_apply_tuning(sdft_batch batch, int* found);

/* Device status word of a batch (as for plans). */
sdft_status sdft_batch_device_status(sdft_batch batch, int clear);

/* Diagnostics: override the bound on device-side waits (0 restores the default)
 * and add `need_bias` to every dependency target. A non-zero bias makes every
 * later-level tile wait for a count that is never reached, so the launch ends
 * with SDFT_ERR_TIMEOUT in the status word after `timeout_ns`: it exists to test
 * that path. */
sdft_status sdft_batch_set_wait(sdft_batch batch, uint64_t timeout_ns, uint32_t need_bias);

/* Order of a batch's work items (see sdft_batch_set_schedule). No paper
 * counterpart: scheduling of many instances is a property of this library. */
typedef enum {
  SDFT_SCHEDULE_AUTO = 0,         /* the library's default (round robin) */
  SDFT_SCHEDULE_LANES = 1,        /* each instance's levels in one CTA, largest first to the least-loaded CTA */
  SDFT_SCHEDULE_ROUND_ROBIN = 2   /* instances in packed order over consecutive CTAs */
} sdft_schedule;

/*
 * sdft_batch_set_schedule - rebuild the batch's work queue with the given item
 * order on `grid` CTAs (0: every co-resident CTA; larger values are clamped to
 * that). Offsets, buffers and results do not change: every instance runs the
 * same arithmetic in any order, so results are bit-identical. The device item
 * list is reallocated: synchronise work using the batch first, and re-capture
 * any CUDA graph holding it. SDFT_ERR_ARG for an unknown schedule.
 */
sdft_status sdft_batch_set_schedule(sdft_batch batch, sdft_schedule schedule, uint32_t grid);

/*
 * sdft_batch_autotune - time the batch under every queue shape (lanes or round
 * robin, on all co-resident CTAs or on half of them), stages-per-pass choice
 * (4, and 3 for complex64), table placement (sdft_batch_set_table_staging;
 * both for complex64) and dependency distance (sdft_batch_set_lag: 4, 6 or
 * 8); one warm-up and `reps` timed runs each,
 * CUDA events on `stream`, the buffers overwritten. Keeps the fastest, reports
 * it (any output may be NULL; `ms_best` is the mean time of one run; the
 * stages per pass: sdft_batch_get_stages_per_pass) and stores it in the
 * tuning cache. Synchronises `stream`. As for sdft_batch_set_schedule, graphs
 * captured before must be re-captured.
 */
sdft_status sdft_batch_autotune(sdft_batch batch, const void* d_samples, void* d_coeffs, void* stream, int reps,
                                sdft_schedule* chosen, uint32_t* chosen_grid, float* ms_best);

/* Work items, dependency counters and grid size (co-resident CTAs) of a batch;
 * returns SDFT_ERR_ARG if the item list breaks its ordering invariants (every
 * dependency target reached exactly, by items at least 4 x grid positions
 * earlier). A batch built from host-only plans (SDFT_PLAN_HOST_ONLY) has its item
 * list for inspection (grid taken as 304) but cannot execute. */
sdft_status sdft_batch_stats(sdft_batch batch, uint64_t* n_items, uint64_t* n_counters, int* grid);

/* Release a batch after synchronising its work. */
sdft_status sdft_batch_destroy(sdft_batch batch);

/* ------------------------------------------------------------------------ */
/* Shift-and-Sample: supports that are not homogeneous                       */
/* ------------------------------------------------------------------------ */

typedef struct sdft_sas_s* sdft_sas;

/*
 * sdft_sas_create - plan Shift-and-Sample (Algorithm "shift-sample", Section
 * "balanced partly homogeneous families") for an arbitrary support J of k
 * distinct frequencies in [0, 2^log2N) (k need not be a power of two).
 *   R     : number of pivots; the pivots are the first R split levels of the
 *           congruence tree T(J), so J is part-homogeneous for them (Definition
 *           "part-H-tree"). 0 chooses R: the smallest operation count of
 *           Lemma "computation_shift_sample" (1.5 R 2^R mu* + 6 sum_v mu(v)^2)
 *           among R whose class systems have 1-norm condition <= 32
 *           (complex64) or <= 100 (complex128), else the best-conditioned R;
 *           under these caps results stay within 1e-5 / 1e-12 (relative L2).
 *   flags : 0, SDFT_PLAN_HOST_ONLY (planning only; cannot execute), and/or
 *           SDFT_SAS_TWO_STAGE (see sdft_sas_execute).
 * The classes of J modulo 2^(r_max+1) hold mu(v) <= mu* <= 64 members. The
 * instance needs mu* x 2^R samples: row a (a < mu*) is f at I_r + a (mod N)
 * (sdft_sas_sample_indices). The plan owns a virtual homogeneous plan with
 * pivots r and, per class, the inverse of its Vandermonde matrix
 * [exp(2 pi i a l / N)] (a < mu(v), l its members; eq. "alg1_system"),
 * computed in FP64 and rounded once to the precision of `prec`.
 * Errors: SDFT_ERR_RANGE (j >= N), SDFT_ERR_DUPLICATE, SDFT_ERR_ARG (R larger
 * than the number of split levels or than 24), SDFT_ERR_UNSUPPORTED (no R
 * keeps mu* <= 64, or a singular class system), SDFT_ERR_NOMEM, SDFT_ERR_CUDA.
 */
sdft_status sdft_sas_create(uint32_t log2N, const uint64_t* J, uint64_t k, sdft_prec prec, uint32_t R,
                            uint32_t flags, sdft_sas* out);

/* sdft_sas_create flag: always run stage 2 as its own launch (the two-launch
 * path), also where both stages fit one launch. */
#define SDFT_SAS_TWO_STAGE 0x4u

/* R, mu*, samples per instance (mu* x 2^R), classes J occupies, and the largest
 * 1-norm condition number of the class systems (any output may be NULL). */
sdft_status sdft_sas_info(sdft_sas sas, uint32_t* R, uint32_t* mu_star, uint64_t* samples_per_instance,
                          uint32_t* occupied_classes, double* max_cond);

/* The R pivots (ascending). */
sdft_status sdft_sas_pivots(sdft_sas sas, uint32_t* r);

/* mu* x 2^R sample indices, row-major by shift a: the order of one instance's
 * samples in the execute buffer. */
sdft_status sdft_sas_sample_indices(sdft_sas sas, uint64_t* idx);

/* The k frequencies in output order (by class, then by value). */
sdft_status sdft_sas_support_order(sdft_sas sas, uint64_t* J);

/* Device workspace that sdft_sas_execute needs for `batch` instances. */
sdft_status sdft_sas_workspace_bytes(sdft_sas sas, uint64_t batch, uint64_t* bytes);

/* How sdft_sas_execute runs this plan when d_samples, d_work and d_coeffs do
 * not overlap (an implementation property, not part of Algorithm
 * "shift-sample"): *launches = 1 where both stages share one launch, else 2
 * (the strided transform itself takes more than one for R > 12);
 * *work_values = the values per instance that stage 1 leaves in d_work: 0
 * (none: one launch, mu* = 1), k (only those the class solves read) or
 * mu* x 2^R (the whole stage-1 output). Either output may be NULL. */
sdft_status sdft_sas_path(sdft_sas sas, uint32_t* launches, uint64_t* work_values);

/*
 * sdft_sas_execute - coefficients of `batch` instances: d_samples holds
 * batch x mu* x 2^R values (sample_indices order), d_coeffs receives batch x k
 * (support_order), d_work is the workspace (it may be d_samples itself, which
 * is then overwritten; it must not overlap d_coeffs). Stage 1 runs the virtual
 * plan over the batch x mu* shifted sample sets (Algorithm 1); stage 2 solves
 * each class with its precomputed inverse. Where one to four virtual
 * instances fill a tile (R in [10, 12] for complex64, [9, 11] for complex128):
 *   - under complete isolation (mu* = 1, k <= 2^12 / 2^11) both stages run in
 *     one launch that keeps the stage-1 output on chip: d_work is then not
 *     touched and d_samples must not overlap d_coeffs;
 *   - with mu* > 1 (k <= 8192) and d_work apart from d_samples, stage 1 writes
 *     to d_work only the k values per instance that the class solves read
 *     (the first batch x k values of d_work), instead of all mu* x 2^R.
 * sdft_sas_path tells which applies. SDFT_SAS_TWO_STAGE keeps the two
 * launches over the whole stage-1 output.
 * All paths give the same bits. Device buffers 16-byte aligned; asynchronous
 * on `stream`. SDFT_ERR_NO_DEVICE for host-only plans.
 */
sdft_status sdft_sas_execute(sdft_sas sas, uint64_t batch, const void* d_samples, void* d_work, void* d_coeffs,
                             void* stream);

/* Release the plan (synchronise work using it first). */
sdft_status sdft_sas_destroy(sdft_sas sas);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of requests under a device-memory budget     */
/* ------------------------------------------------------------------------ */

typedef struct sdft_server_s* sdft_server;

typedef struct {
  uint64_t submitted;        /* requests accepted by sdft_server_submit          */
  uint64_t completed;        /* requests whose coefficients are in host memory   */
  uint64_t failed;           /* requests completed with a non-zero status        */
  uint64_t micro_batches;    /* work-queue launches                              */
  uint64_t coeffs;           /* coefficients of the completed requests           */
  uint64_t inflight;         /* requests admitted and not yet completed          */
  uint64_t max_inflight;     /* largest `inflight` seen                          */
  uint64_t arena_bytes;      /* device arena (the admission budget)              */
  uint64_t arena_peak_bytes; /* largest arena use                                */
  uint64_t planned;          /* supports planned by the server's planner threads */
  uint64_t injected;         /* requests dropped, failed or delayed by sdft_server_inject */
} sdft_server_stats;

/*
 * sdft_server_create - a serving engine on the current device. `budget_bytes`
 * (rounded down to a power of two) is allocated once as the arena that holds
 * the requests' samples and coefficients; a request is admitted when a block of
 * its size (k x element size, at least 128 bytes) is free. Up to `n_slots`
 * micro-batches of up to `max_batch` requests run at once, each one
 * persistent work-queue launch on its own stream, sharing the co-resident CTAs.
 * A worker thread forms micro-batches in arrival order as slots and memory free
 * up (continuous batching). Plans stay owned by the caller and must outlive
 * their requests. `n_planners` threads (0..64) plan the supports submitted
 * with sdft_server_submit_support. No paper counterpart: serving is a property
 * of this library. SDFT_ERR_ARG for out-of-range arguments.
 */
sdft_status sdft_server_create(sdft_prec prec, uint64_t budget_bytes, uint32_t n_slots, uint32_t max_batch,
                               uint32_t n_planners, sdft_server* out);

/* Queue one request: transform k = plan's k samples at h_samples into h_coeffs
 * (host buffers; pinned memory makes the copies asynchronous). The buffers must
 * stay valid until the request completes. `tag` identifies it in poll. */
sdft_status sdft_server_submit(sdft_server srv, sdft_plan plan, const void* h_samples, void* h_coeffs,
                               uint64_t tag);

/*
 * sdft_server_submit_support - queue one request that brings its support
 * instead of a plan: J (k frequencies in [0, 2^log2N), copied during the call)
 * is planned by one of the server's planner threads (as sdft_plan_create with
 * SDFT_PLAN_DEFER_DEVICE: Definitions 8, 9 and the pivoted sampling pattern
 * of Section VII), the request then enters the admission FIFO, and the plan is
 * released when it completes. Planning time counts in the latency. h_samples
 * holds f at the support's sample set I_r in sample order, h_coeffs receives
 * the coefficients in the support's canonical order (the orders
 * sdft_plan_sample_indices / sdft_plan_support_order report for a plan of the
 * same J). A support that fails validation completes with that status
 * (e.g. SDFT_ERR_NOT_HOMOGENEOUS). SDFT_ERR_UNSUPPORTED if the server has no
 * planner threads. Buffers as for sdft_server_submit.
 */
sdft_status sdft_server_submit_support(sdft_server srv, uint32_t log2N, const uint64_t* J, uint64_t k,
                                       const void* h_samples, void* h_coeffs, uint64_t tag);

/* Up to `cap` completed requests since the last poll: tag, latency in seconds
 * (submit to the completion of the copy-out), status (SDFT_OK; SDFT_ERR_BUDGET
 * when a request can never fit the arena; a plan-creation status for a support
 * that failed validation). *n_out = count. */
sdft_status sdft_server_poll(sdft_server srv, uint64_t* tags, double* latency_s, int32_t* status, uint64_t cap,
                             uint64_t* n_out);

/* Wait until every submitted request has completed (0 = no time limit). */
sdft_status sdft_server_drain(sdft_server srv, uint64_t timeout_ms);

sdft_status sdft_server_get_stats(sdft_server srv, sdft_server_stats* stats);

/* Device status word of the server's launches (as for plans). */
sdft_status sdft_server_device_status(sdft_server srv, int clear);

/*
 * sdft_server_inject - host-side fault injection for testing a client's failure
 * handling, with no device involvement: of the requests that reach admission
 * after this call, every `every`-th is
 *   SDFT_INJECT_DROP : discarded (it never completes; a client sees it only by
 *                      its absence, for example when its own deadline passes),
 *   SDFT_INJECT_FAIL : completed at once with SDFT_ERR_CUDA, as if its launch
 *                      had failed (nothing of it runs),
 *   SDFT_INJECT_DELAY: held back `delay_us` microseconds (at most 10 s) before
 *                      it is admitted, then run normally.
 * SDFT_INJECT_OFF (or a later call) stops it. Counted in
 * sdft_server_stats.injected. SDFT_ERR_ARG for an unknown mode or every = 0.
 */
typedef enum { SDFT_INJECT_OFF = 0, SDFT_INJECT_DROP = 1, SDFT_INJECT_FAIL = 2, SDFT_INJECT_DELAY = 3 } sdft_inject;
sdft_status sdft_server_inject(sdft_server srv, uint32_t mode, uint64_t every, uint64_t delay_us);

/* Stop accepting requests, finish the queued ones, release everything. */
sdft_status sdft_server_destroy(sdft_server srv);

/* ------------------------------------------------------------------------ */
/* Tuning cache                                                              */
/* ------------------------------------------------------------------------ */

/*
 * The autotuners (sdft_plan_autotune, sdft_batch_autotune) store their choice
 * in one process-wide cache; sdft_plan_apply_tuning / sdft_batch_apply_tuning
 * apply a stored choice without timing. _save writes the cache as a JSON
 * object, one member per key ("plan/c64/s20/b6": plan of complex64, log2 k =
 * 20, batch in [64, 128); "batch/c64/n13/t26": uneven batch of 2^13..2^14 - 1
 * instances and 2^26..2^27 - 1 values), each an object with the fields
 * strategy, schedule, grid, stages_per_pass, table_staging and ms (the time
 * measured).
 * _load merges such a file into the cache (SDFT_ERR_ARG for a file that
 * cannot be read or parsed; the cache is then unchanged). _clear empties it;
 * _size reports its entries. Host-only; thread-safe. The paper has no
 * counterpart.
 */
sdft_status sdft_autotune_cache_save(const char* path);
sdft_status sdft_autotune_cache_load(const char* path);
sdft_status sdft_autotune_cache_clear(void);
sdft_status sdft_autotune_cache_size(uint64_t* entries);

/* ------------------------------------------------------------------------ */
/* Diagnostics                                                               */
/* ------------------------------------------------------------------------ */

/* Static text for a status code. */
const char* sdft_status_string(sdft_status status);

/* The cudaError_t value behind the last SDFT_ERR_CUDA returned on this thread. */
int sdft_last_cuda_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int sdft_version(void);

/* Range checks of the debug build (compiled with SDFT_BOUNDS_CHECK=1): every
 * TMA tile coordinate, twiddle-table range and work-queue record is checked
 * before use; a violation is counted, recorded as 0x105 in the launch's status
 * word and the access made harmless (no trap). *enabled = 1 in that build, 0
 * otherwise (then *count = 0); *count = violations on the current device since
 * the last clear (clear != 0 resets them). Synchronous. Outputs may be NULL.
 * The paper has no counterpart: a checking aid of this library. */
sdft_status sdft_debug_bounds_violations(int* enabled, uint64_t* count, int clear);

#ifdef __cplusplus
}
#endif

#endif /* SDFT_H */
