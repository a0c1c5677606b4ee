/*
 * topk.h — C ABI of libtopk: exact selection of the k smallest of n keys on
 * one GB300 GPU (sm_103a).
 *
 * Method: sample-based two-pivot selection in the style of distributed
 * Floyd-Rivest selection (Hübschle-Schneider, Sanders, Müller, "Communication
 * Efficient Algorithms for Top-k Selection Problems", Section 2, Algorithm
 * "select"; Section 4.1, Theorem "selectFR"), with the paper's processing
 * elements mapped to on-device partitions and its collective reductions to
 * in-kernel block sums; and multisequence selection on locally sorted runs
 * (Section 4.2; Appendix A, Algorithm msSelect).
 *
 * Conventions shared by every entry point
 *  - Order.  Keys are compared by value (u32, u64 unsigned; i32 signed;
 *    f32 and bf16 by IEEE 754 totalOrder: -NaN < -inf < ... < -0 < +0 < ...
 *    < +inf < +NaN).  Ties are broken by position, as the paper makes every
 *    value unique by pairing it with its object (Section 2): the pair
 *    (key, index) is unique, so the selected set is unique and exact.
 *  - Memory.  Every pointer whose name starts with d_ is GPU global memory
 *    owned by the caller; the library never frees it.  Pointers without the
 *    prefix are host memory.  Inputs are read only.  Outputs must not overlap
 *    inputs or each other.  Keys may sit at any byte offset that is a multiple
 *    of the key size; 16-byte-aligned keys take the vectorised path.
 *  - Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream).  Calls enqueue work and return without waiting.
 *  - Errors.  Argument errors are returned at once and enqueue nothing.
 *    Errors found on the device are latched in the context and returned by
 *    topk_status_sync().  TOPK_ECUDA reports a failed CUDA runtime call.
 *  - Output order.  The k selected pairs are written in no particular order.
 *  - Threads.  A context is used by one host thread at a time.
 */
#ifndef TOPK_H
#define TOPK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TOPK_U32 = 0,  /* uint32_t */
    TOPK_I32 = 1,  /* int32_t */
    TOPK_F32 = 2,  /* IEEE binary32 */
    TOPK_BF16 = 3, /* bfloat16 (upper half of a binary32) */
    TOPK_U64 = 4   /* uint64_t */
} topk_dtype;

typedef enum {
    TOPK_OK = 0,
    TOPK_EINVAL = 1,     /* bad argument; nothing was enqueued */
    TOPK_ENOMEM = 2,     /* device scratch could not be allocated */
    TOPK_ECUDA = 3,      /* a CUDA runtime call failed */
    TOPK_ETIMEOUT = 4,   /* a bounded device wait gave up */
    TOPK_EBUDGET = 5,    /* serving: request exceeds the HBM budget */
    TOPK_EBUSY = 6,      /* serving: no free slot / queue full */
    TOPK_EINTERNAL = 7   /* recursion did not converge within its level limit */
} topk_status;

/* Flags for topk_params.flags. */
#define TOPK_FLAG_CHECK_SORTED 0x1u  /* sorted runs: verify order, else EINVAL */
#define TOPK_FLAG_RAW_DELTA 0x2u     /* use delta_factor alone as the pivot
                                        margin (testing: provokes pivot
                                        failures, results stay exact) */
#define TOPK_FLAG_TINY_CAND 0x4u     /* testing: minimal candidate buffers so
                                        the overflow paths run */
#define TOPK_FLAG_NO_BULK_COPY 0x8u  /* first pass: per-thread vector loads
                                        instead of the bulk-copy pipeline */
#define TOPK_FLAG_LARGEST 0x10u      /* topk_select, topk_select_kth: the
                                        k largest keys instead of the k
                                        smallest (equal keys still by the
                                        smaller position); the rank-k key is
                                        the smallest selected one.  The
                                        batched, tuning and sorted-runs calls
                                        return TOPK_EINVAL for it */

/* Tuning knobs; a zero field means "choose automatically".  None of them can
 * change a result, only the time taken. */
typedef struct {
    uint64_t seed;             /* Philox4x32-10 key for the sampler */
    uint32_t partitions;       /* p: sampling partitions (the paper's PEs) */
    uint32_t sample_size;      /* s: sample drawn per recursion level */
    uint32_t buckets;          /* reserved; the method uses 3 (a, b, c) */
    uint32_t finish_threshold; /* T: at most this many candidates are
                                  finished by one thread block */
    float delta_factor;        /* z: pivot margin in standard deviations */
    uint32_t flags;            /* TOPK_FLAG_* */
    uint32_t block_threads;    /* topk_select_batched: threads per block
                                  (256, 512 or 1024); the block's finish
                                  capacity, and so the largest T, is 16, 8 or
                                  4 Ki composites of 32-bit keys for 1024,
                                  512 or 256 threads (half for u64) */
    uint32_t split_rows;       /* topk_select_batched: rows longer than this
                                  (and than T) take their first level over
                                  the whole GPU instead of one block;
                                  0xFFFFFFFF: no row does */
} topk_params;

/* Counters of the last completed call on a context (valid after
 * topk_status_sync). */
typedef struct {
    uint32_t levels_grid;      /* recursion levels run by the whole grid; for the
                                  sorted-runs calls, pivot rounds run by the grid */
    uint32_t levels_block;     /* recursion levels (sorted runs: rounds) run
                                  inside one block */
    uint32_t pivot_failures;   /* levels whose bracket missed rank k */
    uint32_t overflows;        /* levels whose candidates exceeded the buffer */
    uint64_t first_candidates; /* |b| after the first level */
    uint64_t sample_kept;      /* sample size of the first level */
} topk_stats;

typedef struct topk_ctx topk_ctx;

/* Creates a context on `device`: owns device scratch (grown on demand) and
 * the latched device status.  Returns TOPK_EINVAL for a bad device. */
topk_status topk_ctx_create(topk_ctx **out, int device);

/* Waits for the context's work, frees its scratch and the context. */
void topk_ctx_destroy(topk_ctx *ctx);

/* Pre-allocates scratch for selections of up to n keys of `dtype`, so that
 * later calls of that size allocate nothing (needed before stream capture).
 * Synchronous. */
topk_status topk_ctx_reserve(topk_ctx *ctx, uint64_t n, topk_dtype dtype);

/* Selection of the k smallest of n unsorted keys (Section 2, Algorithm
 * "select"; Section 4.1).
 *   d_keys     n keys of `dtype`, contiguous.
 *   n, k       1 <= k <= n < 2^32.
 *   d_out_keys k keys of `dtype`: the selected keys, bit-identical to the
 *              input (any order).
 *   d_out_idx  k uint32: their positions in d_keys (same order as keys).
 *   d_kth_key  1 key of `dtype`: the key of rank k (the largest selected).
 *   d_kth_idx  1 uint32: its position.
 *   params     NULL or tuning knobs.
 *   stream     cudaStream_t.
 * Returns TOPK_EINVAL for k == 0, k > n, n >= 2^32, a NULL pointer, an
 * unknown dtype or keys not aligned to their size. */
topk_status topk_select(topk_ctx *ctx, const void *d_keys, uint64_t n, uint64_t k,
                        topk_dtype dtype, void *d_out_keys, uint32_t *d_out_idx,
                        void *d_kth_key, uint32_t *d_kth_idx,
                        const topk_params *params, void *stream);

/* The key of rank k alone (Section 4: the problem asks for the k smallest
 * or for the element of rank k): topk_select whose selected set is formed
 * in context-owned device memory (k keys and k uint32 positions, grown on
 * demand; growing waits for the device) and not returned.  Arguments,
 * flags (TOPK_FLAG_LARGEST: the k-th largest) and errors as topk_select. */
topk_status topk_select_kth(topk_ctx *ctx, const void *d_keys, uint64_t n, uint64_t k,
                            topk_dtype dtype, void *d_kth_key, uint32_t *d_kth_idx,
                            const topk_params *params, void *stream);

/* Multisequence selection over p locally sorted runs (Section 4.2;
 * Appendix A, Algorithm msSelect, with several pivots per round as in
 * Section 4.3 "Multiple Concurrent Trials").
 *   d_keys     uint64 keys of all runs back to back (dtype must be TOPK_U64).
 *   d_run_off  p + 1 uint64 offsets: run r is d_keys[off[r] .. off[r+1]),
 *              non-decreasing within the run; off[0] = 0.
 *   p          number of runs, >= 1.
 *   k          1 <= k <= off[p] < 2^32 (k > off[p] is reported by
 *              topk_status_sync() as TOPK_EINVAL, the offsets being device
 *              data); p <= 2^24.
 *   d_split    p uint64: how many of the k smallest lie in run r; the first
 *              d_split[r] keys of run r are selected.
 *   d_kth_key, d_kth_run, d_kth_pos  the pair of rank k: its key, run and
 *              position inside the run.
 * params->sample_size, when set, is the number of pivots per round
 * (default 64, at most 256).
 * Ties are ordered by (run, position).  TOPK_FLAG_CHECK_SORTED makes the
 * device verify the runs' order and report TOPK_EINVAL from
 * topk_status_sync() when a run is not sorted. */
topk_status topk_select_sorted_runs(topk_ctx *ctx, const void *d_keys,
                                    const uint64_t *d_run_off, uint32_t p, uint64_t k,
                                    topk_dtype dtype, uint64_t *d_split,
                                    void *d_kth_key, uint32_t *d_kth_run,
                                    uint64_t *d_kth_pos, const topk_params *params,
                                    void *stream);

/* Flexible-k multisequence selection (Section 4.3, Algorithm amsSelect, with
 * d concurrent trials per round as in "Multiple Concurrent Trials"): selects
 * the k smallest objects of the p sorted runs for some k with
 * kmin <= k <= kmax that the search finds first, and reports that k.  Each
 * trial estimates an object of rank in [kmin, kmax] as the minimum over the
 * runs of each run's x-th smallest undecided object (x a geometric deviate
 * with the success rate the paper derives), or the maximum of x-th largest
 * ones when the range lies in the upper part; a trial whose exact rank falls
 * in the range ends the search, otherwise the tightest under- and
 * over-estimates narrow every run's bracket.  The result is exact for the k
 * returned: the same objects as topk_select_sorted_runs with that k.
 *   Arguments as topk_select_sorted_runs, with 1 <= kmin <= kmax < 2^32
 *   (kmin > off[p] is reported by topk_status_sync() as TOPK_EINVAL; kmax
 *   above off[p] is clamped to it) and
 *   d_k        1 uint64 (caller-owned device memory): the k chosen.
 * params->sample_size, when set, is the number of trials per round
 * (default 64, at most 256); params->seed seeds the deviates.  Which k is
 * chosen depends on the seed and on d; the selection for that k does not. */
topk_status topk_select_sorted_runs_flexible(topk_ctx *ctx, const void *d_keys,
                                             const uint64_t *d_run_off, uint32_t p, uint64_t kmin,
                                             uint64_t kmax, topk_dtype dtype, uint64_t *d_split,
                                             void *d_kth_key, uint32_t *d_kth_run,
                                             uint64_t *d_kth_pos, uint64_t *d_k,
                                             const topk_params *params, void *stream);

/* Bulk deleteMin* of the bulk priority queue (Section 5): the queue is the
 * p sorted runs, each with a cursor; the objects of run r before its cursor
 * are already deleted.  One call deletes the k smallest remaining objects
 * by multisequence selection over the suffixes (Appendix A, msSelect,
 * every bracket starting at the cursor instead of 0) and advances the
 * cursors past them.  The objects deleted by run r are
 * d_keys[off[r] + old cursor .. off[r] + new cursor); they are the k
 * smallest of what remained, ties ordered by (run, position).
 *   Arguments as topk_select_sorted_runs, and
 *   d_cursor   p uint64 (caller-owned device memory, read and written):
 *              in, the cursor of each run (0 <= cursor <= run length, a
 *              larger one is reported by topk_status_sync() as
 *              TOPK_EINVAL); out, the cursor after the deletion.
 *   k          1 <= k < 2^32; k above the objects that remain is reported by
 *              topk_status_sync() as TOPK_EINVAL (cursors then undefined).
 *   d_kth_key, d_kth_run, d_kth_pos  the largest object deleted: its key,
 *              run and position inside the run.
 * Deleting k1 and then k2 leaves the same cursors as deleting k1 + k2 at
 * once.  Insertion (Section 5's insert*) is the caller's: a run appended to
 * d_keys with its offset and a zero cursor joins the queue. */
topk_status topk_runs_delete_min(topk_ctx *ctx, const void *d_keys, const uint64_t *d_run_off,
                                 uint32_t p, uint64_t *d_cursor, uint64_t k, topk_dtype dtype,
                                 void *d_kth_key, uint32_t *d_kth_run, uint64_t *d_kth_pos,
                                 const topk_params *params, void *stream);

/* Flexible bulk deleteMin* (Section 5 with Section 4.3): deletes the k
 * smallest remaining objects for some kmin <= k <= kmax found by the
 * amsSelect search of topk_select_sorted_runs_flexible, writes that k to
 * d_k (1 uint64, caller-owned device memory) and advances the cursors as
 * topk_runs_delete_min does.  kmax above the objects that remain is
 * clamped to them; kmin above them is reported as TOPK_EINVAL. */
topk_status topk_runs_delete_min_flexible(topk_ctx *ctx, const void *d_keys,
                                          const uint64_t *d_run_off, uint32_t p,
                                          uint64_t *d_cursor, uint64_t kmin, uint64_t kmax,
                                          topk_dtype dtype, void *d_kth_key,
                                          uint32_t *d_kth_run, uint64_t *d_kth_pos,
                                          uint64_t *d_k, const topk_params *params,
                                          void *stream);

/* Many independent selections in one persistent launch (no counterpart in the
 * paper: it is the selection of Section 2 run once per row).
 *   d_keys     all rows back to back, `dtype`.
 *   d_row_off  rows + 1 uint64 offsets (row i = keys[off[i] .. off[i+1])).
 *   d_row_k    rows uint32: k of each row, 1 <= k_i <= row length.
 *   rows       >= 1.
 *   d_out_keys, d_out_idx  per row k_i keys / row-local uint32 positions at
 *              [d_out_off[i], d_out_off[i] + k_i).
 *   d_out_off  rows + 1 uint64 output offsets (caller computes the prefix sum
 *              of d_row_k).
 *   d_kth_keys, d_kth_idx  rows entries: each row's key and position of
 *              rank k_i.
 * Row lengths must be < 2^32.  Rows with bad k are reported by
 * topk_status_sync() as TOPK_EINVAL (their outputs are left untouched).
 * Rows longer than the split length (params->split_rows, default 2^15)
 * run their first recursion level over the whole GPU: one block draws the
 * row's sample and pivots, one grid-wide pass classifies the tiles of all
 * such rows, and the persistent kernel finishes them from their candidates
 * (a fixed pool of 2^23 candidate pairs; a row it cannot hold is selected
 * by one block).
 * When params is NULL, or leaves block_threads, sample_size,
 * finish_threshold and split_rows all zero, the choice remembered by
 * topk_tune_batched for this dtype and row count (power-of-two bucket) is
 * used if there is one, else 1024 threads, a 2048-element sample, the
 * largest T and a split length of 2^15. */
topk_status topk_select_batched(topk_ctx *ctx, const void *d_keys,
                                const uint64_t *d_row_off, const uint32_t *d_row_k,
                                uint32_t rows, topk_dtype dtype, void *d_out_keys,
                                uint32_t *d_out_idx, const uint64_t *d_out_off,
                                void *d_kth_keys, uint32_t *d_kth_idx,
                                const topk_params *params, void *stream);

/* ---- Top-k most frequent objects (Section 7) ---- */

#define TOPK_FREQ_PAC 0u /* Section 7.1: sample counts of the sampled objects */
#define TOPK_FREQ_EC 1u  /* Section 7.2: exact counts of the k* candidates */

typedef struct {
    uint32_t algorithm;    /* TOPK_FREQ_PAC or TOPK_FREQ_EC */
    uint32_t k;            /* objects returned, >= 1 */
    double epsilon;        /* accuracy target eps > 0 (error < eps * n) */
    double delta;          /* failure probability, 0 < delta < 1 */
    double rho;            /* sampling probability in (0, 1]; 0 = from eps
                              and delta (PAC: equation sampleSize; EC:
                              2 ln(n / delta) / (eps^2 k*) objects) */
    uint32_t kstar;        /* EC: candidates counted exactly, >= k; 0 = from
                              eps and delta: max(k, sqrt(2 log2(p) / p *
                              ln(n / delta)) / eps) */
    uint32_t pes;          /* p of the k* formula; 0 = 1 (one GPU) */
    uint64_t seed;         /* Philox4x32-10 key of the sample decisions */
    uint64_t max_distinct; /* most distinct sampled objects the hash table
                              must hold (it has the next power of two above
                              twice this many slots, 8 bytes each); 0 = 2^22;
                              lowered to a bound on the sample size (its
                              mean plus eight standard deviations plus 1024,
                              at most n) */
} topk_freq_params;

/* Sampling probability rho and k* that topk_frequent would use for n
 * objects (host only, no device work).  Returns TOPK_EINVAL for a zero k or
 * n, an unknown algorithm, eps <= 0 or delta outside (0, 1) where they are
 * needed, rho outside (0, 1], or k* < k. */
topk_status topk_frequent_plan(uint64_t n, const topk_freq_params *fp, double *rho,
                               uint32_t *kstar);

/* Top-k most frequent objects of n uint32 objects on one GPU (Section 7):
 * a Bernoulli sample with probability rho (object i is sampled iff word
 * i % 4 of Philox4x32-10 at counter (i / 4 low, i / 4 high, 0x53414d50, 0)
 * and key (seed low, seed high) is below floor(rho * 2^32); every object
 * when rho = 1) is counted in a hash table (block-local tables in shared
 * memory flushed into one table in device memory); then
 *   TOPK_FREQ_PAC (Algorithm PAC): the k most frequently sampled objects,
 *     d_out_count = their sample counts (the paper's estimate of an
 *     object's frequency is sample count / rho);
 *   TOPK_FREQ_EC (Algorithm EC): the k* most frequently sampled objects are
 *     counted exactly over the whole input, d_out_count = the exact counts
 *     of the k most frequent of them (k* <= 4096).
 * "Most frequent" orders by count, larger first, equal counts by the
 * smaller object, so the result is unique for a given seed.
 *   d_objects     n uint32 (dtype TOPK_U32), 4-byte aligned, 1 <= n < 2^32 - 1.
 *   d_out_obj     k uint32, d_out_count k uint64 (caller-owned device
 *                 memory): the objects and counts, in no particular order.
 *   d_sample_size NULL or 1 uint64: the number of sampled objects.
 * The hash table and candidates live in context-owned device memory (grown
 * on demand).  Returns TOPK_EINVAL for bad arguments (as
 * topk_frequent_plan, plus k* > 4096 for EC and a NULL pointer).  Reported
 * by topk_status_sync(): TOPK_EINVAL when fewer than k (PAC) or k* (EC)
 * distinct objects were sampled, TOPK_ENOMEM when more distinct objects
 * were sampled than the table holds (raise max_distinct; an overfilled
 * table ends the call in bounded time, its counts then undefined). */
topk_status topk_frequent(topk_ctx *ctx, const void *d_objects, uint64_t n, topk_dtype dtype,
                          const topk_freq_params *fp, uint32_t *d_out_obj,
                          uint64_t *d_out_count, uint64_t *d_sample_size, void *stream);

/* Autotuner of topk_select_batched (no counterpart in the paper): runs the
 * given batch with every candidate block size (256, 512, 1024 threads),
 * sample size (512, 1024, 2048, 4096) and finish threshold (the block's
 * capacity and half of it), then with the fastest of those and every split
 * length of 2^13, 2^15, 2^17 and none, times each with CUDA events on
 * `stream` (best of three after one warm-up), and remembers the fastest for
 * this dtype and row-count bucket (floor(log2(rows))) in the context.
 * Arguments as topk_select_batched; every output is overwritten many times
 * (the last run uses the chosen setting, so the outputs are that call's
 * result).
 *   base   NULL or settings copied into every candidate (seed, partitions,
 *          delta_factor, flags).
 *   best   NULL or receives the chosen settings.
 * Blocks the calling thread until the measurements are done.  Returns the
 * first error of any run (argument errors as topk_select_batched, device
 * errors as topk_status_sync). */
topk_status topk_tune_batched(topk_ctx *ctx, const void *d_keys, const uint64_t *d_row_off,
                              const uint32_t *d_row_k, uint32_t rows, topk_dtype dtype,
                              void *d_out_keys, uint32_t *d_out_idx, const uint64_t *d_out_off,
                              void *d_kth_keys, uint32_t *d_kth_idx, const topk_params *base,
                              topk_params *best, void *stream);

/* The autotuner's remembered choices as a text file: a header line
 * ("topk-tuning 2"), then one line per entry: GPU name, dtype, row-count
 * bucket, block_threads, sample_size, finish_threshold, split_rows, separated
 * by tabs (files of version 1, without split_rows, are read too).  save writes every entry
 * of the context (TOPK_ECUDA if the file cannot be written); load adds the
 * entries whose GPU name matches this context's device and returns
 * TOPK_EINVAL for a missing or malformed file.  Host only; synchronous. */
topk_status topk_tuning_save(topk_ctx *ctx, const char *path);
topk_status topk_tuning_load(topk_ctx *ctx, const char *path);

/* Selection without any allocation: the same computation and result as
 * topk_select, for callers that cannot allocate device memory at the point
 * of the call (no counterpart in the paper).  Such callers include code
 * running inside another framework's allocator or memory-pool callbacks
 * (where allocating again would re-enter that allocator), latency-critical
 * paths that cannot accept the device-wide synchronisation cudaMalloc /
 * cudaFree may cause, and programs that fix their device memory at start-up.
 * The library's scratch for this call (about 12 MiB: state, counters and two
 * candidate buffers of 2^19 pairs) is a fixed array in device memory that is
 * created when the library is loaded and held by every GPU that loads it
 * until the process exits.  No context is needed; the call runs on the
 * current device.
 *   Arguments as topk_select (no params: the default tuning), with n limited
 *   to 2^22 (4194304) keys; larger n returns TOPK_EINVAL and enqueues
 *   nothing.  Every buffer (keys, outputs, d_status) must be memory of the
 *   current device, else TOPK_EINVAL.
 *   d_status   NULL or one caller-owned uint32 in device memory: set to 0 by
 *              the call and to a topk_status code if the device work fails.
 *              With NULL, a failure of the device work is not reported to
 *              the caller at all (the outputs are then undefined).
 * The first call on a device does a one-time set-up there: it looks up the
 * array's device address (cudaGetSymbolAddress) and sets the kernel
 * attributes and launch geometry of all five key types.  The call itself
 * calls no cudaMalloc, cudaFree or other allocating routine.  All calls in
 * the process share the one array per device, which keeps the contents left
 * by the last call (each call clears what must start at zero): calls whose
 * work may overlap on the GPU (different streams, or threads) race and must
 * be serialised by the caller. */
topk_status topk_select_noalloc(const void *d_keys, uint64_t n, uint64_t k,
                                topk_dtype dtype, void *d_out_keys, uint32_t *d_out_idx,
                                void *d_kth_key, uint32_t *d_kth_idx, uint32_t *d_status,
                                void *stream);

/* ------------------------------------------------------------- serving
 * A request loop over one GPU (no counterpart in the paper): requests are
 * submitted without blocking, admitted in arrival order while the bytes they
 * pin on the device (input + outputs + per-request state) stay within
 * `hbm_budget`, and run concurrently on `max_slots` streams.  Waiting
 * requests of at most 2^18 keys and the same key type are grouped into one
 * batched launch as they arrive (continuous batching); larger ones run as
 * single selections on their own stream.  Every request's result is the one
 * topk_select returns for it alone.  Buffers are caller-owned and must stay
 * valid until the request is done. */
typedef struct topk_server topk_server;

typedef struct {
    const void *d_keys;    /* n keys of dtype */
    uint64_t n, k;         /* 1 <= k <= n < 2^32 */
    topk_dtype dtype;
    void *d_out_keys;      /* k keys */
    uint32_t *d_out_idx;   /* k positions */
    void *d_kth_key;       /* 1 key */
    uint32_t *d_kth_idx;   /* 1 position */
    uint64_t arrival_ns;   /* scheduled arrival on topk_serve_now_ns()'s clock;
                              0 = the time of submission */
} topk_request;

typedef struct {
    uint64_t submitted, completed, rejected, failed;
    uint64_t keys;          /* keys of completed requests */
    uint64_t p50_ns, p99_ns, max_ns; /* latency = completion - arrival */
    uint64_t batches;       /* batched launches */
    uint64_t batched_requests;
    uint64_t peak_inflight_bytes;
    double elapsed_s;       /* first arrival to last completion */
    uint64_t reserved_bytes; /* device memory the server's slots hold beside
                                the budget: each slot's scratch (sized at
                                creation for a 2^26-key selection and a
                                2048-row batch, grown by larger requests),
                                its fixed words and pointer arrays */
    uint64_t budget_waits;  /* requests that reached the head of the queue
                               and had to wait for room in the budget */
} topk_serve_report;

/* Creates a server on `device` with `max_slots` streams (1..64) and a
 * budget in bytes.  Starts the server's worker thread.  Every slot owns a
 * context whose scratch is reserved up front for a selection of 2^26 64-bit
 * keys and a batch of 2048 rows (about 0.6 GiB per slot, outside the
 * budget, which covers the requests' own inputs, outputs and state), so that
 * serving seldom allocates; larger requests grow it on first use.
 * topk_serve_stats reports what the slots hold as reserved_bytes.
 * TOPK_ENOMEM if that memory is not available. */
topk_status topk_serve_create(topk_server **out, int device, uint64_t hbm_budget,
                              uint32_t max_slots);

/* Queues a request; *ticket identifies it.  Returns TOPK_EINVAL for bad
 * arguments and TOPK_EBUDGET when the request alone exceeds the budget
 * (counted as rejected); nothing is queued then.  Never blocks on the GPU. */
topk_status topk_serve_submit(topk_server *srv, const topk_request *req, uint64_t *ticket);

/* *done = 1 when the request has finished (its outputs are written). */
topk_status topk_serve_poll(topk_server *srv, uint64_t ticket, int *done);

/* Waits up to timeout_ns for the request: returns its final status, or
 * TOPK_ETIMEOUT if it is still running (it keeps running). */
topk_status topk_serve_wait(topk_server *srv, uint64_t ticket, uint64_t timeout_ns);

/* Counters and latency percentiles of the requests completed so far. */
topk_status topk_serve_stats(topk_server *srv, topk_serve_report *out);

/* Open-loop replay of a request trace (a load generator; no counterpart in
 * the paper): submits reqs[i] when topk_serve_now_ns() reaches
 * reqs[i].arrival_ns (at once when that is 0 or past), in order, from the
 * calling thread.  done_before[i] (< i, or -1 for none) names the earliest
 * earlier requests whose outputs reqs[i] reuses: the call first waits until
 * every request with index <= done_before[i] has finished.  tickets[i]
 * receives the ticket (0 when the request was rejected); lag_ns (NULL or
 * count entries) how late each submission was against its schedule.  All
 * arrays are host memory.  Returns when the last request is submitted (not
 * finished); TOPK_ETIMEOUT if a wait exceeded 60 s, TOPK_EINVAL for bad
 * arguments (done_before[i] >= i included). */
topk_status topk_serve_replay(topk_server *srv, const topk_request *reqs, const int64_t *done_before,
                              uint64_t count, uint64_t *tickets, uint64_t *lag_ns);

/* The server's clock (steady, nanoseconds), for topk_request.arrival_ns. */
uint64_t topk_serve_now_ns(topk_server *srv);

/* Drains every queued and running request, stops the worker, frees the
 * server. */
void topk_serve_destroy(topk_server *srv);

/* Synchronises `stream`, then returns and clears the first error latched by
 * device code of this context (TOPK_OK if none). */
topk_status topk_status_sync(topk_ctx *ctx, void *stream);

/* Counters of the last selection (call after topk_status_sync). */
topk_status topk_last_stats(topk_ctx *ctx, topk_stats *out);

/* Human-readable name of a status code (static string). */
const char *topk_status_string(topk_status s);

/* Measurement hooks (off by default).  When enabled, every call on the
 * context counts its kernel launches, and the first-level pass of
 * topk_select (the kernel that streams all n keys) is bracketed by CUDA
 * events recorded on the call's stream.  topk_ctx_profile_read() synchronises
 * those events and returns the summed pass time in milliseconds, the number
 * of passes timed and the number of kernel launches since the last reset. */
topk_status topk_ctx_profile(topk_ctx *ctx, int enable);
topk_status topk_ctx_profile_read(topk_ctx *ctx, double *pass_ms, uint64_t *passes,
                                  uint64_t *launches, int reset);

/* Diagnostic: fills d_out[4*i .. 4*i+3] with Philox4x32-10 (Salmon, Moraes,
 * Dror, Shaw, SC'11) of counter {c0 + i, c1, c2, c3} and key {k0, k1}, for
 * i < count, on the device.  Lets a test pin the sampler's generator to the
 * published known-answer vectors.  Synchronous. */
topk_status topk_debug_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                              uint32_t k0, uint32_t k1, uint32_t *d_out,
                              uint32_t count);

/* Diagnostic of the failure path of device waits (no counterpart in the
 * paper): enqueues on `stream` one block that waits, bounded by limit_us
 * microseconds (1 .. 10^6), for a pipeline barrier that nothing completes.
 * The wait expires, TOPK_ETIMEOUT is latched in the context exactly as a
 * stalled bulk-copy pipeline latches it, and the kernel returns: the next
 * topk_status_sync() reports TOPK_ETIMEOUT (and clears it), and the context
 * stays usable.  Returns TOPK_EINVAL for a NULL context or a limit out of
 * range. */
topk_status topk_debug_wait_timeout(topk_ctx *ctx, uint32_t limit_us, void *stream);

#ifdef __cplusplus
}
#endif
#endif
