/*
 * cq.h -- C ABI of the B300 continuous windowed group-by engine.
 *
 * One query maintains, for every group g in [0, groups), the aggregates
 * SUM (int64), COUNT (int32), MIN (int32), MAX (int32) and AVG (double) of
 * the int32 values of the tuples currently in a count-based sliding window.
 * This is the continuous aggregate query of Section 3 of the paper (a
 * group-by over (id, attr) tuples whose aggregate depends on a fixed-size
 * window of the most recent values), fed in iterations of batches
 * (Section 3.1), with skewed group ids handled at run time (Section 4).
 *
 * Window reading: the window is global and count based.  After pushes that
 * total N tuples (stream indices 0 .. N-1) it holds the tuples with stream
 * index in [max(0, N - window), N).  A batch longer than the window
 * contributes only its last `window` tuples.  Results are emitted after
 * every push for every group: an empty group reads SUM 0, COUNT 0,
 * MIN INT32_MAX, MAX INT32_MIN and AVG the quiet NaN 0x7FF8000000000000;
 * otherwise AVG = (double)SUM / (double)COUNT in IEEE binary64 with round to
 * nearest even (both the conversion and the division).  All results are
 * exact; they do not depend on launch shape, tuning options or the order in
 * which the GPU applies updates.
 *
 * Pointers: arguments named d_* are device pointers (cudaMalloc / torch
 * CUDA tensors) of the current device; h_* are host pointers (pinned or
 * pageable).  Sizes are element counts.  The library never frees caller
 * memory and never keeps a caller pointer after the call's stream work has
 * completed.
 *
 * Streams: every call of a query is ordered on that query's CUDA stream
 * (the one given to cq_create, or a library-owned stream if NULL).  Calls
 * return as soon as the work is enqueued unless stated otherwise.
 *
 * Errors: every call returns a cq_status.  A key outside [0, groups) found
 * by a push poisons the query: the push (or, because pushes are
 * asynchronous, the next call that observes it -- at the latest cq_sync)
 * returns CQ_EKEY and every later call except cq_destroy returns
 * CQ_EPOISONED.  Kernels never read or write outside the query's buffers,
 * whatever the keys.  A CUDA failure returns CQ_ECUDA.  A push (or group
 * push, for each member it had begun) that fails after its window
 * bookkeeping began -- a launch error, or scratch it could not allocate --
 * leaves the query's window state inconsistent: that push returns the
 * failure (CQ_ECUDA, CQ_ENOMEM) and poisons the query, so that every later
 * call except cq_destroy returns CQ_EPOISONED.
 *
 * Threading: a query has no internal lock; drive one query from one host
 * thread at a time.  Different queries may be driven concurrently.
 */
#ifndef CQ_H
#define CQ_H

#include <stdint.h>

#if defined(__GNUC__)
#define CQ_API __attribute__((visibility("default")))
#else
#define CQ_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cq_query cq_query;

typedef enum cq_status {
    CQ_OK = 0,
    CQ_EINVAL = 1,      /* bad argument (size out of range, NULL pointer with n > 0, ...) */
    CQ_ENOMEM = 2,      /* device or host allocation failed */
    CQ_EKEY = 3,        /* a pushed key was outside [0, groups); the query is now poisoned */
    CQ_ECUDA = 4,       /* a CUDA runtime call failed */
    CQ_ETIMEOUT = 5,    /* a bounded device wait gave up */
    CQ_EBUSY = 6,       /* resource in use (e.g. a query already in a group) */
    CQ_EPOISONED = 7,   /* the query saw a bad key earlier */
    CQ_EBUDGET = 8,     /* admission refused: the device-memory budget is exhausted */
    CQ_ESCRATCH = 9     /* cq_push_noalloc: the batch needs more than its fixed scratch area */
} cq_status;

/* Aggregate selection for cq_create.  AVG implies SUM and COUNT internally;
 * MIN and MAX enable the exact min/max-under-retraction machinery. */
enum {
    CQ_SUM = 1,
    CQ_COUNT = 2,
    CQ_MIN = 4,
    CQ_MAX = 8,
    CQ_AVG = 16,
    CQ_ALL = 31
};

/* Device-resident result arrays of one query, struct-of-arrays, `groups`
 * entries each.  Library-owned; valid until the next cq_push* or
 * cq_destroy of the query.  Arrays of aggregates that were not requested
 * hold the empty-group sentinels. */
typedef struct cq_result_view {
    int64_t groups;
    const int64_t *sum;
    const int32_t *count;
    const int32_t *min;
    const int32_t *max;
    const double *avg;
} cq_result_view;

/* Create a query over `groups` groups (1 .. 2^30-2) and a window of
 * `window` tuples (1 .. 2^31-1).  `aggs` is a non-empty subset of CQ_ALL.
 * `cuda_stream` is a cudaStream_t (NULL: the library creates its own).
 * Allocates the device-resident state (window ring, per-group state and
 * results; see cq_footprint_bytes).  On success *out owns the query. */
CQ_API cq_status cq_create(int64_t groups, int64_t window, uint32_t aggs, void *cuda_stream, cq_query **out);

/* Device-memory footprint in bytes that cq_create would allocate. */
CQ_API int64_t cq_footprint_bytes(int64_t groups, int64_t window, uint32_t aggs);

/* Push a batch of n >= 0 tuples (d_keys[i], d_vals[i]), i = 0 .. n-1, in
 * stream order (Section 3.1: one iteration).  The tuples entering the
 * window are folded in, the tuples leaving it are retracted and the results
 * of every touched group are rewritten, all on the query's stream.  n = 0 is
 * a no-op; NULL pointers with n > 0 return CQ_EINVAL.  The caller keeps
 * ownership of the batch and may reuse it once the push has completed on
 * the stream (after cq_sync, or after later work ordered on that stream). */
CQ_API cq_status cq_push(cq_query *q, const int32_t *d_keys, const int32_t *d_vals, int64_t n);

/* Same as cq_push for host arrays: the library copies the batch (only the
 * last min(n, window) tuples, the only ones that can enter the window) to
 * one of two library-owned device buffers and pushes it on the query's
 * stream.  The copy runs on a library-owned copy stream as soon as that
 * buffer's previous batch has been pushed, so with pinned host arrays it
 * overlaps the pushes and result copies enqueued before it.  Returns after
 * the copy and the push have been enqueued; the host arrays must stay
 * unchanged until the push has completed (cq_sync). */
CQ_API cq_status cq_push_host(cq_query *q, const int32_t *h_keys, const int32_t *h_vals, int64_t n);

/* Optional per-batch outputs of cq_push_many: device arrays of the caller,
 * NULL when not wanted.  The five result arrays are given all together or
 * not at all; entry (j, g) of each, at j * groups + g, holds group g's
 * result after batch j, as cq_results would have shown it then.  stamps
 * holds 2 * k words of %globaltimer nanoseconds: word j is when the first
 * CTA began work on batch j, word k + j when the last CTA finished it (its
 * latency is the difference; the words are written only by the persistent
 * launch: cq_stats last_path 4). */
typedef struct cq_many_out {
    int64_t *sum;
    int32_t *count;
    int32_t *min;
    int32_t *max;
    double *avg;
    uint64_t *stamps;
} cq_many_out;

/* Push k >= 0 batches in order: batch j is the n[j] tuples (d_keys[j][i],
 * d_vals[j][i]) (host arrays of k device pointers and k lengths).  The
 * results are those of k calls of cq_push with the same batches -- after the
 * call, those after the last batch; `out` (may be NULL) receives the results
 * after every batch.  Iterations of the paper's loop (Section 3.1) run back
 * to back in one persistent cooperative launch (one of each two CTAs of an
 * SM cuts batches into key-range runs, claiming chunks from a per-batch
 * counter, while the other folds earlier batches' runs into the key range
 * it keeps in shared memory; CQ_OPT_STREAM_PRODUCERS can give some SMs two
 * producers), so the per-launch cost is paid once per sequence instead of
 * once per batch.  The
 * launch is split where the MIN/MAX structure must flip (the flip runs
 * between the parts) and every kSMaxBatches (2048) batches.  Queries with
 * more groups than the consumers can keep (about 150,000 with MIN/MAX,
 * 300,000 without), a CQ_OPT_PATH other than 0, or a device where two
 * launch CTAs do not fit one SM, are pushed batch by batch with cq_push's
 * kernels instead, with the same results.  Ownership, ordering and errors
 * are those of cq_push; the batches must stay unchanged until the pushes
 * complete.  Scratch (about 24 bytes per tuple of the longest batch, for
 * each of the four batches in flight) grows on demand like cq_push's. */
CQ_API cq_status cq_push_many(cq_query *q, int k, const int32_t *const *d_keys, const int32_t *const *d_vals,
                              const int64_t *n, const cq_many_out *out);

/* Wait for the query's stream, then fill *out with the device result
 * arrays.  Returns CQ_EKEY / CQ_EPOISONED for a poisoned query. */
CQ_API cq_status cq_results(cq_query *q, cq_result_view *out);

/* Copy the results to host arrays of `groups` elements (any may be NULL)
 * and wait for the copies. */
CQ_API cq_status cq_results_copy(cq_query *q, int64_t *h_sum, int32_t *h_count, int32_t *h_min, int32_t *h_max,
                          double *h_avg);

/* The same copies, enqueued on the query's stream after the pushes before
 * them, without waiting: the host arrays (pinned, for the copies to be
 * asynchronous) hold the results once cq_sync returns or later work on the
 * stream has completed.  A later push does not change them. */
CQ_API cq_status cq_results_copy_async(cq_query *q, int64_t *h_sum, int32_t *h_count, int32_t *h_min,
                                       int32_t *h_max, double *h_avg);

/* Wait for all work of the query; reports a pending bad-key error. */
CQ_API cq_status cq_sync(cq_query *q);

/* Release the query and its device memory (waits for its stream first). */
CQ_API void cq_destroy(cq_query *q);

/* Static description of a status code. */
CQ_API const char *cq_strerror(cq_status s);

/* Tuning knobs.  None of them changes any result; they only change how
 * the work is spread over the GPU.  Values outside a knob's range return
 * CQ_EINVAL. */
typedef enum cq_option {
    CQ_OPT_HOT_KEYS = 1,      /* max heavy hitters privatised per push, 0 .. 128 (0 = off), default  */
                              /* 128; a key with more than n/cap of a push's n inserts always gets  */
                              /* one of the slots in the next push                                    */
    CQ_OPT_HOT_THRESHOLD = 3, /* inserts per push that make a key hot for the next push, 0 = auto   */
    CQ_OPT_WARP_AGG = 4,      /* direct path: 1 combines equal keys within a warp before atomics   */
    CQ_OPT_CTAS_PER_SM = 5,   /* upper bound on co-resident CTAs per SM, 1 .. 8                    */
    CQ_OPT_PARTITION_BITS = 7,/* log2 of the groups per key-range partition, 0 = automatic, 1 .. 11 */
    CQ_OPT_PATH = 8,          /* 0 automatic, 1 partitioned (TMA-staged when aligned), 2 direct   */
                              /* global atomics, 3 partitioned with register-staged chunks only   */
                              /* (cq_push_many: any value but 0 pushes batch by batch that way)   */
    CQ_OPT_WAIT_LIMIT_US = 9, /* bound of every device-side wait of cq_push_many, in microseconds, */
                              /* 1 .. 60,000,000, default 2,000,000; a wait that runs out ends the */
                              /* launch and the query reports CQ_ETIMEOUT (then CQ_EPOISONED)      */
    CQ_OPT_STALL_BATCH = 10,  /* test hook of the timeout path, default -1 (off): in the next      */
                              /* cq_push_many launches one producer CTA never reports this batch   */
                              /* (index within a launch), so the launch's waits on it run out;     */
                              /* results after it are undefined and the query ends poisoned        */
    CQ_OPT_STREAM_PRODUCERS = 11 /* cq_push_many: SMs whose two CTAs both cut batches (producers)  */
                              /* instead of one producer and one consumer, 0 .. 4096 (capped at    */
                              /* the SMs - 1), -1 = automatic (default); a key space too wide for  */
                              /* the fewer consumers' shared memory takes 0.  Never changes results */
} cq_option;

CQ_API cq_status cq_set_option(cq_query *q, cq_option opt, int64_t value);
CQ_API cq_status cq_get_option(const cq_query *q, cq_option opt, int64_t *value);

/* Counters of a query (host-side bookkeeping; no device sync). */
typedef struct cq_query_stats {
    int64_t tuples_seen;     /* N: tuples pushed so far                         */
    int64_t window_len;      /* tuples currently in the window, min(N, window)   */
    int64_t pushes;          /* successful cq_push* calls with n > 0             */
    int64_t flips;           /* front/back flips of the min/max structure         */
    int64_t resets;          /* pushes that replaced the whole window             */
    int64_t hot_keys;        /* heavy hitters the last push detected: the next push privatises them (the
                                call waits for the query's stream to read it) */
    int64_t device_bytes;    /* device memory held by the query                   */
    int64_t kernel_launches; /* kernels launched by the query's pushes so far      */
    int64_t last_path;       /* last push: 1 partitioned, 2 direct, 3 partitioned TMA-staged, 4 the
                                persistent multi-batch launch of cq_push_many */
    int64_t heavy_folds;     /* runs of keys found heavy within a push and folded out of their key
                                range (skew met before the heavy-hitter list knew it), so far */
} cq_query_stats;

CQ_API cq_status cq_stats(const cq_query *q, cq_query_stats *out);

/* Heavy hitters the next push privatises (skew handling, Section 4 of the
 * paper: load is moved off an overloaded worker one batch later): the keys
 * the last push detected, those sure of a slot first (more than n/cap of its
 * n inserts), then the others, at most CQ_OPT_HOT_KEYS in all.  keys[i] and
 * counts[i] (the key's inserts in the detecting push; counts may be NULL)
 * receive min(*n, cap) entries, host memory owned by the caller; *n is the
 * number of entries in the list.  Waits for the query's stream.  CQ_EINVAL
 * for a NULL q, n or keys with cap > 0, or cap < 0. */
CQ_API cq_status cq_hot_list(const cq_query *q, int32_t *keys, int32_t *counts, int cap, int *n);

/* Autotuner.  Measures candidate settings of the tuning knobs (push path,
 * partition width, heavy-hitter cap and threshold, and for the
 * register-staged path CQ_OPT_CTAS_PER_SM = 1 against the query's
 * setting) on a private copy of the
 * query (same groups, window and aggregates, own device memory) fed `trials`
 * pushes of the sample batch (d_keys, d_vals, n device tuples), and applies
 * the fastest to q.  q's window and results are not touched; the call
 * synchronises and allocates a copy of q's state for its duration.  If best
 * is not NULL it receives the chosen settings' mean time per push in
 * microseconds.  A push path pinned with CQ_OPT_PATH (not 0) is kept and
 * only the other knobs are tuned: a query pushed in group launches (cqg_push)
 * is tuned with CQ_OPT_PATH = 1, the group kernel's path, so that it stays a
 * member of the launch.  Tuning never changes any result. */
CQ_API cq_status cq_autotune(cq_query *q, const int32_t *d_keys, const int32_t *d_vals, int64_t n, int trials,
                             double *best_us);

/* Device-side phase tracing (a profiling aid; off by default).  While
 * enabled, every partitioned push overwrites d_stamps with %globaltimer
 * values (nanoseconds): for each CTA b of the launch, CQ_TRACE_STAMPS
 * consecutive words at d_stamps[b * CQ_TRACE_STAMPS] -- kernel start, hot
 * set loaded, phase A done, barrier passed, all deltas gathered and folded,
 * groups finalised, then the first gather batch copied in and applied.  `slots` is the number of 64-bit
 * words of d_stamps (a launch with more CTAs than fit is not traced).
 * A group launch (cqg_push) stamps into the buffer of the first query passed
 * to it, and is then enqueued without its CUDA graph.
 * d_stamps = NULL disables tracing.  The caller owns the buffer. */
#define CQ_TRACE_STAMPS 8
CQ_API cq_status cq_trace(cq_query *q, uint64_t *d_stamps, int64_t slots);

/* Self-check of the AVG division (a diagnostic; touches no query).  Every
 * published AVG is RN(RN(s) / c), the fp64 quotient of a group's SUM s and
 * COUNT c rounded to nearest even (Section 2); the finalisations take it by
 * integer long division, with the fp64 division only for |s| >= 2^53.  This
 * call draws n (s, c) pairs on the current device from the splitmix64 stream
 * seeded by `seed` (|s| of bit length uniform in 0 .. 63 with a random sign,
 * c of bit length uniform in 1 .. 31), computes both quotients there and
 * writes to *mismatches (host memory) how many pairs differ in any bit.
 * Synchronous.  CQ_EINVAL for n < 0 or mismatches = NULL. */
CQ_API cq_status cq_check_avg(int64_t n, uint64_t seed, int64_t *mismatches);

/* ---- many standing queries pushed together ----
 *
 * A group pushes one batch to each of several queries in a single cooperative
 * launch: every query's chunks and key ranges share the GPU, so many small
 * or uneven queries keep all SMs busy where one launch per query would leave
 * most of them idle.  Each query keeps its own options, results and error
 * state.  The group orders its launch after all work already enqueued on
 * each query's stream and makes each query's stream wait for the launch, so
 * group pushes and single pushes of a query may be interleaved freely. */
typedef struct cq_group cq_group;

/* Create a group launching on `cuda_stream` (NULL: a library-owned stream). */
CQ_API cq_status cqg_create(void *cuda_stream, cq_group **out);

/* Push batch i (d_keys[i], d_vals[i], n[i] tuples, device pointers) to
 * queries[i], i = 0 .. nq-1, all in one launch.  Queries must be distinct
 * and on the group's device; a query with n[i] = 0 is skipped.  If status is
 * not NULL, status[i] receives the query's own result (CQ_OK, CQ_EINVAL,
 * CQ_EKEY / CQ_EPOISONED for a poisoned query, whose batch is not pushed).
 * Returns CQ_OK if the launch was enqueued (even when some queries were
 * refused), CQ_EINVAL for bad arguments, CQ_ECUDA on a CUDA failure. */
CQ_API cq_status cqg_push(cq_group *g, int nq, cq_query *const *queries, const int32_t *const *d_keys,
                          const int32_t *const *d_vals, const int64_t *n, cq_status *status);

/* Wait for the group's stream. */
CQ_API cq_status cqg_sync(cq_group *g);

/* Launches made by the group's pushes, and how many of them replayed a
 * captured CUDA graph (a launch is captured once per shape -- number of
 * queries, chunks, key ranges -- and replayed while the shape repeats). */
CQ_API cq_status cqg_stats(const cq_group *g, int64_t *launches, int64_t *graph_launches);

/* Release the group (queries are not affected). */
CQ_API void cqg_destroy(cq_group *g);

/* ---- serving loop ----
 *
 * A server runs many standing queries fed by requests arriving over time
 * (each request: one batch for one query).  One dispatcher thread pushes, in
 * a single group launch, the oldest pending batch of every query that has
 * one (continuous batching; a query's batches are pushed in arrival order),
 * while the previous launch still runs; one completion thread stamps each
 * batch's completion time when its launch has finished.  The latency of a
 * batch is its completion stamp minus its arrival stamp, both read from the
 * host's monotonic clock (cqs_now_ns).  Serving allocates no device memory:
 * a query's state and the push scratch of batches up to its declared maximum
 * are allocated when it is admitted. */
typedef struct cqs_server cqs_server;

typedef struct cqs_server_stats {
    int64_t queries;              /* admitted queries */
    int64_t reserved_bytes;       /* device bytes the admitted queries hold */
    int64_t budget_bytes;
    int64_t submitted, completed; /* batches, since creation or the last reset */
    int64_t tuples;               /* tuples of the completed batches */
    int64_t launches;             /* group launches */
    int64_t batches_launched;     /* batches those launches carried */
    double latency_p50_us, latency_p99_us, latency_max_us, latency_mean_us;  /* of completed batches */
    double busy_s;                /* first arrival to last completion */
} cqs_server_stats;

/* Nanoseconds on the host monotonic clock the server stamps arrivals and
 * completions with. */
CQ_API int64_t cqs_now_ns(void);

/* Create a server on the current device with a device-memory budget of
 * budget_bytes for its queries, launching on `cuda_stream` (NULL: a
 * library-owned stream).  Starts the dispatcher and completion threads. */
CQ_API cq_status cqs_create(int64_t budget_bytes, void *cuda_stream, cqs_server **out);

/* Admit a query (arguments of cq_create) that will take batches of at most
 * max_batch tuples.  Its footprint -- cq_footprint_bytes plus the push
 * scratch of a max_batch batch -- is reserved against the budget: CQ_EBUDGET
 * if it does not fit what is left (nothing is allocated then).  Queries of
 * more than 2^20 groups are refused (CQ_EINVAL): every served query runs in
 * the one group launch.  The query belongs to the server, which destroys it;
 * do not push to it, change its options or destroy it yourself.  Its results
 * (cq_results, cq_results_copy) may be read once cqs_drain has returned and
 * until the next cqs_submit. */
CQ_API cq_status cqs_admit(cqs_server *s, int64_t groups, int64_t window, uint32_t aggs, int64_t max_batch,
                           cq_query **out);

/* Queue a batch of n tuples (device pointers, owned by the caller, who must
 * keep them unchanged until the batch completes) for admitted query q.
 * arrival_ns is the request's arrival on the cqs_now_ns clock (negative: now).
 * *ticket (if not NULL) receives the batch's id for cqs_wait.  CQ_EINVAL for
 * an unknown query or n > its max_batch.  Thread-safe. */
CQ_API cq_status cqs_submit(cqs_server *s, cq_query *q, const int32_t *d_keys, const int32_t *d_vals, int64_t n,
                            int64_t arrival_ns, int64_t *ticket);

/* Wait for batch `ticket`; returns its status (that of the push, as cq_push
 * would report it; a bad key surfaces on a later batch of the query). */
CQ_API cq_status cqs_wait(cqs_server *s, int64_t ticket);

/* Wait until every submitted batch has completed. */
CQ_API cq_status cqs_drain(cqs_server *s);

/* Open-loop load: submit batch i (queries[i], d_keys[i], d_vals[i], n[i]) at
 * arrival_ns[i] nanoseconds (non-decreasing) after the call starts,
 * whatever the backlog, from the calling thread; then drain. */
CQ_API cq_status cqs_replay(cqs_server *s, int64_t nb, cq_query *const *queries, const int64_t *arrival_ns,
                            const int32_t *const *d_keys, const int32_t *const *d_vals, const int64_t *n);

/* Counters and latency percentiles (nearest rank) since creation or the last
 * reset. */
CQ_API cq_status cqs_stats(cqs_server *s, cqs_server_stats *out);

/* Clear counters, latencies and tickets (CQ_EBUSY unless drained). */
CQ_API cq_status cqs_reset_stats(cqs_server *s);

/* Drain, stop the threads and destroy the server and its queries. */
CQ_API void cqs_destroy(cqs_server *s);

/* ---- one window per group (the paper's own workload) ----
 *
 * Every group g in [0, groups) keeps a window of the last `window` values of
 * its tuples (Section 3.2: a ring per group with a pointer to its oldest
 * value).  Tuples are taken in stream order; after a tuple (k, v) enters
 * group k's window, the window's SUM is recomputed from scratch -- scanned
 * `passes` times, as in the paper's heavier variant (Section 5.1) -- and is
 * that tuple's output.  The sums are exact int64. */
typedef struct cqw_query cqw_query;

#define CQW_MAX_WINDOW (1 << 20)
#define CQW_MAX_PASSES 1000

/* Create on the current device: groups in [1, 2^31 - 1], window in
 * [1, CQW_MAX_WINDOW], passes in [1, CQW_MAX_PASSES]; cuda_stream as for
 * cq_create.  Holds 4 * groups * window bytes of windows plus 12 bytes per
 * group; every window starts empty. */
CQ_API cq_status cqw_create(int64_t groups, int32_t window, int32_t passes, void *cuda_stream, cqw_query **out);

/* Push n tuples (device pointers d_keys, d_vals, owned by the caller); the
 * window SUM after tuple i is written to d_sums[i] (device, n int64, owned
 * by the caller).  Stream-ordered like cq_push; a key outside [0, groups)
 * leaves every window unchanged, poisons the query and is reported by a
 * later call (CQ_EKEY, then CQ_EPOISONED). */
CQ_API cq_status cqw_push(cqw_query *q, const int32_t *d_keys, const int32_t *d_vals, int64_t n, int64_t *d_sums);

/* Wait for the query's stream; reports a poisoned query. */
CQ_API cq_status cqw_sync(cqw_query *q);

/* Tuples pushed, pushes and kernel launches so far (NULL to skip any). */
CQ_API cq_status cqw_stats(const cqw_query *q, int64_t *tuples_seen, int64_t *pushes, int64_t *kernel_launches);

/* Release the query (waits for its stream). */
CQ_API void cqw_destroy(cqw_query *q);

/* ---- the paper's owner-computes execution, with its rebalancing ----
 *
 * The paper's own way to run the per-group windows above (Sections 3.1, 3.2
 * and 4), kept as an ablation beside the build's sort-based cqw path: every
 * GPU thread owns a list of groups and processes their tuples one after
 * another, in stream order; the host keeps the group-to-thread and
 * thread-to-groups mappings, lays each batch out so that a thread's tuples are
 * adjacent (two passes: count per thread, then place), and after laying out a
 * batch runs one of the paper's six policies, which move groups from the most
 * to the least loaded threads for the NEXT batch (a delay of one batch).
 * Initially thread t of T owns groups [t G / T, (t + 1) G / T).  Outputs are
 * those of cqw_push: the window SUM after every tuple, exact.
 *
 * Readings of the policies (where the paper leaves a choice open): the most
 * and least loaded threads break ties by the lower index; moving a group moves
 * its tuples of the current batch; a moved group joins the end of the least
 * loaded thread's list, except that shift and shiftLocal keep ids in order
 * (a group moving down joins the end of the lower thread's list, one moving
 * up the front of the upper's); a thread's tuples are read from its segment
 * of the laid-out batch, restricted to the groups it still owns;
 * checkAll/bestBalance break ties by first occurrence there; probCheck
 * compares count >= pot * tpt / ngroups in double precision; shift moves
 * each thread's group of one step at once; a policy's loop also stops after
 * an iteration that moves nothing and after G moves. */
typedef enum cqo_policy {
    CQO_NONE = 0,          /* no balance                                               */
    CQO_GET_FIRST = 1,     /* move the first group of the most loaded thread             */
    CQO_CHECK_ALL = 2,     /* ... its most frequent group (scans its tuples)             */
    CQO_PROB_CHECK = 3,    /* ... the first group seen pot x (its average) times         */
    CQO_BEST_BALANCE = 4,  /* ... the group whose move best evens the pair                */
    CQO_SHIFT = 5,         /* every thread between the pair passes one group to its side  */
    CQO_SHIFT_LOCAL = 6    /* one pass over neighbours, each pair evened by one group     */
} cqo_policy;

/* OR-ed into cqo_create's policy: lay each batch out and run the policy on
 * the device (Section 4's loop moved onto the GPU).  The mapping lives in
 * device memory; per batch, the tuples are sorted stably by owner thread on
 * the GPU (and, for checkAll, probCheck and bestBalance, by group, for each
 * tuple's rank in its group), the owner kernel runs, and one CTA runs the
 * policy on a second stream while it does; the next batch waits for it (the
 * same delay of one batch).  Offered for CQO_NONE .. CQO_BEST_BALANCE with
 * T <= 16384; the moves, mappings and outputs equal the host mode's.
 * cqo_stats and cqo_mapping then wait for the policy of the last push. */
#define CQO_ON_DEVICE 16

typedef struct cqo_query cqo_query;

typedef struct cqo_stats_t {
    int64_t tuples_seen;   /* tuples pushed                                               */
    int64_t pushes;        /* pushes with n > 0                                           */
    int64_t moves;         /* groups moved between threads so far                         */
    int64_t last_moves;    /* groups moved after the last push                            */
    int64_t last_max_tpt;  /* the last push's largest tuples-per-thread, before its moves */
    int64_t last_min_tpt;  /* ... and smallest                                           */
    int64_t host_ns;       /* host time spent laying batches out and rebalancing (device
                              mode: staging the batch and launching)                  */
} cqo_stats_t;

/* Create on the current device: groups, window and passes as cqw_create;
 * grid = blocks of 256 threads (T = 256 grid owner threads, grid >= 1,
 * T <= groups); policy a cqo_policy; threshold = the tuple-count gap that
 * marks an imbalance (the paper's threadThreshold, >= 0); pot in (0, 1]
 * (probCheck's fraction); cuda_stream as for cq_create. */
CQ_API cq_status cqo_create(int64_t groups, int32_t window, int32_t passes, int32_t grid, int32_t policy,
                            int64_t threshold, double pot, void *cuda_stream, cqo_query **out);

/* Push n tuples from HOST memory (h_keys, h_vals; read before the call
 * returns); the window SUM after tuple i goes to d_sums[i] (device, n int64,
 * owned by the caller), stream-ordered.  A key outside [0, groups) is found
 * on the host: the call returns CQ_EKEY with every window unchanged, and the
 * query is poisoned (later calls: CQ_EPOISONED). */
CQ_API cq_status cqo_push(cqo_query *q, const int32_t *h_keys, const int32_t *h_vals, int64_t n, int64_t *d_sums);

/* Wait for the query's stream. */
CQ_API cq_status cqo_sync(cqo_query *q);

CQ_API cq_status cqo_stats(const cqo_query *q, cqo_stats_t *out);

/* The current thread-to-groups mapping: groups[off[t] .. off[t + 1]) are
 * thread t's, in order (host arrays of T + 1 and G entries, owned by the
 * caller). */
CQ_API cq_status cqo_mapping(const cqo_query *q, int32_t *off, int32_t *groups);

/* One rebalancing step on the host, with no query and no device: the
 * mapping (off, groups as cqo_mapping returns it, T threads, G groups), a
 * batch's keys in stream order (n of them, each in [0, G)) and a policy;
 * writes the mapping the policy leaves (out_off, out_groups) and the number
 * of groups moved.  The step cqo_push runs after laying out a batch. */
CQ_API cq_status cqo_rebalance(int32_t policy, int32_t T, int64_t G, const int32_t *off, const int32_t *groups,
                               const int32_t *keys, int64_t n, int64_t threshold, double pot, int32_t *out_off,
                               int32_t *out_groups, int64_t *moves);

CQ_API void cqo_destroy(cqo_query *q);

/* ---- push without allocation ----
 *
 * The paper has no counterpart: this is a library entry point for callers
 * that may not allocate device memory while they push.  cq_push grows the
 * query's scratch (the partitioned kernel's staged deltas and its table of
 * per-range runs) with cudaMalloc/cudaFree when a batch is
 * larger than any before.  Callers that cannot have that are (a) a server
 * that admitted the query against a fixed device-memory budget
 * (cq_footprint_bytes counts the query's state, not push scratch), so a push
 * must not add to it; and (b) a latency-bound loop with other streams in
 * flight, because cudaFree waits for the whole device and cudaMalloc may.
 *
 * cq_push_noalloc pushes the batch with the results of cq_push (bit for bit)
 * but always through the TMA-staged group kernel, whatever the query's
 * CQ_OPT_PATH setting and whatever path cq_push would pick by itself (the
 * direct-atomics path, or the register-staged kernel cq_push prefers for
 * more than 2^19 groups with short runs).  It takes that kernel's scratch
 * from one fixed area of CQ_NOALLOC_SCRATCH_BYTES bytes per device, a static
 * device array of the library, and calls no allocator (no cudaMalloc,
 * cudaFree or allocating library).  Arguments are those of cq_push; the
 * tuples are device pointers owned by the caller.
 *
 * Set-up: the FIRST call on each device looks up the area's address
 * (cudaGetSymbolAddress), which makes the driver load the library module
 * holding the array and reserve its memory.  Make that first call before any
 * stream capture on the device.
 *
 * Limits and errors: the batch's scratch (about 32 bytes per tuple of the
 * last min(n, window) tuples, plus the run table) must fit the area -- about
 * 770,000 tuples at 100,000 groups, 610,000 at 10^6 groups -- else
 * CQ_ESCRATCH is returned; so it is for a
 * query of more than 2^20 groups, beyond the kernel's 1,024 key-range
 * partitions.  Both checks happen before anything is enqueued: a rejected
 * call leaves the query unchanged.  Other statuses are those of cq_push.
 *
 * Zeroing: only the area's first 8 bytes (the kernel's grid-barrier counter)
 * must start at zero; every call clears them on the query's stream before its
 * launch.  Everything else the kernel writes before it reads it.
 *
 * Races: the area is shared by every query on the device.  Calls whose
 * launches can overlap on the device -- queries on different streams with no
 * ordering between them, or calls from several host threads -- race on it and
 * corrupt each other's results.  Calls ordered on one stream do not. */
#define CQ_NOALLOC_SCRATCH_BYTES (32LL << 20)
CQ_API cq_status cq_push_noalloc(cq_query *q, const int32_t *d_keys, const int32_t *d_vals, int64_t n);

#ifdef __cplusplus
}
#endif

#endif /* CQ_H */
