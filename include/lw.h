/*
 * lw.h -- C ABI of the GB300 Lance-Williams clustering library (liblw.so).
 *
 * The library computes an agglomerative hierarchical clustering (a
 * dendrogram) of n objects from their dissimilarity matrix, smaller meaning
 * more similar (Yarmish, Listowsky, Dexter, "Distributed Lance-William
 * Clustering Algorithm": Abstract and Section 1 state the problem, Section 4 the
 * iteration, Table 1 the coefficients).  Each of the n - 1 merges
 *   1. finds the minimum remaining distance D(i, j), i < j (Section 4 step 1),
 *   2. combines i and j into one cluster kept in slot i; slot j is never used
 *      again (Section 4 step 2; Section 5.3 step 6),
 *   3. recomputes, for every other live cluster k,
 *        D(k, i+j) = a_i D(k,i) + a_j D(k,j) + b D(i,j) + g |D(k,i) - D(k,j)|
 *      with the Table 1 coefficients of the chosen linkage (Section 4 step 3),
 *   4. outputs the step (i, j, D(i, j)) of the tree (Section 4 step 4).
 * All n - 1 merges run inside one persistent cooperative CUDA kernel on one
 * GPU (sm_103a).
 *
 * Exact arithmetic contract (bit-exact, ties included):
 *   - cells are IEEE FP32; every product and sum is rounded to nearest even,
 *     no fused multiply-add; the four terms are added left to right in the
 *     order printed above, all four always evaluated;
 *   - group average: a_i = fl(n_i/(n_i+n_j)), a_j = fl(n_j/(n_i+n_j));
 *     Ward: T = n_i+n_j+n_k, a_i = fl((n_i+n_k)/T), a_j = fl((n_j+n_k)/T),
 *     b = -fl(n_k/T), g = 0; single: (0.5, 0.5, 0, -0.5);
 *     complete: (0.5, 0.5, 0, 0.5) (the form of Section 5.3 step 6);
 *     weighted average: (0.5, 0.5, 0, 0); centroid: a_i, a_j as group
 *     average, b = -fl(float(n_i n_j) / float((n_i+n_j)^2)), the integers
 *     exact, each converted once;
 *   - the minimum is the smallest (value, i, j) in lexicographic order, so
 *     equal distances go to the lowest row i, then the lowest column j.
 *
 * Storage (Section 5.1 / 5.2 keep only the upper triangle): the matrix is the packed
 * row-major strict upper triangle, n(n-1)/2 floats; cell (r, c), r < c, is at
 * index r*n - r*(r+1)/2 + (c - r - 1) (64-bit arithmetic).
 *
 * Errors: every call returns an lw_status; nothing aborts, throws or exits.
 * Device waits inside kernels are bounded; a wait that runs out reports
 * LW_ERR_TIMEOUT and leaves the CUDA context usable.
 */
#ifndef LW_H
#define LW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Linkage rows of Table 1 that this library implements. */
typedef enum {
    LW_SINGLE = 0,   /* a_i = a_j = 1/2, b = 0, g = -1/2 */
    LW_COMPLETE = 1, /* a_i = a_j = 1/2, b = 0, g = +1/2 */
    LW_AVERAGE = 2,  /* a_i = n_i/(n_i+n_j), a_j = n_j/(n_i+n_j), b = g = 0 */
    LW_WARD = 3,     /* a_i = (n_i+n_k)/T, a_j = (n_j+n_k)/T, b = -n_k/T, g = 0 */
    LW_WEIGHTED = 4, /* weighted average: a_i = a_j = 1/2, b = g = 0 */
    LW_CENTROID = 5  /* a_i = n_i/(n_i+n_j), a_j = n_j/(n_i+n_j),
                        b = -n_i n_j/(n_i+n_j)^2, g = 0 (heights may decrease) */
} lw_linkage;

typedef enum {
    LW_OK = 0,
    LW_ERR_INVALID_ARG = 1,   /* bad n, linkage, pointer or handle */
    LW_ERR_INVALID_INPUT = 2, /* a NaN, infinite or negative distance */
    LW_ERR_OOM = 3,           /* device or host allocation failed */
    LW_ERR_CUDA = 4,          /* a CUDA runtime call failed, or the kernel stopped on an
                                 internal check (see lw_last_error); the bounds-checked
                                 build of the library (liblw_checked.so, -DLW_CHECKED,
                                 for testing) reports here a merge-kernel access outside
                                 the job's buffers, with its source line */
    LW_ERR_TIMEOUT = 5,       /* a bounded device wait ran out */
    LW_ERR_BUSY = 6,          /* the context is in use by another call */
    LW_ERR_CANCELLED = 7      /* a served request was cancelled before it ran */
} lw_status;

/* Largest n accepted: cluster sizes stay exact in FP32 and packed indices
 * fit in 64 bits.  The matrix itself must also fit in device memory. */
#define LW_MAX_N (1 << 24)

typedef struct lw_ctx lw_ctx;

/*
 * lw_create -- make a context bound to CUDA device `device`.
 *   out          receives the handle (host pointer, must not be NULL).
 *   cuda_stream  a cudaStream_t on that device to issue all work on, or NULL
 *                for a stream owned by the context.
 * The context owns its device workspace (row-minimum keys 8n B, cluster
 * sizes 4n B, per-CTA exchange records, barrier words) and reuses it across
 * calls; it grows on demand.  Returns LW_ERR_INVALID_ARG for a bad device,
 * LW_ERR_CUDA if the device cannot be used.
 */
lw_status lw_create(lw_ctx **out, int device, void *cuda_stream);

/*
 * lw_cluster -- cluster one matrix; blocks until the outputs are written.
 *   dist         packed upper triangle, n(n-1)/2 FP32 cells, row-major.
 *                If it is a DEVICE pointer it may be used as the working
 *                matrix and OVERWRITTEN in place (the paper's update rewrites
 *                row and column i in place, Section 5.3 step 6): keep a copy
 *                if needed.
 *                If it is a HOST pointer the host array is left unchanged:
 *                page-locked (pinned, mapped) memory is read in place by the
 *                GPU, in one pass over the host link, when the run uses the
 *                row-log layout (multi-CTA runs with room for it, see
 *                LW_OPT_LAYOUT); otherwise, and for pageable memory, the
 *                library copies it to a device buffer owned by the context.
 *                Either way all n(n-1)/2 cells must be readable.
 *   n            number of objects, 1 <= n <= LW_MAX_N.  n == 1: no merges.
 *   linkage      an lw_linkage value.
 *   merges_out   int32[2*(n-1)], host or device: step t is
 *                (merges_out[2t], merges_out[2t+1]) = (i, j), i < j, the
 *                slots of the two clusters merged; slot i keeps the result.
 *   heights_out  float[n-1], host or device: heights_out[t] = D(i, j).
 * Errors: LW_ERR_INVALID_ARG (n out of range, bad linkage, NULL pointer),
 * LW_ERR_INVALID_INPUT (a NaN/inf/negative cell; outputs unspecified and a
 * device dist possibly partly rewritten: -0 cells become +0),
 * LW_ERR_OOM, LW_ERR_CUDA, LW_ERR_TIMEOUT.
 */
lw_status lw_cluster(lw_ctx *ctx, float *dist, int64_t n, int linkage,
                     int32_t *merges_out, float *heights_out);

/*
 * lw_cluster_async -- as lw_cluster for DEVICE pointers only (dist,
 * merges_out, heights_out), but returns as soon as the work is queued on the
 * context's stream.  The status of the run is read by lw_wait.  Returns
 * LW_ERR_INVALID_ARG if a pointer is not device memory.
 */
lw_status lw_cluster_async(lw_ctx *ctx, float *dist, int64_t n, int linkage,
                           int32_t *merges_out, float *heights_out);

/* lw_wait -- synchronise the context's stream and return the status of the
 * last queued run (LW_OK, LW_ERR_INVALID_INPUT, LW_ERR_TIMEOUT, ...). */
lw_status lw_wait(lw_ctx *ctx);

/*
 * lw_get_stats -- counters of the last completed run, written to the host
 * array `stats` (first `count` entries; entries past the last counter are 0):
 *   [0] rounds (each certifies one or more consecutive merges between two
 *       grid barriers),
 *   [1] rounds that certified no merge (waiting for a row refill),
 *   [2] cells rewritten by the update formula (sum over merges of m_t - 2),
 *   [3] CTAs of the persistent grid,
 *   [4] row refills served by all CTAs together,
 *   [5] live cells read by those refills,
 *   [6] refills installed by the rows' owners,
 *   [7] published entries the walks visited (all rounds),
 *   [8..13] with LW_OPT_PHASE_TIMES on: wall-clock nanoseconds summed over
 *       the CTAs of the grid, per phase of a round: [8] barrier waits,
 *       [9] exchange, walk, refill installs and scans, [10] pass 1 (new cells, read
 *       only), [11] the cells after two merges, computed in the window of
 *       the second barrier, [12] certification and bookkeeping, [13] pass 2
 *       (writes, cache upkeep) and publish;
 *   [14] rows rescanned at once by their owner (cache emptied),
 *   [15] live cells read by those rescans,
 *   [16..25] with LW_OPT_PHASE_TIMES on, a finer split of [9], [11], [12]
 *       and [13] (same units): [16] reading the CTAs' records, [17] the
 *       walk with the refill installs and scans beside it, [18] the
 *       chain's sizes, stamps and member
 *       cells, [19] the cross-CTA minima of the new cells, [20] the
 *       certification, [21] bookkeeping and survivor caches, [22] pass 2,
 *       [23] owner rescans; refill scans in the row-log layout: [24] the
 *       log part, [25] the matrix part; [26] the walk alone (part of [17]);
 *   [27..32] with LW_OPT_PHASE_TIMES on, the barriers' own cost: [27] the
 *       waits (ns) of the CTA that arrived last, summed over the barriers
 *       of the loop, [28] those barriers (as counted by the CTAs that
 *       completed them), [29] of them the second barrier of a round, [30]
 *       second barriers completed by a CTA serving a refill that round,
 *       [31] first barriers completed by such a CTA, [32] barriers
 *       completed by CTA 0.
 */
lw_status lw_get_stats(lw_ctx *ctx, int64_t *stats, int count);

/*
 * lw_set_option -- knobs of the context (value 0 = automatic / default):
 *   LW_OPT_GRID       CTAs of the persistent grid, 1..SM count (clamped to
 *                     what fits co-resident);
 *   LW_OPT_TIMEOUT_MS bound of every device wait in milliseconds (default
 *                     5000);
 *   LW_OPT_TEST_SKIP_ARRIVE  failure-detection test hook: CTA `value` of a
 *                     multi-CTA grid returns before the first grid barrier,
 *                     so the other CTAs' bounded waits run out and the call
 *                     reports LW_ERR_TIMEOUT with the context still usable;
 *                     -1 switches it off (the default);
 *   LW_OPT_PHASE_TIMES  1: accumulate per-phase time (lw_get_stats [8..23]);
 *   LW_OPT_BATCH_SPLIT  largest n a batch runs on a single CTA (0: the
 *                     largest that fits one CTA's shared memory); larger
 *                     jobs of a batch run over the whole device;
 *   LW_OPT_CTA_THREADS  threads per CTA of lw_cluster's kernel: 128, 256 or
 *                     512 (0: 512).  Smaller CTAs suit small matrices run
 *                     side by side (several fit one SM);
 *   LW_OPT_LAYOUT     working matrix of a multi-CTA lw_cluster run: 0
 *                     (default) or 1 the row-log layout -- a symmetric n x n
 *                     copy whose rows are rewritten whole, an n x n log of
 *                     each row's cells to later-merged slots and a stamp per
 *                     slot (8n^2 bytes held by the context, used when they
 *                     fit in half the free device memory, else the packed
 *                     triangle), so that every merge moves contiguous words;
 *                     2 the packed triangle (dist itself, no extra memory).
 *                     One-CTA runs always use the packed triangle.  Results
 *                     are the same either way;
 *   LW_OPT_TEST_FAIL_ALLOC  failure-injection test hook: the next `value`
 *                     device allocations of the context (workspace, matrix
 *                     copy, working layout, batch plans) fail on the host,
 *                     before cudaMalloc is called; the call reports
 *                     LW_ERR_OOM and the context stays usable.
 * Returns LW_ERR_INVALID_ARG for an unknown option or value.
 */
enum {
    LW_OPT_GRID = 1,
    LW_OPT_TIMEOUT_MS = 2,
    LW_OPT_TEST_SKIP_ARRIVE = 3,
    LW_OPT_PHASE_TIMES = 4,
    LW_OPT_BATCH_SPLIT = 5,
    LW_OPT_CTA_THREADS = 6,
    LW_OPT_LAYOUT = 7,
    LW_OPT_TEST_FAIL_ALLOC = 8
};
lw_status lw_set_option(lw_ctx *ctx, int option, int64_t value);

/*
 * lw_cluster_noalloc -- lw_cluster for callers that must not allocate.
 * (Not a step of the paper: the paper has no counterpart; this is a service
 * of the library.)
 *
 * For code that cannot call cudaMalloc/cudaFree when it clusters -- inside a
 * memory pool or arena that owns every allocation, inside a host
 * application's plug-in, or in a loop that must never enter the allocator.
 * It needs no lw_ctx and allocates nothing, host or device: the kernel's
 * global scratch (cluster sizes, exchange records, refill lists, barrier
 * words) is a fixed file-scope device array of 2 MB in liblw.so.  The array
 * exists on a device from the moment the library's device code is loaded
 * there -- with CUDA's lazy module loading that is the first call on that
 * device -- and is held until the process exits.  The working matrix is the
 * caller's packed triangle.
 *   dist, merges_out, heights_out  DEVICE pointers as for lw_cluster (dist is
 *                overwritten in place); n <= LW_NOALLOC_MAX_N.
 *   cuda_stream  stream to run on (NULL: the legacy default stream); the call
 *                blocks until the run is finished.
 * Each call looks up the scratch address (cudaGetSymbolAddress) with the
 * current device; the first call on a device also loads the module, so make
 * it before any stream capture begins.  All calls share the one scratch
 * array, which keeps the last call's contents (each call clears what must
 * start zeroed), so calls that overlap on the GPU -- from several host
 * threads or streams at once -- race and must be serialised by the caller.
 * Errors: LW_ERR_INVALID_ARG for n > LW_NOALLOC_MAX_N, a bad linkage or a
 * pointer that is not device memory; LW_ERR_INVALID_INPUT, LW_ERR_TIMEOUT
 * and LW_ERR_CUDA as for lw_cluster.
 */
#define LW_NOALLOC_MAX_N 16384
lw_status lw_cluster_noalloc(float *dist, int64_t n, int linkage, int32_t *merges_out,
                             float *heights_out, void *cuda_stream);

/*
 * Batches: many independent clusterings in one persistent launch.
 *
 * A job whose n is at most the split size (LW_OPT_BATCH_SPLIT, default the
 * largest n one CTA's shared memory can hold) runs entirely on one CTA: the
 * batch kernel keeps one CTA per SM slot busy, each CTA taking the next job
 * from a device work queue until the queue is empty, so thousands of small
 * jobs cost one launch.  Larger jobs run one after another over the whole
 * device, as lw_cluster would run them.  Results are bit-identical to
 * lw_cluster on each job alone.
 */
typedef struct lw_job {
    float *dist;          /* DEVICE packed upper triangle, n(n-1)/2 floats, overwritten */
    int64_t n;            /* 1 <= n <= LW_MAX_N */
    int32_t linkage;      /* lw_linkage */
    int32_t status;       /* out: lw_status of this job (written by lw_batch_wait) */
    int32_t *merges_out;  /* DEVICE int32[2(n-1)] */
    float *heights_out;   /* DEVICE float[n-1] */
} lw_job;

typedef struct lw_batch lw_batch;

/*
 * lw_batch_create -- plan a batch: checks every job (LW_ERR_INVALID_ARG for a
 * bad n, linkage or non-device pointer, with the job's index in
 * lw_last_error), copies the job table to the device, sizes the per-CTA
 * scratch and records the small-job launch as a CUDA graph on the context's
 * stream.  The plan can be run many times; the jobs' buffers must stay valid
 * until lw_batch_destroy.  Nothing runs yet.
 */
lw_status lw_batch_create(lw_ctx *ctx, const lw_job *jobs, int32_t njobs, lw_batch **out);

/* lw_batch_run -- queue one run of the plan on the context's stream (graph
 * replay, then the large jobs); returns without waiting. */
lw_status lw_batch_run(lw_batch *batch);

/* lw_batch_wait -- wait for the last run; writes each job's status into
 * jobs[q].status when jobs is not NULL (same order as at creation) and
 * returns LW_OK if every job succeeded, else the first failing status. */
lw_status lw_batch_wait(lw_batch *batch, lw_job *jobs);

/* lw_batch_destroy -- free the plan (NULL is a no-op). */
void lw_batch_destroy(lw_batch *batch);

/*
 * lw_set_batch_classes -- how one-CTA batch jobs are grouped: class q takes
 * the jobs with n_hi[q-1] < n <= n_hi[q] (n_hi ascending, count <= 16) and
 * runs them with CTAs of cta_threads[q] threads (128, 256 or 512: smaller
 * CTAs let several jobs share an SM).  Each class is its own persistent
 * launch; the classes run side by side as branches of the batch's CUDA
 * graph.  count = 0 restores the default (one class of 512-thread CTAs).
 * The autotuner of the Python package measures and sets this table.
 */
lw_status lw_set_batch_classes(lw_ctx *ctx, const int64_t *n_hi, const int32_t *cta_threads,
                               int32_t count);

/* lw_cluster_batch -- create, run, wait and destroy in one blocking call. */
lw_status lw_cluster_batch(lw_ctx *ctx, lw_job *jobs, int32_t njobs);

/*
 * Serving: a request loop with continuous batching.
 *
 * A server owns a device memory pool of `budget_bytes` and `lanes` execution
 * lanes (a CUDA stream and a context each) on `device`.  Submitted requests
 * queue on the host; a scheduler thread admits one as soon as a lane is free
 * and the pool can hold its packed matrix (n(n-1)/2 * 4 bytes, rounded up to
 * 256): the matrix is copied into the pool, clustered on the lane's stream,
 * and the results copied to the caller's buffers.  Lanes run side by side,
 * so requests that arrive while others are on the GPU start as soon as a
 * lane and memory free up; a request that does not fit the pool yet is
 * passed over by smaller ones behind it.  Every result is bit-identical to
 * lw_cluster on the same input.  All server calls are thread-safe.
 */
typedef struct lw_server lw_server;

typedef struct lw_server_stats {
    int64_t submitted, completed, failed;
    int64_t peak_bytes;    /* largest sum of footprints admitted at once */
    int64_t budget_bytes;  /* the pool size */
    int32_t peak_inflight; /* most requests admitted at once */
    int32_t cancelled;     /* requests cancelled while queued */
    double p50_ms, p99_ms, mean_ms; /* latency, submission to completion */
    double wall_s;         /* first submission to last completion */
} lw_server_stats;

/* lw_server_create -- allocate the pool (one cudaMalloc of budget_bytes),
 * the lanes (1..256) and start the scheduler.  LW_ERR_OOM if the pool does
 * not fit, LW_ERR_INVALID_ARG for a bad device, budget or lane count. */
lw_status lw_server_create(int device, int64_t budget_bytes, int32_t lanes, lw_server **out);

/* lw_server_submit -- queue one request and return its ticket.  dist (host
 * or device, read-only, pinned host memory for an asynchronous copy),
 * merges_out and heights_out (host or device) must stay valid until the
 * request completes.  LW_ERR_INVALID_ARG for bad arguments or a matrix
 * larger than the whole pool. */
lw_status lw_server_submit(lw_server *srv, const float *dist, int64_t n, int linkage,
                           int32_t *merges_out, float *heights_out, uint64_t *ticket);

/* lw_server_poll -- *done = 1 once the request finished; then *status is its
 * lw_status and *latency_ms the time from submission to completion. */
lw_status lw_server_poll(lw_server *srv, uint64_t ticket, int32_t *done, lw_status *status,
                         double *latency_ms);

/* lw_server_cancel -- withdraw a request that is still queued: it never
 * runs, and lw_server_poll reports it done with LW_ERR_CANCELLED.  Returns
 * LW_ERR_BUSY if the request was admitted already (it runs to the end) and
 * LW_ERR_INVALID_ARG for an unknown ticket.  (Not a step of the paper: a
 * service of the request loop.) */
lw_status lw_server_cancel(lw_server *srv, uint64_t ticket);

/* lw_server_drain -- block until every submitted request finished; returns
 * LW_OK if all succeeded (cancelled requests do not count as failures). */
lw_status lw_server_drain(lw_server *srv);

/* lw_server_get_stats -- counters, latency percentiles and wall time. */
lw_status lw_server_get_stats(lw_server *srv, lw_server_stats *stats);

/* lw_server_destroy -- finish the queued work, stop the scheduler, free
 * everything (NULL is a no-op). */
void lw_server_destroy(lw_server *srv);

/* lw_status_string -- static text for a status code. */
const char *lw_status_string(lw_status s);

/* lw_last_error -- detail text of the last failure on this context. */
const char *lw_last_error(lw_ctx *ctx);

/* lw_destroy -- free the context and its device workspace (NULL is a no-op). */
void lw_destroy(lw_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* LW_H */
