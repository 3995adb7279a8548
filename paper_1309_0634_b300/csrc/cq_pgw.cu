/*
 * cq_pgw.cu -- the paper's own aggregate: one count-based window of w values
 * per group, whose SUM is recomputed from scratch after every tuple
 * (Sections 3.2 and 5.1), as the cqw_* calls of cq.h.
 *
 * The paper's GPU kernel walks each group's tuples in order on the thread
 * that owns the group, so a hot group serialises on one thread and its
 * skew handling (Section 4) moves groups between threads.  Here the order
 * dependence is removed instead: after a stable sort of the batch by group,
 * the window of a group's r-th new tuple is known without walking the
 * earlier ones -- it is the newest min(w, fill + r + 1) values of
 * (the group's old window ++ its first r + 1 new values).  So every tuple is
 * one independent thread that scans its own window slice, and a hot group is
 * spread over as many threads as it has tuples.
 *
 * Per push of n tuples:
 *   1. load: validate keys, copy (key, position, value);
 *   2. stable radix sort of (key, position, value) by key (shared with the
 *      MIN/MAX flip);
 *   3. runs: the run of group k in the sorted batch is [start[k], stop[k]),
 *      written at the run's two ends (groups without tuples are not read);
 *   4. sums: the window SUM after each tuple, scanning the slice `passes`
 *      times, written at the tuple's position of the output array;
 *   5. ring: the newest w values of each group's run overwrite its oldest
 *      cells; 6. pointers: nextPos and fill of each group advance.
 * A key outside [0, G) makes every later step a no-op and poisons the query.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include <new>

#include "cq.h"
#include "cq_internal.h"

static_assert(CQW_MAX_WINDOW <= 2147483647LL - 64, "the window sum's 32-bit ring index needs w + kSumLanes <= INT32_MAX");

namespace {

constexpr int kThreads = 256;
constexpr int kSlots = 4;   /* pushes whose argument copies may be in flight */

/* A push's batch and output: read by the kernels from device memory, so
 * that a captured graph of the push can be replayed for any batch of the
 * same length. */
struct PgwArgs {
    const int32_t *keys, *vals;
    long long *sums;
    long long pad;
};

__global__ void pgw_load_kernel(const PgwArgs *args, int64_t n, int64_t G, uint32_t *key, uint32_t *pos,
                                int32_t *val, int *err) {
    const int32_t *keys = args->keys, *vals = args->vals;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = keys[i];
        if ((uint32_t)k >= (uint32_t)G) {
            atomicOr(err, 1);
            continue;
        }
        key[i] = (uint32_t)k;
        pos[i] = (uint32_t)i;
        val[i] = vals[i];
    }
}

/* Each group's run in the sorted batch, [start, stop), from its two ends. */
__global__ void pgw_runs_kernel(const uint32_t *key, int64_t n, uint32_t *start, uint32_t *stop, const int *err) {
    if (*(volatile int *)err) return;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t k = key[j];
    if (j == 0 || key[j - 1] != k) start[k] = (uint32_t)j;
    if (j == n - 1 || key[j + 1] != k) stop[k] = (uint32_t)(j + 1);
}

/* Window SUM right after each tuple, from scratch, `passes` times.  Each
 * tuple's window is summed by kSumLanes lanes, each taking every kSumLanes-th
 * value, so that its reads are in flight together; the lanes' partial sums
 * are then added (integers: the order does not change the result). */
constexpr int kSumLanes = 4;

__global__ void pgw_sum_kernel(const uint32_t *key, const uint32_t *pos, const int32_t *val, int64_t n,
                               const uint32_t *start, const int32_t *cells, const int32_t *next, const int32_t *fill,
                               int32_t w, int32_t passes, const PgwArgs *args, const int *err) {
    if (*(volatile int *)err) return;
    long long *out = args->sums;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kSumLanes;
    const int sub = (int)(threadIdx.x % kSumLanes);
    long long sum = 0;
    if (j < n) {   /* no return: every lane joins the shuffles below */
        const uint32_t k = key[j];
        const int64_t r = j - (int64_t)start[k];   /* the tuple's rank among its group's new tuples */
        const int32_t f = fill[k], nx = next[k];
        const int64_t c = min((int64_t)w, (int64_t)f + r + 1);   /* values in the window after the tuple */
        const int64_t c1 = min(c, r + 1);                        /* of them, new values: sorted [j - c1 + 1, j] */
        const int64_t c0 = c - c1;                               /* old values: the newest c0 of the old window */
        const int32_t *win = cells + (int64_t)k * w;
        for (int32_t p = 0; p < passes; p++) {
            /* each pass re-reads the window: the compiler may not reuse a pass */
            asm volatile("" ::: "memory");
            sum = 0;
            /* old values: cell (nx - f + t) mod w, in 32-bit arithmetic: t < f <= w and
               t + kSumLanes stays below w + kSumLanes <= INT32_MAX (static_assert below) */
            for (int32_t t = f - (int32_t)c0 + sub; t < f; t += kSumLanes) {
                int32_t cell = nx - f + t;
                if (cell < 0) cell += w;
                sum += win[cell];
            }
            for (int64_t i = j - c1 + 1 + sub; i <= j; i += kSumLanes) sum += val[i];
        }
    }
#pragma unroll
    for (int o = kSumLanes / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o, kSumLanes);
    if (j < n && sub == 0) out[pos[j]] = sum;
}

/* The newest w values of each group's run go to the ring, the r-th new value
 * of group k to cell (next + r) mod w. */
__global__ void pgw_ring_kernel(const uint32_t *key, const int32_t *val, int64_t n, const uint32_t *start,
                                const uint32_t *stop, int32_t *cells, const int32_t *next, int32_t w,
                                const int *err) {
    if (*(volatile int *)err) return;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t k = key[j];
    const int64_t r = j - (int64_t)start[k], m = (int64_t)stop[k] - (int64_t)start[k];
    if (r < m - w) return;
    cells[(int64_t)k * w + (next[k] + r) % w] = val[j];
}

/* nextPos and fill of every group with new tuples (one thread per run). */
__global__ void pgw_ptr_kernel(const uint32_t *key, int64_t n, const uint32_t *start, const uint32_t *stop,
                               int32_t *next, int32_t *fill, int32_t w, const int *err) {
    if (*(volatile int *)err) return;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t k = key[j];
    if (j + 1 != (int64_t)stop[k]) return;   /* the run's last tuple */
    const int64_t m = (int64_t)stop[k] - (int64_t)start[k];
    next[k] = (int32_t)((next[k] + m) % w);
    fill[k] = (int32_t)min((int64_t)w, (int64_t)fill[k] + m);
}

int64_t div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

struct cqw_query {
    int64_t G = 0;
    int32_t w = 0, passes = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int32_t *cells = nullptr, *next = nullptr, *fill = nullptr;
    uint32_t *start = nullptr, *stop = nullptr;   /* each group's run in the sorted batch */
    int *err = nullptr, *h_err = nullptr;
    PgwArgs *h_args = nullptr, *d_args = nullptr;   /* kSlots argument blocks */
    cudaEvent_t ev[kSlots] = {};
    cudaGraphExec_t graph[kSlots] = {};
    int64_t graph_n = -1;                            /* batch length the graphs were captured for */
    bool graphs_off = false;
    int slot = 0;
    cq::SortBuffers sort{};
    int64_t sort_cap = 0;   /* tuples the sort buffers hold */
    int64_t seen = 0, pushes = 0, launches = 0, per_push_launches = 0;
    cq_status poison = CQ_OK;
    bool poison_reported = false;
};

namespace {

void free_sort(cqw_query *q) {
    cq::sort_free(q->sort);
    q->sort_cap = 0;
}

void drop_graphs(cqw_query *q) {
    for (int i = 0; i < kSlots; i++)
        if (q->graph[i]) {
            cudaGraphExecDestroy(q->graph[i]);
            q->graph[i] = nullptr;
        }
    q->graph_n = -1;
}

void free_query(cqw_query *q) {
    drop_graphs(q);
    for (int i = 0; i < kSlots; i++)
        if (q->ev[i]) cudaEventDestroy(q->ev[i]);
    if (q->h_args) cudaFreeHost(q->h_args);
    cudaFree(q->d_args);
    cudaFree(q->cells);
    cudaFree(q->next);
    cudaFree(q->fill);
    cudaFree(q->start);
    cudaFree(q->stop);
    cudaFree(q->err);
    if (q->h_err) cudaFreeHost(q->h_err);
    free_sort(q);
    if (q->own_stream && q->stream) cudaStreamDestroy(q->stream);
}

cudaError_t ensure_sort(cqw_query *q, int64_t n) {
    if (q->sort_cap >= n) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(q->stream);
    if (e != cudaSuccess) return e;
    drop_graphs(q);   /* they name the old buffers */
    free_sort(q);
    int64_t cap = 1 << 16;
    while (cap < n) cap *= 2;
    e = cq::sort_alloc(q->sort, cap, q->G, q->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_sort(q);
        return e;
    }
    q->sort_cap = cap;
    return cudaSuccess;
}

cq_status status_of(cudaError_t e) {
    return e == cudaSuccess ? CQ_OK : (e == cudaErrorMemoryAllocation ? CQ_ENOMEM : CQ_ECUDA);
}

cq_status poison_status(cqw_query *q) {
    if (!q->poison && *(volatile int *)q->h_err) q->poison = CQ_EKEY;
    if (!q->poison) return CQ_OK;
    if (!q->poison_reported) {
        q->poison_reported = true;
        return q->poison;
    }
    return CQ_EPOISONED;
}

/* The work of one push of n tuples whose arguments are in block `sl`. */
cudaError_t enqueue_push(cqw_query *q, int64_t n, int sl) {
    cudaStream_t s = q->stream;
    int64_t launches = 0;
    cudaError_t e = cudaMemcpyAsync(q->d_args + sl, q->h_args + sl, sizeof(PgwArgs), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    const int grid = (int)(div_up(n, kThreads) < 148 * 16 ? div_up(n, kThreads) : 148 * 16);
    pgw_load_kernel<<<grid, kThreads, 0, s>>>(q->d_args + sl, n, q->G, q->sort.k[0], q->sort.p[0], q->sort.v[0],
                                              q->err);
    const int cur = cq::stable_sort_by_key(q->sort, n, q->G, nullptr, s, q->err, &launches);
    if (cur < 0) return cudaErrorInvalidConfiguration;
    const unsigned blocks = (unsigned)div_up(n, kThreads);
    pgw_runs_kernel<<<blocks, kThreads, 0, s>>>(q->sort.k[cur], n, q->start, q->stop, q->err);
    pgw_sum_kernel<<<(unsigned)div_up(n * kSumLanes, kThreads), kThreads, 0, s>>>(
        q->sort.k[cur], q->sort.p[cur], q->sort.v[cur], n, q->start, q->cells, q->next, q->fill, q->w, q->passes,
        q->d_args + sl, q->err);
    pgw_ring_kernel<<<blocks, kThreads, 0, s>>>(q->sort.k[cur], q->sort.v[cur], n, q->start, q->stop, q->cells,
                                                q->next, q->w, q->err);
    pgw_ptr_kernel<<<blocks, kThreads, 0, s>>>(q->sort.k[cur], n, q->start, q->stop, q->next, q->fill, q->w,
                                               q->err);
    /* the error flag goes to the host copy, read by the next call's poison check */
    e = cudaMemcpyAsync(q->h_err, q->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    q->per_push_launches = launches + 5;
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

}  // namespace

extern "C" {

cq_status cqw_create(int64_t groups, int32_t window, int32_t passes, void *cuda_stream, cqw_query **out) {
    if (!out) return CQ_EINVAL;
    *out = nullptr;
    if (groups < 1 || groups > 2147483647LL || window < 1 || window > CQW_MAX_WINDOW || passes < 1 ||
        passes > CQW_MAX_PASSES)
        return CQ_EINVAL;
    cqw_query *q = new (std::nothrow) cqw_query();
    if (!q) return CQ_ENOMEM;
    q->G = groups;
    q->w = window;
    q->passes = passes;
    cudaError_t e = cudaGetDevice(&q->device);
    if (e == cudaSuccess) {
        if (cuda_stream) {
            q->stream = (cudaStream_t)cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking);
            q->own_stream = e == cudaSuccess;
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&q->cells, sizeof(int32_t) * groups * window);
    if (e == cudaSuccess) e = cudaMalloc(&q->next, sizeof(int32_t) * groups);
    if (e == cudaSuccess) e = cudaMalloc(&q->fill, sizeof(int32_t) * groups);
    if (e == cudaSuccess) e = cudaMalloc(&q->start, sizeof(uint32_t) * groups);
    if (e == cudaSuccess) e = cudaMalloc(&q->stop, sizeof(uint32_t) * groups);
    if (e == cudaSuccess) e = cudaMalloc(&q->err, sizeof(int));
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&q->h_err, sizeof(int), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&q->h_args, sizeof(PgwArgs) * kSlots, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&q->d_args, sizeof(PgwArgs) * kSlots);
    for (int i = 0; i < kSlots && e == cudaSuccess; i++) {
        e = cudaEventCreateWithFlags(&q->ev[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(q->ev[i], q->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(q->cells, 0, sizeof(int32_t) * groups * window, q->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(q->next, 0, sizeof(int32_t) * groups, q->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(q->fill, 0, sizeof(int32_t) * groups, q->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(q->err, 0, sizeof(int), q->stream);
    if (e == cudaSuccess) *q->h_err = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_query(q);
        delete q;
        return status_of(e);
    }
    *out = q;
    return CQ_OK;
}

cq_status cqw_push(cqw_query *q, const int32_t *d_keys, const int32_t *d_vals, int64_t n, int64_t *d_sums) {
    if (!q) return CQ_EINVAL;
    cq_status st = poison_status(q);
    if (st != CQ_OK) return st;
    if (n < 0) return CQ_EINVAL;
    if (n == 0) return CQ_OK;
    if (!d_keys || !d_vals || !d_sums || n > 2147483647LL) return CQ_EINVAL;
    cudaSetDevice(q->device);
    cudaError_t e = ensure_sort(q, n);
    if (e == cudaSuccess) e = cq::sort_prepare();
    if (e != cudaSuccess) return status_of(e);
    /* the slot's previous push has copied its arguments: the block is free */
    const int sl = q->slot;
    q->slot = (q->slot + 1) % kSlots;
    e = cudaEventSynchronize(q->ev[sl]);
    if (e != cudaSuccess) return status_of(e);
    q->h_args[sl].keys = d_keys;
    q->h_args[sl].vals = d_vals;
    q->h_args[sl].sums = (long long *)d_sums;
    if (q->graph_n != n) drop_graphs(q);
    e = cq::sort_maintain(q->sort, q->stream);   /* outside any capture */
    if (e != cudaSuccess) return status_of(e);
    if (q->graph[sl]) {
        e = cudaGraphLaunch(q->graph[sl], q->stream);
    } else if (q->graphs_off) {
        e = enqueue_push(q, n, sl);
    } else {
        /* capture the push once per slot and batch length, replay after */
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(q->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t r = enqueue_push(q, n, sl);
            e = cudaStreamEndCapture(q->stream, &g);
            if (r != cudaSuccess) e = r;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&q->graph[sl], g, 0);
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess) {
            q->graph_n = n;
            e = cudaGraphLaunch(q->graph[sl], q->stream);
        } else {   /* capture unavailable (e.g. the legacy stream): launch directly from now on */
            cudaGetLastError();
            q->graph[sl] = nullptr;
            q->graphs_off = true;
            e = enqueue_push(q, n, sl);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(q->ev[sl], q->stream);
    if (e != cudaSuccess) return status_of(e);
    q->launches += q->per_push_launches;
    q->seen += n;
    q->pushes++;
    return CQ_OK;
}

cq_status cqw_sync(cqw_query *q) {
    if (!q) return CQ_EINVAL;
    cudaError_t e = cudaStreamSynchronize(q->stream);
    if (e != cudaSuccess) return status_of(e);
    return poison_status(q);
}

cq_status cqw_stats(const cqw_query *q, int64_t *tuples_seen, int64_t *pushes, int64_t *kernel_launches) {
    if (!q) return CQ_EINVAL;
    if (tuples_seen) *tuples_seen = q->seen;
    if (pushes) *pushes = q->pushes;
    if (kernel_launches) *kernel_launches = q->launches;
    return CQ_OK;
}

void cqw_destroy(cqw_query *q) {
    if (!q) return;
    if (q->stream) cudaStreamSynchronize(q->stream);
    free_query(q);
    delete q;
}

}  /* extern "C" */
