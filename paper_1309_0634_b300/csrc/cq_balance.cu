/*
 * cq_balance.cu -- the owner-computes mode's lay-out and rebalancing on the
 * device (cqo_create with CQO_ON_DEVICE): the host steps of Section 3.1 (the
 * two-pass reorder and the threadDataIndicator) and the Section 4 policies
 * getFirst, checkAll, probCheck and bestBalance, moved onto the GPU so that no
 * batch passes through a host lay-out and no host loop follows a batch.
 *
 * Per batch, on the query's stream:
 *   map        each tuple's owner thread, own[g], and each group's count;
 *   sort       the tuples stably by owner (the radix sort of cq_sort.cu):
 *              the threads' segments, stream order within each -- the
 *              reordered batch of Section 3.1;
 *   indicator  each thread's first tuple, by binary search of the owners;
 *   gather     the values in that order, for the owner kernel;
 * then, on a second stream while the owner kernel runs:
 *   ranks      (checkAll, probCheck, bestBalance) the tuples stably by
 *              group: each tuple's rank among its group's tuples;
 *   policy     one CTA of 1024 threads runs the policy's loop;
 * the next batch's map waits for the policy (the paper's delay of one batch).
 *
 * The policy CTA keeps tpt in shared memory under a three-level tree of
 * 32-way arg-max and arg-min nodes (one redux.sync per level): the paper's
 * two heaps, updated in O(log32 T) after a move.  The mapping stays on the
 * device as doubly linked group lists, their heads in shared memory during
 * the loop.
 *   getFirst      warp 0 alone, with no block barrier.
 *   probCheck     every group's tuples lie in the laid-out segment of the
 *                 thread that owned it at lay-out, in stream order, and a
 *                 group moves as a whole; so the tuple at which the running
 *                 count of g first reaches the limit is g's tuple of rank
 *                 L - 1, with L = ceil(pot tpt[tmax] / ngroups) (a count c
 *                 satisfies c >= limit exactly when c >= L).  One pass over
 *                 tmax's segment takes the first such tuple whose group tmax
 *                 still owns.
 *   checkAll,     likewise a group's first occurrence is its rank-0 tuple and
 *   bestBalance   its count in the segment is its count in the batch: one
 *                 pass reduces (score, position) to the best.
 * The readings (ties, move order, stopping) are those of the host policies.
 * shift and shiftLocal are not offered: each of their steps is a chain of
 * neighbour moves that depend one on the other.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>
#include <vector>

#include "cq_balance.h"

namespace cq {
namespace {

constexpr int kMapT = 256;
constexpr int kBT = 1024;                      /* the policy CTA */
constexpr int kN1 = kBalMaxThreads / 32;       /* tree level 1: nodes of 32 threads */
constexpr int kN2 = kN1 / 32;                  /* level 2: nodes of 1024 threads; the root covers these */
constexpr unsigned kAll = 0xFFFFFFFFu;
static_assert(kN2 <= 32, "the root is one warp's reduction");

int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }

/* Owner of every tuple, its position and group (the by-owner sort's input);
 * the by-group sort's input when bk is set; each group's count in the batch. */
__global__ void __launch_bounds__(kMapT) map_kernel(const int32_t *keys, int64_t n, const int32_t *own, uint32_t *ak,
                                                     uint32_t *ap, int32_t *av, uint32_t *bk, uint32_t *bp,
                                                     int32_t *bv, int32_t *count) {
    const int64_t i = (int64_t)blockIdx.x * kMapT + threadIdx.x;
    const bool live = i < n;
    const unsigned m = __ballot_sync(kAll, live);
    if (!live) return;
    const int32_t g = keys[i];
    ak[i] = (uint32_t)own[g];
    ap[i] = (uint32_t)i;
    av[i] = g;
    if (bk) {
        bk[i] = (uint32_t)g;
        bp[i] = (uint32_t)i;
        bv[i] = 0;
    }
    const unsigned peers = __match_any_sync(m, g);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(count + g, __popc(peers));
}

/* ind[t] = the first laid-out tuple of thread t (the lower bound of t in the
 * sorted owners), ind[T] = n. */
__global__ void indicator_kernel(const uint32_t *owner, int64_t n, int T, uint32_t *ind) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > T) return;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)owner[mid] < t) lo = mid + 1;
        else hi = mid;
    }
    ind[t] = (uint32_t)lo;
}

/* The values in laid-out order, for the owner threads' serial loops. */
__global__ void gather_values_kernel(const uint32_t *pos, const int32_t *vals, int64_t n, int32_t *rv) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) rv[j] = vals[pos[j]];
}

/* In the by-group order: where each group's run starts ... */
__global__ void run_start_kernel(const uint32_t *key, int64_t n, uint32_t *gstart) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t g = key[j];
    if (j == 0 || key[j - 1] != g) gstart[g] = (uint32_t)j;
}

/* ... and each tuple's rank in its run, stored by stream position. */
__global__ void rank_kernel(const uint32_t *key, const uint32_t *pos, int64_t n, const uint32_t *gstart,
                            uint32_t *rank) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    rank[pos[j]] = (uint32_t)j - gstart[key[j]];
}

/* ---- the policy CTA ---- */

struct Lists {
    int32_t *own, *nxt, *prv, *tail, *len;
};

struct BalArgs {
    const uint32_t *seg_group;   /* laid-out tuples: their groups */
    const uint32_t *seg_pos;     /* ... and stream positions */
    const uint32_t *ind;
    const uint32_t *rank;        /* by stream position (rank policies) */
    const int32_t *count;
    int32_t *head;               /* global copy of the list heads */
    Lists L;
    int T;
    int64_t G;
    int policy;
    long long threshold;
    double pot;
    BalStats *st;
};

struct Arg {
    int mx, mn;
};

/* The lowest index of the largest and of the smallest value over a warp
 * (lanes out of range pass INT_MIN / INT_MAX values and index INT_MAX). */
__device__ __forceinline__ Arg warp_arg(int vmax, int vmin, int imax, int imin) {
    const int a = __reduce_max_sync(kAll, vmax);
    const int b = __reduce_min_sync(kAll, vmin);
    Arg r;
    r.mx = __reduce_min_sync(kAll, vmax == a ? imax : INT_MAX);
    r.mn = __reduce_min_sync(kAll, vmin == b ? imin : INT_MAX);
    return r;
}

struct Tree {
    int *mx1, *mn1, *mx2, *mn2;
    int n1, n2;
};

/* level 1 node a: the arg-max / arg-min of threads [32a, 32a + 32) */
__device__ __forceinline__ void tree_level1(const Tree &tr, const int *tpt, int T, int a, int lane) {
    const int t = (a << 5) + lane;
    const bool ok = t < T;
    const int v = ok ? tpt[t] : 0;
    const Arg r = warp_arg(ok ? v : INT_MIN, ok ? v : INT_MAX, ok ? t : INT_MAX, ok ? t : INT_MAX);
    if (lane == 0) {
        tr.mx1[a] = r.mx;
        tr.mn1[a] = r.mn;
    }
}

/* level 2 node b: over level-1 nodes [32b, 32b + 32) */
__device__ __forceinline__ void tree_level2(const Tree &tr, const int *tpt, int b, int lane) {
    const int c = (b << 5) + lane;
    const bool ok = c < tr.n1;
    const int i = ok ? tr.mx1[c] : INT_MAX, j = ok ? tr.mn1[c] : INT_MAX;
    const Arg r = warp_arg(ok ? tpt[i] : INT_MIN, ok ? tpt[j] : INT_MAX, i, j);
    if (lane == 0) {
        tr.mx2[b] = r.mx;
        tr.mn2[b] = r.mn;
    }
}

__device__ __forceinline__ Arg tree_root(const Tree &tr, const int *tpt, int lane) {
    const bool ok = lane < tr.n2;
    const int i = ok ? tr.mx2[lane] : INT_MAX, j = ok ? tr.mn2[lane] : INT_MAX;
    return warp_arg(ok ? tpt[i] : INT_MIN, ok ? tpt[j] : INT_MAX, i, j);
}

/* Re-reduce the nodes over threads ta and tb after both changed: the two
 * paths' reductions are independent, so they overlap. */
__device__ __forceinline__ void tree_fix2(const Tree &tr, const int *tpt, int T, int ta, int tb, int lane) {
    {
        const int na = ta >> 5, nb = tb >> 5;
        const int t1 = (na << 5) + lane, t2 = (nb << 5) + lane;
        const bool ok1 = t1 < T, ok2 = t2 < T;
        const int v1 = ok1 ? tpt[t1] : 0, v2 = ok2 ? tpt[t2] : 0;
        const Arg r1 = warp_arg(ok1 ? v1 : INT_MIN, ok1 ? v1 : INT_MAX, ok1 ? t1 : INT_MAX, ok1 ? t1 : INT_MAX);
        const Arg r2 = warp_arg(ok2 ? v2 : INT_MIN, ok2 ? v2 : INT_MAX, ok2 ? t2 : INT_MAX, ok2 ? t2 : INT_MAX);
        if (lane == 0) {
            tr.mx1[na] = r1.mx;
            tr.mn1[na] = r1.mn;
            tr.mx1[nb] = r2.mx;
            tr.mn1[nb] = r2.mn;
        }
    }
    __syncwarp();
    {
        const int na = ta >> 10, nb = tb >> 10;
        const int c1 = (na << 5) + lane, c2 = (nb << 5) + lane;
        const bool ok1 = c1 < tr.n1, ok2 = c2 < tr.n1;
        const int i1 = ok1 ? tr.mx1[c1] : INT_MAX, j1 = ok1 ? tr.mn1[c1] : INT_MAX;
        const int i2 = ok2 ? tr.mx1[c2] : INT_MAX, j2 = ok2 ? tr.mn1[c2] : INT_MAX;
        const Arg r1 = warp_arg(ok1 ? tpt[i1] : INT_MIN, ok1 ? tpt[j1] : INT_MAX, i1, j1);
        const Arg r2 = warp_arg(ok2 ? tpt[i2] : INT_MIN, ok2 ? tpt[j2] : INT_MAX, i2, j2);
        if (lane == 0) {
            tr.mx2[na] = r1.mx;
            tr.mn2[na] = r1.mn;
            tr.mx2[nb] = r2.mx;
            tr.mn2[nb] = r2.mn;
        }
    }
    __syncwarp();
}

/* Move group g from src's list to the end of dst's (one thread).  The four
 * reads go out together: the stores below touch neither tail[dst] (src !=
 * dst) nor g's own links before they are read. */
__device__ void move_group(const BalArgs &a, int *head, int *tpt, int g, int src, int dst) {
    const Lists &L = a.L;
    const int p = L.prv[g], q = L.nxt[g], t = L.tail[dst];
    const int c = __ldg(a.count + g);
    if (p >= 0) L.nxt[p] = q;
    else head[src] = q;
    if (q >= 0) L.prv[q] = p;
    else L.tail[src] = p;
    L.prv[g] = t;
    L.nxt[g] = -1;
    if (t >= 0) L.nxt[t] = g;
    else head[dst] = g;
    L.tail[dst] = g;
    L.own[g] = dst;
    L.len[src]--;
    L.len[dst]++;
    tpt[src] -= c;
    tpt[dst] += c;
}

/* One move by warp 0 and the tree repaired; returns the new (tmax, tmin). */
__device__ __forceinline__ Arg warp_move(const BalArgs &a, const Tree &tr, int *head, int *tpt, int g, int hi,
                                         int lo, int lane) {
    if (lane == 0) move_group(a, head, tpt, g, hi, lo);
    __syncwarp();
    tree_fix2(tr, tpt, a.T, hi, lo, lane);
    return tree_root(tr, tpt, lane);
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(kAll, x, o);
        x = y < x ? y : x;
    }
    return x;
}

__global__ void __launch_bounds__(kBT, 1) balance_kernel(BalArgs a) {
    extern __shared__ int smem[];
    int *tpt = smem;          /* T */
    int *head = smem + a.T;   /* T */
    __shared__ int s_mx1[kN1], s_mn1[kN1], s_mx2[32], s_mn2[32];
    __shared__ int s_hi, s_lo;
    __shared__ long long s_want;
    __shared__ unsigned long long s_best;
    __shared__ long long s_moves;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = a.T;
    Tree tr{s_mx1, s_mn1, s_mx2, s_mn2, (T + 31) >> 5, 0};
    tr.n2 = (tr.n1 + 31) >> 5;

    for (int t = tid; t < T; t += kBT) {
        tpt[t] = (int)(a.ind[t + 1] - a.ind[t]);
        head[t] = a.head[t];
    }
    if (tid == 0) {
        s_best = ~0ull;
        s_moves = 0;
    }
    __syncthreads();
    for (int n = warp; n < tr.n1; n += kBT / 32) tree_level1(tr, tpt, T, n, lane);
    __syncthreads();
    for (int n = warp; n < tr.n2; n += kBT / 32) tree_level2(tr, tpt, n, lane);
    __syncthreads();
    if (warp == 0) {
        const Arg r = tree_root(tr, tpt, lane);
        if (lane == 0) {
            s_hi = r.mx;
            s_lo = r.mn;
            a.st->last_max = tpt[r.mx];
            a.st->last_min = tpt[r.mn];
        }
    }
    __syncthreads();

    const long long thr = a.threshold;
    if (a.policy == CQO_GET_FIRST) {
        if (warp == 0) {   /* the whole loop in one warp: O(1) list work and the tree per move */
            int hi = s_hi, lo = s_lo;
            long long moves = 0;
            while ((long long)tpt[hi] - tpt[lo] > thr && moves < a.G) {
                const int g = head[hi];
                if (g < 0) break;
                const Arg r = warp_move(a, tr, head, tpt, g, hi, lo, lane);
                hi = r.mx;
                lo = r.mn;
                moves++;
            }
            if (lane == 0) s_moves = moves;
        }
    } else if (a.policy == CQO_CHECK_ALL || a.policy == CQO_PROB_CHECK || a.policy == CQO_BEST_BALANCE) {
        long long moves = 0;
        for (;;) {
            const int hi = s_hi, lo = s_lo;
            if (!((long long)tpt[hi] - tpt[lo] > thr && moves < a.G)) break;
            if (tid == 0) {
                long long want = 0;   /* the rank whose tuples are candidates; -1: none */
                if (a.policy == CQO_PROB_CHECK) {
                    const int ngroups = a.L.len[hi];
                    if (ngroups <= 0) {
                        want = -1;
                    } else {
                        const double limit = a.pot * (double)tpt[hi] / (double)ngroups;
                        const double L = ceil(limit);
                        want = L > 4294967296.0 ? -1 : (long long)L - 1;
                    }
                }
                s_want = want;
            }
            __syncthreads();
            const long long want = s_want;
            if (want < 0) break;
            const uint32_t s0 = a.ind[hi], e0 = a.ind[hi + 1];
            const long long th = tpt[hi], tl = tpt[lo];
            unsigned long long best = ~0ull;
            for (uint32_t j = s0 + tid; j < e0; j += kBT) {
                if ((long long)a.rank[a.seg_pos[j]] != want) continue;
                const int g = (int)a.seg_group[j];
                if (a.L.own[g] != hi) continue;
                unsigned long long key = j;   /* probCheck: the first position */
                if (a.policy == CQO_CHECK_ALL) {
                    key |= (unsigned long long)(uint32_t)(INT_MAX - __ldg(a.count + g)) << 32;
                } else if (a.policy == CQO_BEST_BALANCE) {
                    const long long c = __ldg(a.count + g);
                    long long gap = (th - c) - (tl + c);
                    gap = gap < 0 ? -gap : gap;
                    key |= (unsigned long long)gap << 32;
                }
                best = key < best ? key : best;
            }
            best = warp_min_u64(best);
            if (lane == 0 && best != ~0ull) atomicMin(&s_best, best);
            __syncthreads();
            const unsigned long long chosen = s_best;
            __syncthreads();   /* everyone has read s_best */
            if (chosen == ~0ull) break;
            if (warp == 0) {
                const int g = (int)a.seg_group[(uint32_t)chosen];
                if (lane == 0) s_best = ~0ull;
                const Arg r = warp_move(a, tr, head, tpt, g, hi, lo, lane);
                if (lane == 0) {
                    s_hi = r.mx;
                    s_lo = r.mn;
                }
            }
            moves++;
            __syncthreads();
        }
        if (tid == 0) s_moves = moves;
    }
    __syncthreads();
    const long long moves = s_moves;
    if (moves > 0)
        for (int t = tid; t < T; t += kBT) a.head[t] = head[t];
    if (tid == 0) {
        a.st->moves += moves;
        a.st->last_moves = moves;
    }
}

}  // namespace

cudaError_t owner_dev_alloc(OwnerDev &d, int64_t G, int T, const int32_t *h_off, const int32_t *h_order,
                            cudaStream_t s) {
    d.G = G;
    d.T = T;
    std::vector<int32_t> own(G), nxt(G), prv(G), head(T), tail(T), len(T);
    for (int t = 0; t < T; t++) {
        const int32_t a = h_off[t], b = h_off[t + 1];
        head[t] = a < b ? h_order[a] : -1;
        tail[t] = a < b ? h_order[b - 1] : -1;
        len[t] = b - a;
        for (int32_t j = a; j < b; j++) {
            const int32_t g = h_order[j];
            own[g] = t;
            prv[g] = j > a ? h_order[j - 1] : -1;
            nxt[g] = j + 1 < b ? h_order[j + 1] : -1;
        }
    }
    cudaError_t e = cudaSuccess;
    int32_t **gbufs[] = {&d.own, &d.nxt, &d.prv, &d.count};
    for (int32_t **p : gbufs)
        if (e == cudaSuccess) e = cudaMalloc(p, sizeof(int32_t) * G);
    int32_t **tbufs[] = {&d.head, &d.tail, &d.len};
    for (int32_t **p : tbufs)
        if (e == cudaSuccess) e = cudaMalloc(p, sizeof(int32_t) * T);
    for (LaySet &ls : d.set)
        if (e == cudaSuccess) e = cudaMalloc(&ls.ind, sizeof(uint32_t) * (T + 1));
    if (e == cudaSuccess) e = cudaMalloc(&d.gstart, sizeof(uint32_t) * G);
    if (e == cudaSuccess) e = cudaMalloc(&d.st, sizeof(BalStats));
    if (e == cudaSuccess) e = cudaMalloc(&d.err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.own, own.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.nxt, nxt.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.prv, prv.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.head, head.data(), sizeof(int32_t) * T, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.tail, tail.data(), sizeof(int32_t) * T, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.len, len.data(), sizeof(int32_t) * T, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.count, 0, sizeof(int32_t) * G, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.st, 0, sizeof(BalStats), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   /* the host vectors go out of scope */
    if (e == cudaSuccess) {
        e = raise_dyn_smem((const void *)balance_kernel, (int)(2 * sizeof(int) * kBalMaxThreads));
    }
    return e;
}

cudaError_t owner_dev_reserve(OwnerDev &d, int64_t n, cudaStream_t s) {
    if (n <= d.cap) return cudaSuccess;
    int64_t cap = 1 << 16;
    while (cap < n) cap *= 2;
    for (LaySet &ls : d.set) {
        sort_free(ls.by_owner);
        cudaFree(ls.rv);
        ls.rv = nullptr;
    }
    sort_free(d.by_group);
    cudaFree(d.rank);
    d.rank = nullptr;
    d.cap = 0;
    cudaError_t e = cudaSuccess;
    for (LaySet &ls : d.set) {
        if (e == cudaSuccess) e = sort_alloc(ls.by_owner, cap, d.T, s);
        if (e == cudaSuccess) e = cudaMalloc(&ls.rv, sizeof(int32_t) * cap);
    }
    if (e == cudaSuccess) e = sort_alloc(d.by_group, cap, d.G, s);
    if (e == cudaSuccess) e = cudaMalloc(&d.rank, sizeof(uint32_t) * cap);
    if (e == cudaSuccess) d.cap = cap;
    return e;
}

void owner_dev_free(OwnerDev &d) {
    for (LaySet &ls : d.set) {
        sort_free(ls.by_owner);
        cudaFree(ls.ind);
        cudaFree(ls.rv);
    }
    sort_free(d.by_group);
    int32_t *i32[] = {d.own, d.nxt, d.prv, d.head, d.tail, d.len, d.count};
    for (int32_t *p : i32) cudaFree(p);
    cudaFree(d.gstart);
    cudaFree(d.rank);
    cudaFree(d.st);
    cudaFree(d.err);
    d = OwnerDev{};
}

int owner_dev_lay_out(OwnerDev &d, int si, const int32_t *d_keys, const int32_t *d_vals, int64_t n, bool ranks,
                      cudaEvent_t after_map, cudaStream_t s, int64_t *launches) {
    if (n <= 0 || n > d.cap) return -1;
    LaySet &ls = d.set[si];
    if (cudaMemsetAsync(d.count, 0, sizeof(int32_t) * d.G, s) != cudaSuccess) return -1;
    if (sort_maintain(ls.by_owner, s) != cudaSuccess) return -1;
    const unsigned nb = (unsigned)ceil_div64(n, kMapT);
    SortBuffers &b = ls.by_owner;
    map_kernel<<<nb, kMapT, 0, s>>>(d_keys, n, d.own, b.k[0], b.p[0], b.v[0], ranks ? d.by_group.k[0] : nullptr,
                                    d.by_group.p[0], d.by_group.v[0], d.count);
    if (after_map && cudaEventRecord(after_map, s) != cudaSuccess) return -1;
    const int idx = stable_sort_by_key(b, n, d.T, nullptr, s, d.err, launches);
    if (idx < 0) return -1;
    indicator_kernel<<<(unsigned)ceil_div64(d.T + 1, 256), 256, 0, s>>>(b.k[idx], n, d.T, ls.ind);
    gather_values_kernel<<<nb, kMapT, 0, s>>>(b.p[idx], d_vals, n, ls.rv);
    if (launches) *launches += 3;
    return cudaGetLastError() == cudaSuccess ? idx : -1;
}

cudaError_t owner_dev_ranks(OwnerDev &d, int64_t n, cudaStream_t s, int64_t *launches) {
    const unsigned nb = (unsigned)ceil_div64(n, kMapT);
    cudaError_t e = sort_maintain(d.by_group, s);
    if (e != cudaSuccess) return e;
    const int gi = stable_sort_by_key(d.by_group, n, d.G, nullptr, s, d.err, launches);
    if (gi < 0) return cudaErrorInvalidConfiguration;
    run_start_kernel<<<nb, kMapT, 0, s>>>(d.by_group.k[gi], n, d.gstart);
    rank_kernel<<<nb, kMapT, 0, s>>>(d.by_group.k[gi], d.by_group.p[gi], n, d.gstart, d.rank);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

cudaError_t owner_dev_balance(OwnerDev &d, int si, int idx, int policy, int64_t threshold, double pot,
                              cudaStream_t s) {
    BalArgs a;
    const LaySet &ls = d.set[si];
    a.seg_group = (const uint32_t *)ls.by_owner.v[idx];
    a.seg_pos = ls.by_owner.p[idx];
    a.ind = ls.ind;
    a.rank = d.rank;
    a.count = d.count;
    a.head = d.head;
    a.L = Lists{d.own, d.nxt, d.prv, d.tail, d.len};
    a.T = d.T;
    a.G = d.G;
    a.policy = policy;
    a.threshold = threshold;
    a.pot = pot;
    a.st = d.st;
    balance_kernel<<<1, kBT, 2 * sizeof(int) * d.T, s>>>(a);
    return cudaGetLastError();
}

cudaError_t owner_dev_mapping(const OwnerDev &d, int32_t *off, int32_t *groups) {
    std::vector<int32_t> head(d.T), nxt(d.G);
    cudaError_t e = cudaMemcpy(head.data(), d.head, sizeof(int32_t) * d.T, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(nxt.data(), d.nxt, sizeof(int32_t) * d.G, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    int64_t at = 0;
    for (int t = 0; t < d.T; t++) {
        off[t] = (int32_t)at;
        for (int32_t g = head[t]; g >= 0; g = nxt[g]) {
            if (at >= d.G || g >= d.G) return cudaErrorUnknown;   /* a broken list */
            groups[at++] = g;
        }
    }
    off[d.T] = (int32_t)at;
    return at == d.G ? cudaSuccess : cudaErrorUnknown;
}

}  // namespace cq
