/*
 * cq_owner.cu -- the paper's owner-computes execution of its per-group window
 * workload, with its six rebalancing policies (Sections 3.1, 3.2 and 4), as
 * the cqo_* calls of cq.h: an ablation beside the build's own skew handling
 * (the sort-based cqw_* path and the partitioned kernels).
 *
 * Host (C++), per push of n tuples:
 *   1. the keys are checked against [0, G);
 *   2. the batch is laid out in two passes (Section 3.1): each owner
 *      thread's tuple count (tpt), its start (the threadDataIndicator), then
 *      every tuple after the earlier ones of its thread -- key, value and
 *      stream position, into pinned staging (two buffers, used in turn);
 *   3. one copy to the device and the kernel launch, on the query's stream;
 *   4. while the GPU runs, the policy moves groups between threads on the
 *      host; the new mapping lays out the NEXT batch (a delay of one batch).
 * Device: owner thread t walks its tuples in stream order; for each one it
 * writes the value at its group's nextPos, advances nextPos, and sums the
 * group's whole window `passes` times (Section 5.1's demanding task), the
 * sum being the tuple's output.  A group's tuples all belong to one thread,
 * so the windows need no atomics -- and a heavy group serialises on it,
 * which is what the policies try to spread.
 *
 * The policies follow Section 4; the most and least loaded threads come
 * from an ordered set of (tuples, thread) pairs (the paper's two heaps).
 * Where the algorithms leave a choice open, the readings are those stated in
 * cq.h and kept identical to the test oracle's.
 */
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <climits>
#include <new>
#include <set>
#include <utility>
#include <vector>

#include "cq.h"
#include "cq_balance.h"

namespace {

constexpr int kBlock = 256;   /* the paper's block size */

/* Owner thread t: its tuples [ind[t], ind[t + 1]) of the laid-out batch. */
__global__ void __launch_bounds__(kBlock) owner_kernel(const int32_t *rk, const int32_t *rv, const uint32_t *rpos,
                                                       const uint32_t *ind, int T, int32_t *cells, int32_t *next,
                                                       int32_t *fill, int32_t w, int32_t passes, long long *out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const uint32_t j1 = ind[t + 1];
    for (uint32_t j = ind[t]; j < j1; j++) {
        const int32_t g = rk[j];
        int32_t *win = cells + (int64_t)g * w;
        const int32_t nx = next[g];
        win[nx] = rv[j];
        next[g] = nx + 1 == w ? 0 : nx + 1;
        int32_t f = fill[g];
        if (f < w) fill[g] = ++f;
        /* until the ring wraps the values sit in cells 0 .. f-1, then in all w */
        long long sum = 0;
        for (int32_t p = 0; p < passes; p++) {
            asm volatile("" ::: "memory");   /* every pass re-reads the window */
            sum = 0;
            for (int32_t c = 0; c < f; c++) sum += win[c];
        }
        out[rpos[j]] = sum;
    }
}


/* The thread-to-groups lists and the group-to-thread map. */
struct Mapping {
    std::vector<std::vector<int32_t>> groups;
    std::vector<int32_t> own;

    void init(int T, int64_t G) {
        groups.assign(T, {});
        own.assign(G, 0);
        for (int t = 0; t < T; t++)
            for (int64_t g = (int64_t)t * G / T; g < (int64_t)(t + 1) * G / T; g++) {
                groups[t].push_back((int32_t)g);
                own[g] = t;
            }
    }
};

/* Two-pass lay-out of a batch by the current mapping: tpt, the indicator
 * (T + 1 starts) and the tuples in thread order (keys, values, stream
 * positions); count[g] += g's tuples. */
void lay_out(const Mapping &mp, const int32_t *keys, const int32_t *vals, int64_t n, int32_t *rk, int32_t *rv,
             uint32_t *rpos, uint32_t *ind, std::vector<int64_t> &tpt, int32_t *count) {
    const int T = (int)mp.groups.size();
    tpt.assign(T, 0);
    for (int64_t i = 0; i < n; i++) {
        tpt[mp.own[keys[i]]]++;
        count[keys[i]]++;
    }
    std::vector<int64_t> cur(T);
    ind[0] = 0;
    for (int t = 0; t < T; t++) {
        cur[t] = ind[t];
        ind[t + 1] = (uint32_t)(ind[t] + tpt[t]);
    }
    for (int64_t i = 0; i < n; i++) {
        const int64_t at = cur[mp.own[keys[i]]]++;
        rk[at] = keys[i];
        if (rv) rv[at] = vals[i];
        if (rpos) rpos[at] = (uint32_t)i;
    }
}

/* One policy step (Section 4) after laying out a batch: moves groups for the
 * next batch.  rk / ind: the laid-out keys; count: each group's tuples in the
 * batch; occ: G zeroed words of scratch (left zeroed).  Returns the moves. */
struct Balancer {
    Mapping &mp;
    const int32_t *rk;
    const uint32_t *ind;
    const int32_t *count;
    int32_t *occ;
    std::vector<int64_t> tpt;
    std::set<std::pair<int64_t, int>> load;   /* (tuples, thread): the heaps' role */

    int tmax() const {
        const int64_t top = load.rbegin()->first;
        return load.lower_bound(std::make_pair(top, INT_MIN))->second;   /* ties: the lower index */
    }
    int tmin() const { return load.begin()->second; }

    void move(int32_t g, int src, int dst, bool front) {
        std::vector<int32_t> &s = mp.groups[src];
        for (size_t i = 0; i < s.size(); i++)
            if (s[i] == g) {
                s.erase(s.begin() + (long)i);
                break;
            }
        std::vector<int32_t> &d = mp.groups[dst];
        if (front) d.insert(d.begin(), g);
        else d.push_back(g);
        mp.own[g] = dst;
        load.erase(std::make_pair(tpt[src], src));
        load.erase(std::make_pair(tpt[dst], dst));
        tpt[src] -= count[g];
        tpt[dst] += count[g];
        load.insert(std::make_pair(tpt[src], src));
        load.insert(std::make_pair(tpt[dst], dst));
    }

    /* thread t's tuples of the laid-out batch, of groups it still owns,
       counted in occ; `seen` gets the groups in order of first occurrence */
    void count_segment(int t, std::vector<int32_t> &seen) {
        seen.clear();
        for (uint32_t j = ind[t]; j < ind[t + 1]; j++) {
            const int32_t g = rk[j];
            if (mp.own[g] != t) continue;
            if (occ[g]++ == 0) seen.push_back(g);
        }
    }
    void clear_occ(const std::vector<int32_t> &seen) {
        for (int32_t g : seen) occ[g] = 0;
    }

    int64_t run(int policy, int64_t threshold, double pot) {
        const int T = (int)mp.groups.size();
        const int64_t G = (int64_t)mp.own.size();
        if (policy == CQO_NONE || T < 2) return 0;
        int64_t moves = 0;
        if (policy == CQO_SHIFT_LOCAL) {
            for (int i = 0; i + 1 < T; i++) {
                if (tpt[i] - tpt[i + 1] > threshold && !mp.groups[i].empty()) {
                    move(mp.groups[i].back(), i, i + 1, true);
                    moves++;
                } else if (tpt[i + 1] - tpt[i] > threshold && !mp.groups[i + 1].empty()) {
                    move(mp.groups[i + 1].front(), i + 1, i, false);
                    moves++;
                }
            }
            return moves;
        }
        {   /* a balanced batch needs no ordered set (building one costs ~1 ms at 16K threads) */
            int a = 0, b = 0;
            for (int t = 1; t < T; t++) {
                if (tpt[t] > tpt[a]) a = t;
                if (tpt[t] < tpt[b]) b = t;
            }
            if (tpt[a] - tpt[b] <= threshold) return 0;
        }
        for (int t = 0; t < T; t++) load.insert(std::make_pair(tpt[t], t));
        std::vector<int32_t> seen;
        int hi = tmax(), lo = tmin();
        while (tpt[hi] - tpt[lo] > threshold && moves < G) {
            int64_t moved = 0;
            if (policy == CQO_GET_FIRST) {
                if (!mp.groups[hi].empty()) {
                    move(mp.groups[hi].front(), hi, lo, false);
                    moved = 1;
                }
            } else if (policy == CQO_CHECK_ALL || policy == CQO_BEST_BALANCE) {
                count_segment(hi, seen);
                int32_t chosen = -1;
                int64_t best = 0;
                for (int32_t g : seen) {
                    if (policy == CQO_CHECK_ALL) {
                        if (chosen < 0 || occ[g] > best) {
                            chosen = g;
                            best = occ[g];
                        }
                    } else {
                        int64_t gap = (tpt[hi] - occ[g]) - (tpt[lo] + occ[g]);
                        if (gap < 0) gap = -gap;
                        if (chosen < 0 || gap < best) {
                            chosen = g;
                            best = gap;
                        }
                    }
                }
                clear_occ(seen);
                if (chosen >= 0) {
                    move(chosen, hi, lo, false);
                    moved = 1;
                }
            } else if (policy == CQO_PROB_CHECK) {
                const size_t ngroups = mp.groups[hi].size();
                if (ngroups) {
                    const double limit = pot * (double)tpt[hi] / (double)ngroups;
                    seen.clear();
                    int32_t chosen = -1;
                    for (uint32_t j = ind[hi]; j < ind[hi + 1]; j++) {
                        const int32_t g = rk[j];
                        if (mp.own[g] != hi) continue;
                        if (occ[g]++ == 0) seen.push_back(g);
                        if ((double)occ[g] >= limit) {
                            chosen = g;
                            break;
                        }
                    }
                    clear_occ(seen);
                    if (chosen >= 0) {
                        move(chosen, hi, lo, false);
                        moved = 1;
                    }
                }
            } else if (policy == CQO_SHIFT) {
                /* every thread between the pair passes one group towards lo, at once */
                std::vector<std::pair<int32_t, int>> step;
                if (hi > lo) {
                    for (int i = lo + 1; i <= hi; i++)
                        if (!mp.groups[i].empty()) step.push_back(std::make_pair(mp.groups[i].front(), i));
                    for (auto &s : step) move(s.first, s.second, s.second - 1, false);
                } else {
                    for (int i = hi; i < lo; i++)
                        if (!mp.groups[i].empty()) step.push_back(std::make_pair(mp.groups[i].back(), i));
                    for (auto &s : step) move(s.first, s.second, s.second + 1, true);
                }
                moved = (int64_t)step.size();
            }
            if (moved == 0) break;
            moves += moved;
            hi = tmax();
            lo = tmin();
        }
        return moves;
    }
};

bool valid_policy(int p) { return p >= CQO_NONE && p <= CQO_SHIFT_LOCAL; }

/* the policies the device mode runs (cq_balance.cu) */
bool device_policy(int p) { return p >= CQO_NONE && p <= CQO_BEST_BALANCE; }

/* ... and those of them that read each tuple's rank in its group */
bool needs_ranks(int p) { return p == CQO_CHECK_ALL || p == CQO_PROB_CHECK || p == CQO_BEST_BALANCE; }

cq_status status_of(cudaError_t e) {
    return e == cudaSuccess ? CQ_OK : (e == cudaErrorMemoryAllocation ? CQ_ENOMEM : CQ_ECUDA);
}

}  // namespace

struct cqo_query {
    int64_t G = 0;
    int32_t w = 0, passes = 1, grid = 1, policy = CQO_NONE;
    int T = 0;
    int64_t threshold = 1000;
    double pot = 0.5;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    /* device mode: lay-out and policy on the GPU, the policy on a second stream */
    bool on_device = false;
    cq::OwnerDev dev;
    cudaStream_t lay = nullptr, side = nullptr;
    cudaEvent_t ev_map = nullptr, ev_lay = nullptr, ev_bal = nullptr, ev_own[2] = {nullptr, nullptr};
    int set = 0;
    int32_t *cells = nullptr, *next = nullptr, *fill = nullptr;
    Mapping mp;
    std::vector<int32_t> count, occ;   /* per group: the batch's tuples; scratch of the policies */
    std::vector<int64_t> tpt;
    /* two pinned staging buffers (keys | values | positions | indicator) and their device copies */
    int32_t *h_stage[2] = {nullptr, nullptr};
    int32_t *d_stage[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int64_t cap = 0;
    int slot = 0;
    bool poisoned = false;
    cqo_stats_t st{};
};

namespace {

void free_stage(cqo_query *q) {
    for (int b = 0; b < 2; b++) {
        if (q->h_stage[b]) cudaFreeHost(q->h_stage[b]);
        cudaFree(q->d_stage[b]);
        q->h_stage[b] = q->d_stage[b] = nullptr;
    }
    q->cap = 0;
}

cudaError_t ensure_stage(cqo_query *q, int64_t n) {
    if (n <= q->cap) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(q->stream);
    if (e != cudaSuccess) return e;
    free_stage(q);
    int64_t cap = 1 << 16;
    while (cap < n) cap *= 2;
    const size_t bytes = sizeof(int32_t) * (size_t)(3 * cap + q->T + 1);
    for (int b = 0; b < 2 && e == cudaSuccess; b++) {
        e = cudaHostAlloc((void **)&q->h_stage[b], bytes, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc(&q->d_stage[b], bytes);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_stage(q);
        return e;
    }
    q->cap = cap;
    return cudaSuccess;
}

void free_query(cqo_query *q) {
    free_stage(q);
    for (int b = 0; b < 2; b++)
        if (q->ev[b]) cudaEventDestroy(q->ev[b]);
    if (q->lay) cudaStreamSynchronize(q->lay);
    if (q->side) cudaStreamSynchronize(q->side);
    cq::owner_dev_free(q->dev);
    cudaEvent_t evs[] = {q->ev_map, q->ev_lay, q->ev_bal, q->ev_own[0], q->ev_own[1]};
    for (cudaEvent_t ev : evs)
        if (ev) cudaEventDestroy(ev);
    if (q->lay) cudaStreamDestroy(q->lay);
    if (q->side) cudaStreamDestroy(q->side);
    cudaFree(q->cells);
    cudaFree(q->next);
    cudaFree(q->fill);
    if (q->own_stream && q->stream) cudaStreamDestroy(q->stream);
}

/* Device mode: the batch goes up as it is; lay-out, owner kernel and policy
 * run on the GPU (cq_balance.cu), on three streams:
 *   lay    the copy up, then the lay-out into set[b & 1], once the previous
 *          batch's policy has settled the mapping and the owner kernel of
 *          two batches back has released the set;
 *   query  the owner kernel (the caller's stream: outputs are ordered there);
 *   side   the ranks (after the lay-out's map step) and the policy, beside
 *          the owner kernel. */
cq_status push_device(cqo_query *q, const int32_t *h_keys, const int32_t *h_vals, int64_t n, int64_t *d_sums) {
    cudaError_t e = cudaSuccess;
    if (n > q->cap || n > q->dev.cap) {   /* growing: drain every stream first */
        cudaStream_t all[] = {q->stream, q->lay, q->side};
        for (cudaStream_t st : all)
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = ensure_stage(q, n);
        if (e == cudaSuccess) e = cq::owner_dev_reserve(q->dev, n, q->lay);
        if (e != cudaSuccess) return status_of(e);
    }
    const int sl = q->slot;
    q->slot ^= 1;
    e = cudaEventSynchronize(q->ev[sl]);   /* the slot's previous batch has been laid out */
    if (e != cudaSuccess) return status_of(e);
    const auto t0 = std::chrono::steady_clock::now();
    int32_t *h = q->h_stage[sl], *d = q->d_stage[sl];
    memcpy(h, h_keys, sizeof(int32_t) * n);
    memcpy(h + n, h_vals, sizeof(int32_t) * n);
    const int si = q->set;
    q->set ^= 1;
    e = cudaMemcpyAsync(d, h, sizeof(int32_t) * 2 * n, cudaMemcpyHostToDevice, q->lay);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(q->lay, q->ev_bal, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(q->lay, q->ev_own[si], 0);
    if (e != cudaSuccess) return status_of(e);
    const bool ranks = needs_ranks(q->policy);
    const int idx =
        cq::owner_dev_lay_out(q->dev, si, d, d + n, n, ranks, ranks ? q->ev_map : nullptr, q->lay, nullptr);
    if (idx < 0) return CQ_ECUDA;
    e = cudaEventRecord(q->ev[sl], q->lay);
    if (e == cudaSuccess) e = cudaEventRecord(q->ev_lay, q->lay);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(q->stream, q->ev_lay, 0);
    if (e == cudaSuccess) {
        const cq::LaySet &ls = q->dev.set[si];
        owner_kernel<<<q->grid, kBlock, 0, q->stream>>>(ls.by_owner.v[idx], ls.rv, ls.by_owner.p[idx], ls.ind, q->T,
                                                        q->cells, q->next, q->fill, q->w, q->passes,
                                                        (long long *)d_sums);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(q->ev_own[si], q->stream);
    /* the ranks need only the map step: they sort beside the lay-out's own sort */
    if (e == cudaSuccess && ranks) e = cudaStreamWaitEvent(q->side, q->ev_map, 0);
    if (e == cudaSuccess && ranks) e = cq::owner_dev_ranks(q->dev, n, q->side, nullptr);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(q->side, q->ev_lay, 0);
    if (e == cudaSuccess) e = cq::owner_dev_balance(q->dev, si, idx, q->policy, q->threshold, q->pot, q->side);
    if (e == cudaSuccess) e = cudaEventRecord(q->ev_bal, q->side);
    if (e != cudaSuccess) return status_of(e);
    q->st.host_ns +=
        std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0).count();
    q->st.tuples_seen += n;
    q->st.pushes++;
    return CQ_OK;
}

}  // namespace

extern "C" {

cq_status cqo_create(int64_t groups, int32_t window, int32_t passes, int32_t grid, int32_t policy,
                     int64_t threshold, double pot, void *cuda_stream, cqo_query **out) {
    if (!out) return CQ_EINVAL;
    *out = nullptr;
    const bool on_device = (policy & CQO_ON_DEVICE) != 0;
    policy &= ~CQO_ON_DEVICE;
    if (groups < 1 || groups > 2147483647LL || window < 1 || window > CQW_MAX_WINDOW || passes < 1 ||
        passes > CQW_MAX_PASSES || grid < 1 || (int64_t)grid * kBlock > groups || !valid_policy(policy) ||
        threshold < 0 || !(pot > 0.0 && pot <= 1.0))
        return CQ_EINVAL;
    if (on_device && (!device_policy(policy) || (int64_t)grid * kBlock > cq::kBalMaxThreads)) return CQ_EINVAL;
    cqo_query *q = new (std::nothrow) cqo_query();
    if (!q) return CQ_ENOMEM;
    q->G = groups;
    q->w = window;
    q->passes = passes;
    q->grid = grid;
    q->T = grid * kBlock;
    q->policy = policy;
    q->threshold = threshold;
    q->pot = pot;
    q->on_device = on_device;
    try {
        q->mp.init(q->T, groups);
        q->count.assign(groups, 0);
        q->occ.assign(groups, 0);
    } catch (...) {
        delete q;
        return CQ_ENOMEM;
    }
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
    for (int b = 0; b < 2 && e == cudaSuccess; b++) {
        e = cudaEventCreateWithFlags(&q->ev[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(q->ev[b], q->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(q->cells, 0, sizeof(int32_t) * groups * window, q->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(q->next, 0, sizeof(int32_t) * groups, q->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(q->fill, 0, sizeof(int32_t) * groups, q->stream);
    if (e == cudaSuccess && on_device) {
        e = cudaStreamCreateWithFlags(&q->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q->lay, cudaStreamNonBlocking);
        cudaEvent_t *evs[] = {&q->ev_map, &q->ev_lay, &q->ev_bal, &q->ev_own[0], &q->ev_own[1]};
        for (cudaEvent_t *ev : evs)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(q->ev_bal, q->side);
        for (int b = 0; b < 2 && e == cudaSuccess; b++) e = cudaEventRecord(q->ev_own[b], q->stream);
        for (int b = 0; b < 2 && e == cudaSuccess; b++) e = cudaEventRecord(q->ev[b], q->lay);
        if (e == cudaSuccess) {
            try {
                std::vector<int32_t> off(q->T + 1), order;
                order.reserve(groups);
                for (int t = 0; t < q->T; t++) {
                    off[t] = (int32_t)order.size();
                    order.insert(order.end(), q->mp.groups[t].begin(), q->mp.groups[t].end());
                }
                off[q->T] = (int32_t)order.size();
                e = cq::owner_dev_alloc(q->dev, groups, q->T, off.data(), order.data(), q->stream);
            } catch (...) {
                e = cudaErrorMemoryAllocation;
            }
        }
    }
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

cq_status cqo_push(cqo_query *q, const int32_t *h_keys, const int32_t *h_vals, int64_t n, int64_t *d_sums) {
    if (!q) return CQ_EINVAL;
    if (q->poisoned) return CQ_EPOISONED;
    if (n < 0) return CQ_EINVAL;
    if (n == 0) return CQ_OK;
    if (!h_keys || !h_vals || !d_sums || n > 2147483647LL) return CQ_EINVAL;
    for (int64_t i = 0; i < n; i++)
        if (h_keys[i] < 0 || (int64_t)h_keys[i] >= q->G) {
            q->poisoned = true;
            return CQ_EKEY;
        }
    cudaSetDevice(q->device);
    if (q->on_device) return push_device(q, h_keys, h_vals, n, d_sums);
    cudaError_t e = ensure_stage(q, n);
    if (e != cudaSuccess) return status_of(e);
    const int sl = q->slot;
    q->slot ^= 1;
    e = cudaEventSynchronize(q->ev[sl]);   /* the slot's previous copy has read it */
    if (e != cudaSuccess) return status_of(e);
    const auto t0 = std::chrono::steady_clock::now();
    int32_t *h = q->h_stage[sl];
    int32_t *rk = h, *rv = h + n;
    uint32_t *rpos = (uint32_t *)(h + 2 * n), *ind = (uint32_t *)(h + 3 * n);
    lay_out(q->mp, h_keys, h_vals, n, rk, rv, rpos, ind, q->tpt, q->count.data());
    /* one copy and the kernel; the host rebalances while they run */
    const size_t bytes = sizeof(int32_t) * (size_t)(3 * n + q->T + 1);
    int32_t *d = q->d_stage[sl];
    e = cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, q->stream);
    if (e == cudaSuccess) {
        owner_kernel<<<q->grid, kBlock, 0, q->stream>>>(d, d + n, (const uint32_t *)(d + 2 * n),
                                                        (const uint32_t *)(d + 3 * n), q->T, q->cells, q->next,
                                                        q->fill, q->w, q->passes, (long long *)d_sums);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(q->ev[sl], q->stream);
    if (e != cudaSuccess) return status_of(e);
    int64_t hi = 0, lo = INT64_MAX;
    for (int64_t x : q->tpt) {
        hi = x > hi ? x : hi;
        lo = x < lo ? x : lo;
    }
    Balancer bal{q->mp, rk, ind, q->count.data(), q->occ.data(), q->tpt, {}};
    const int64_t moves = bal.run(q->policy, q->threshold, q->pot);
    for (int64_t i = 0; i < n; i++) q->count[h_keys[i]] = 0;
    q->st.host_ns +=
        std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0).count();
    q->st.tuples_seen += n;
    q->st.pushes++;
    q->st.moves += moves;
    q->st.last_moves = moves;
    q->st.last_max_tpt = hi;
    q->st.last_min_tpt = lo;
    return CQ_OK;
}

cq_status cqo_sync(cqo_query *q) {
    if (!q) return CQ_EINVAL;
    cudaError_t e = cudaStreamSynchronize(q->stream);
    if (e == cudaSuccess && q->on_device) {
        e = cudaStreamSynchronize(q->lay);
        if (e == cudaSuccess) e = cudaStreamSynchronize(q->side);
        int err = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&err, q->dev.err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && err) return CQ_ETIMEOUT;   /* a look-back wait of the lay-out sort gave up */
    }
    return status_of(e);
}

cq_status cqo_stats(const cqo_query *q, cqo_stats_t *out) {
    if (!q || !out) return CQ_EINVAL;
    *out = q->st;
    if (q->on_device) {   /* the policy's figures live on the device */
        cq::BalStats b;
        cudaError_t e = cudaStreamSynchronize(q->side);
        if (e == cudaSuccess) e = cudaMemcpy(&b, q->dev.st, sizeof(b), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return status_of(e);
        out->moves = b.moves;
        out->last_moves = b.last_moves;
        out->last_max_tpt = b.last_max;
        out->last_min_tpt = b.last_min;
    }
    return CQ_OK;
}

cq_status cqo_mapping(const cqo_query *q, int32_t *off, int32_t *groups) {
    if (!q || !off || !groups) return CQ_EINVAL;
    if (q->on_device) {
        cudaError_t e = cudaStreamSynchronize(q->side);
        if (e == cudaSuccess) e = cq::owner_dev_mapping(q->dev, off, groups);
        return status_of(e);
    }
    int64_t at = 0;
    for (int t = 0; t < q->T; t++) {
        off[t] = (int32_t)at;
        for (int32_t g : q->mp.groups[t]) groups[at++] = g;
    }
    off[q->T] = (int32_t)at;
    return CQ_OK;
}

cq_status cqo_rebalance(int32_t policy, int32_t T, int64_t G, const int32_t *off, const int32_t *groups,
                        const int32_t *keys, int64_t n, int64_t threshold, double pot, int32_t *out_off,
                        int32_t *out_groups, int64_t *moves) {
    if (T < 1 || G < 1 || G > 2147483647LL || !off || !groups || (n > 0 && !keys) || n < 0 || !out_off ||
        !out_groups || !moves || !valid_policy(policy) || threshold < 0 || !(pot > 0.0 && pot <= 1.0))
        return CQ_EINVAL;
    try {
        Mapping mp;
        mp.groups.assign(T, {});
        mp.own.assign(G, -1);
        if (off[0] != 0 || off[T] != G) return CQ_EINVAL;
        for (int t = 0; t < T; t++) {
            if (off[t + 1] < off[t]) return CQ_EINVAL;
            for (int32_t j = off[t]; j < off[t + 1]; j++) {
                const int32_t g = groups[j];
                if (g < 0 || g >= G || mp.own[g] != -1) return CQ_EINVAL;   /* every group exactly once */
                mp.groups[t].push_back(g);
                mp.own[g] = t;
            }
        }
        for (int64_t i = 0; i < n; i++)
            if (keys[i] < 0 || keys[i] >= G) return CQ_EKEY;
        std::vector<int32_t> rk(n > 0 ? n : 1), count(G, 0), occ(G, 0);
        std::vector<uint32_t> ind(T + 1);
        std::vector<int64_t> tpt;
        lay_out(mp, keys, nullptr, n, rk.data(), nullptr, nullptr, ind.data(), tpt, count.data());
        Balancer bal{mp, rk.data(), ind.data(), count.data(), occ.data(), tpt, {}};
        *moves = bal.run(policy, threshold, pot);
        int64_t at = 0;
        for (int t = 0; t < T; t++) {
            out_off[t] = (int32_t)at;
            for (int32_t g : mp.groups[t]) out_groups[at++] = g;
        }
        out_off[T] = (int32_t)at;
    } catch (...) {
        return CQ_ENOMEM;
    }
    return CQ_OK;
}

void cqo_destroy(cqo_query *q) {
    if (!q) return;
    if (q->stream) cudaStreamSynchronize(q->stream);
    free_query(q);
    delete q;
}

}  /* extern "C" */
