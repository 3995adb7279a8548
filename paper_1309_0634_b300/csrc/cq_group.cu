/*
 * cq_group.cu -- the partitioned push of one or many queries in one
 * cooperative launch.
 *
 * Every query contributes chunks of consecutive effective tuples (<= 2048;
 * <= 4096 for a single query whose push replaces its whole window) and key
 * ranges of its groups; the launch walks the concatenated lists, two CTAs
 * per SM.
 *
 * Phase A (per chunk, CTAs in turn over the global chunk list):
 *   - the chunk's new keys and values and, unless the push replaces the
 *     whole window, the ring slots they overwrite are staged in shared memory:
 *     by cp.async.bulk on an mbarrier when the batch and the ring are 16-byte
 *     aligned, else by coalesced loads.  A single query's first two chunks,
 *     error flag and heavy-hitter list are requested at kernel start, and its
 *     chunk inputs are double-buffered when two CTAs per SM still fit;
 *   - the new tuples go back to the ring (bulk store, or plain stores);
 *   - a delta of one of the query's heavy hitters (chosen at its previous
 *     push) is folded into a private record -- the heaviest one in registers,
 *     the others in shared memory -- and the chunk's records are added by
 *     device atomics to one of 32 replicated accumulators per heavy hitter,
 *     so a heavy hitter's work is split over all chunks instead of landing on
 *     one owner (the paper's remedy for skew, Section 4: load moves off an
 *     overloaded worker, decided per batch and applied one batch later as in
 *     Section 3.1);
 *   - every other delta is counting-sorted by key-range partition (the
 *     paper's two-pass reordering of a batch, Section 3.1, done per chunk on
 *     the GPU) into runs padded to 16 bytes and written out by one bulk
 *     store; each key range's (begin, length) run in the chunk goes to a
 *     range-major table (the paper's threadDataIndicator).
 * Grid-wide barrier (bounded; the launch is cooperative).  A single query's
 * first key range has its state requested, and its table cleared, before it.
 * Phase B (per key range, CTAs in turn over the global range list):
 *   - the range's state (SUM, COUNT, epoch-tagged extrema) and its run table
 *     row arrive by bulk loads; each chunk's run of the range is gathered by
 *     one bulk copy per chunk, in batches of <= 8192 deltas;
 *   - the runs are folded into a shared-memory table with 32-bit shared
 *     atomics only: a sum is carried as the signed sums of the 16-bit halves
 *     of the values (exact within a batch) and folded into an int64;
 *   - one warp per heavy hitter of the range sums its replicated
 *     accumulators and puts them back to identity;
 *   - every touched group's SUM/COUNT, MIN/MAX segments and published
 *     MIN/MAX/AVG are rewritten (for a replaced window, from the new tuples
 *     alone, and groups that held tuples but got none are emptied);
 *   - groups whose insert count reached the threshold become the query's
 *     heavy hitters for its next push (an exact counting sketch).
 * Per-group state is never touched by global atomics; results are exact.
 * Every wait is bounded; a wait that gives up marks the queries of the
 * launch timed out.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "cq_group.cuh"
#include "cq_heavy.cuh"
#include "cq_internal.h"
#include "cq_push_dev.cuh"
#include "cq_avg.cuh"
#include "cq_tags.cuh"
#include "cq_tma.cuh"

namespace cq {

namespace {

using namespace pushdev;
using namespace tma;

constexpr int kT = kGThreads;
constexpr int kW = kT / 32;
constexpr uint32_t kDummy = kPadWord;   /* key word of padding deltas: never a group */

/* Runtime-flag forms of the accumulator updates (the flags vary by query). */
__device__ __forceinline__ void acc_ins(const Acc &a, int i, int32_t v, bool minmax) {
    atomicAdd(a.f(A_LO, i), v & 0xFFFF);
    atomicAdd(a.f(A_HI, i), v >> 16);
    atomicAdd(a.f(A_INS, i), 1);
    if (minmax) {
        if (v < *(volatile int32_t *)a.f(A_IMIN, i)) atomicMin(a.f(A_IMIN, i), v);
        if (v > *(volatile int32_t *)a.f(A_IMAX, i)) atomicMax(a.f(A_IMAX, i), v);
    }
}

__device__ __forceinline__ void acc_ret(const Acc &a, int i, int32_t v, bool front_dep) {
    atomicAdd(a.f(A_LO, i), -(v & 0xFFFF));
    atomicAdd(a.f(A_HI, i), -(v >> 16));
    atomicAdd(a.f(A_RET, i), 1);
    if (front_dep) atomicAdd(a.f(A_FDEP, i), 1);
}

/* Phase-B forms: the table's groups see few updates each (heavy hitters are
 * folded in phase A), so the extrema are updated unconditionally. */
__device__ __forceinline__ void tab_ins(const Acc &a, int i, int32_t v, bool minmax) {
    atomicAdd(a.f(A_LO, i), v & 0xFFFF);
    atomicAdd(a.f(A_HI, i), v >> 16);
    atomicAdd(a.f(A_INS, i), 1);
    if (minmax) {
        atomicMin(a.f(A_IMIN, i), v);
        atomicMax(a.f(A_IMAX, i), v);
    }
}

__device__ __forceinline__ void tab_ret(const Acc &a, int i, int32_t v, bool front_dep) {
    atomicAdd(a.f(A_LO, i), -(v & 0xFFFF));
    atomicAdd(a.f(A_HI, i), -(v >> 16));
    atomicAdd(a.f(A_RET, i), 1);
    if (front_dep) atomicAdd(a.f(A_FDEP, i), 1);
}

/* Bulk loads of a chunk's inputs: len4 new keys and values from the batch
 * and, when old tuples leave (`ring`), the ring slots from s0 on, all
 * completing on `bar`.  Issued by one thread. */
__device__ __forceinline__ void issue_chunk_loads(const int32_t *keys, const int32_t *vals, const int32_t *ring_k,
                                                  const int32_t *ring_v, int64_t W, int64_t cbeg, int64_t s0,
                                                  int len4, bool ring, int32_t *sk, int32_t *sv, int32_t *srk,
                                                  int32_t *srv, unsigned long long *bar) {
    mbar_expect(bar, (ring ? 16u : 8u) * (uint32_t)len4);
    tma_load(sk, keys + cbeg, 4u * len4, bar);
    tma_load(sv, vals + cbeg, 4u * len4, bar);
    if (ring) {
        ring_load(srk, ring_k, W, s0, len4, bar);
        ring_load(srv, ring_v, W, s0, len4, bar);
    }
}

__host__ __device__ constexpr int64_t pad16(int64_t x) { return (x + 15) / 16 * 16; }

/* Bulk loads of a key range's state (SUM, COUNT and, as the query needs
 * them, the back and front extrema tags) for groups [g0, g0 + range4),
 * completing on `bar`.  Issued by one thread. */
__device__ __forceinline__ void issue_range_state(const QDesc *D, int64_t g0, int range4, bool minmax, bool front,
                                                  unsigned long long *st_sum, int32_t *st_cnt,
                                                  unsigned long long *st_bmin, unsigned long long *st_bmax,
                                                  unsigned long long *st_fmin, unsigned long long *st_fmax,
                                                  unsigned long long *bar) {
    mbar_expect(bar, 12u * range4 + (minmax ? 16u * range4 : 0u) + (front ? 16u * range4 : 0u));
    tma_load(st_sum, D->sum + g0, 8u * range4, bar);
    tma_load(st_cnt, D->cnt + g0, 4u * range4, bar);
    if (minmax) {
        tma_load(st_bmin, D->bmin + g0, 8u * range4, bar);
        tma_load(st_bmax, D->bmax + g0, 8u * range4, bar);
    }
    if (front) {
        tma_load(st_fmin, D->fmin + g0, 8u * range4, bar);
        tma_load(st_fmax, D->fmax + g0, 8u * range4, bar);
    }
}

/* Tuples of chunk c (of S tuples; the last is shorter) taken by bulk copy:
 * the chunk's length rounded down to a multiple of 4. */
__device__ __forceinline__ int chunk_len4(int64_t S, int64_t n, int64_t c) {
    const int64_t b = min(c * S, n);
    return (int)(min(b + S, n) - b) & ~3;
}

/* Shared-memory layout: a fixed region (barriers, the current query's
 * descriptor, heavy-hitter hash and records, query bases), then phase A
 * (chunk inputs, flags, partition counts and cursors, sorted deltas) or
 * phase B (group table, gathered deltas, runs, prefetched state). */
struct GLayout {
    int64_t bars = 0, desc, hkey, hidx, hlist, hcnt, hw, h64, qbase, uni;
    int64_t a_in, a_arr, a_set, a_flag, a_cnt, a_cur, a_stage, a_end;
    int64_t b_acc64, b_w, b_dstage, b_pairs, b_sum, b_cnt, b_bmin, b_bmax, b_fmin, b_fmax, b_end;
    __host__ __device__ GLayout(int maxP, int maxC, int maxS, int tcap, int dcap, int dsize, int nq, bool dbuf,
                                bool replace_all) {
        desc = bars + 64;
        hkey = desc + pad16(sizeof(QDesc));
        hidx = hkey + kHotSlots * 4;
        hlist = hidx + kHotSlots * 2;
        hcnt = hlist + kMaxHot * 4;
        hw = hcnt + kMaxHot * 4;
        h64 = hw + (int64_t)A_NUM * kMaxHot * 4;
        qbase = h64 + kMaxHot * 8;
        uni = qbase + pad16((int64_t)(nq > 1 ? 2 * (nq + 1) : 0) * 4);
        /* input sets: keys, values, ring keys, ring values, one or two sets; a
           launch whose queries all replace their windows reads no ring slots
           and forms one delta per tuple */
        a_in = uni;
        a_arr = pad16((int64_t)maxS * 4);
        a_set = a_arr * (replace_all ? 2 : 4);
        a_flag = a_in + (dbuf ? 2 : 1) * a_set;
        a_cnt = a_flag + pad16(maxS);
        a_cur = a_cnt + pad16((int64_t)(maxP + 1) * 4);
        a_stage = a_cur + pad16((int64_t)(maxP + 1) * 4);
        a_end = a_stage + (int64_t)((replace_all ? 1 : 2) * maxS + maxP + 2) * dsize;
        b_acc64 = uni;
        b_w = b_acc64 + (int64_t)tcap * 8;
        b_dstage = b_w + pad16((int64_t)A_NUM * tcap * 4);
        b_pairs = b_dstage + (int64_t)dcap * dsize;
        b_sum = b_pairs + pad16((int64_t)(maxC + 1) * 8);
        b_cnt = b_sum + (int64_t)tcap * 8;
        b_bmin = b_cnt + pad16((int64_t)tcap * 4);
        b_bmax = b_bmin + (int64_t)tcap * 8;
        b_fmin = b_bmax + (int64_t)tcap * 8;
        b_fmax = b_fmin + (int64_t)tcap * 8;
        b_end = b_fmax + (int64_t)tcap * 8;
    }
    __host__ __device__ int64_t total() const { return a_end > b_end ? a_end : b_end; }
};

/* Array `arr` of input set `set` (0 keys, 1 values, 2 ring keys, 3 ring
 * values). */
__device__ __forceinline__ int32_t *in_arr(unsigned char *smem, const GLayout &L, int set, int arr) {
    return (int32_t *)(smem + L.a_in + (int64_t)set * L.a_set + (int64_t)arr * L.a_arr);
}

/* largest q with base[q] <= g */
__device__ __forceinline__ int find_query(const int *base, int nq, int g) {
    int lo = 0, hi = nq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int *q_err(const GroupArgs &ga, int q) { return ga.nq == 1 ? ga.q0.err : ga.qs[q].err; }
__device__ __forceinline__ int *q_err_host(const GroupArgs &ga, int q) {
    return ga.nq == 1 ? ga.q0.err_host : ga.qs[q].err_host;
}
__device__ __forceinline__ int *q_bad(const GroupArgs &ga, int q) { return ga.nq == 1 ? ga.q0.bad : ga.qs[q].bad; }
__device__ __forceinline__ int *q_hot_next_n(const GroupArgs &ga, int q) {
    return ga.nq == 1 ? ga.q0.hot_next_n : ga.qs[q].hot_next_n;
}

__device__ void mark_timeout(const GroupArgs &ga) {
    for (int q = threadIdx.x; q < ga.nq; q += kT) {
        atomicOr(q_err(ga, q), 2);
        int *eh = q_err_host(ga, q);
        if (eh) *(volatile int *)eh = 2;
    }
}

/* Index in a two-tier list (kMaxHot words a tier) of entry h of the combined
 * list: the n1 first-tier keys, then the second tier's. */
__device__ __forceinline__ int hot_slot(int n1, int h) { return h < n1 ? h : kMaxHot + (h - n1); }

/* Set up the current query (its descriptor already in shared memory):
 * whether it is poisoned, its heavy hitters (list, and in phase A the hash
 * and the heaviest one). */
__device__ __noinline__ void setup_query(const QDesc *D, bool with_hash, int32_t *hkey, int16_t *hidx, int32_t *hlist,
                                         int *s_skip, int *s_nhot, int *s_top) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __shared__ int s_n1;
    if (tid == 0) {
        *s_skip = *(volatile int *)D->err;   /* set only by earlier launches */
        const int n1 = *s_skip ? 0 : min(D->hot_cur_n[0], D->hot_cap);
        s_n1 = n1;
        *s_nhot = *s_skip ? 0 : n1 + min(D->hot_cur_n[1], D->hot_cap - n1);
    }
    for (int s = tid; s < kHotSlots; s += kT) hkey[s] = -1;
    __syncthreads();
    const int n_hot = *s_nhot, n1 = s_n1;
    for (int h = tid; h < n_hot; h += kT) {
        const int32_t k = D->hot_cur[hot_slot(n1, h)];
        hlist[h] = k;
        if (with_hash) {
            uint32_t s = hot_hash(k);
            for (int probe = 0; probe < kHotSlots; probe++) {
                const int prev = atomicCAS(&hkey[s], -1, k);
                if (prev == -1 || prev == k) {
                    hidx[s] = (int16_t)h;
                    break;
                }
                s = (s + 1) & (kHotSlots - 1);
            }
        }
    }
    if (warp == 0) {
        int best = -1, bestc = -1;
        if (with_hash)
            for (int h = lane; h < n_hot; h += 32) {
                const int c = D->hot_cur_cnt[hot_slot(n1, h)];
                if (c > bestc || (c == bestc && h < best)) {
                    bestc = c;
                    best = h;
                }
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int oc = __shfl_xor_sync(kFull, bestc, o), ob = __shfl_xor_sync(kFull, best, o);
            if (oc > bestc || (oc == bestc && ob >= 0 && (best < 0 || ob < best))) {
                bestc = oc;
                best = ob;
            }
        }
        if (lane == 0) *s_top = best;
    }
    __syncthreads();
}

/* setup_query for a single-query launch whose error flag and heavy-hitter
 * count were read, and whose heavy-hitter list and counts were bulk-loaded
 * into hlist / hcnt (completing on `bar`), at kernel start. */
__device__ __noinline__ void setup_query_prefetched(const QDesc *D, int err, int n1raw, int n2raw,
                                                    unsigned long long *bar, int32_t *hkey, int16_t *hidx,
                                                    int32_t *hlist, const int32_t *hcnt, const int32_t *hsecond,
                                                    int *s_skip, int *s_nhot, int *s_top, bool *timed_out) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int s = tid; s < kHotSlots; s += kT) hkey[s] = -1;
    if (tid == 0) {
        if (!mbar_wait(bar, 0)) *timed_out = true;
        *s_skip = err;
    }
    const int n1 = err ? 0 : min(n1raw, D->hot_cap);
    const int n_hot = n1 + (err ? 0 : min(n2raw, D->hot_cap - n1));
    if (tid == 0) *s_nhot = n_hot;
    __syncthreads();
    /* entry h of the list: the first tier's (in hlist), then the second
       tier's (bulk-loaded to hsecond), each moved to hlist[h] by its thread */
    for (int h = tid; h < n_hot; h += kT) {
        const int32_t k = h < n1 ? hlist[h] : hsecond[h - n1];
        if (h >= n1) hlist[h] = k;
        uint32_t s = hot_hash(k);
        for (int probe = 0; probe < kHotSlots; probe++) {
            const int prev = atomicCAS(&hkey[s], -1, k);
            if (prev == -1 || prev == k) {
                hidx[s] = (int16_t)h;
                break;
            }
            s = (s + 1) & (kHotSlots - 1);
        }
    }
    if (warp == 0) {
        int best = -1, bestc = -1;
        for (int h = lane; h < n_hot; h += 32) {
            const int c = h < n1 ? hcnt[h] : hsecond[kMaxHot + h - n1];
            if (c > bestc || (c == bestc && h < best)) {
                bestc = c;
                best = h;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int oc = __shfl_xor_sync(kFull, bestc, o), ob = __shfl_xor_sync(kFull, best, o);
            if (oc > bestc || (oc == bestc && ob >= 0 && (best < 0 || ob < best))) {
                bestc = oc;
                best = ob;
            }
        }
        if (lane == 0) *s_top = best;
    }
    __syncthreads();
}

/* Exclusive scan of the .y fields of a[0, n) in place; returns the total. */
template <int NT>
__device__ __noinline__ uint32_t block_scan_pairs(uint2 *a, int n) {
    constexpr int kWarps = NT / 32;
    __shared__ uint32_t wsum[kWarps];
    __shared__ uint32_t tot;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + NT - 1) / NT;
    const int b0 = tid * per;
    uint32_t s = 0;
    for (int j = 0; j < per; j++)
        if (b0 + j < n) s += a[b0 + j].y;
    uint32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < kWarps ? wsum[lane] : 0;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kWarps) wsum[lane] = wi - w;
        if (lane == kWarps - 1) tot = wi;
    }
    __syncthreads();
    uint32_t run = wsum[warp] + incl - s;
    for (int j = 0; j < per; j++)
        if (b0 + j < n) {
            const uint32_t x = a[b0 + j].y;
            a[b0 + j].y = run;
            run += x;
        }
    const uint32_t total = tot;
    __syncthreads();
    return total;
}

template <int DS>
__global__ void __launch_bounds__(kT, 2) group_kernel(const GroupArgs ga) {
    typedef uint2 Delta;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const GLayout L(ga.maxP, ga.maxC, ga.maxS, ga.tcap, ga.dcap, DS, ga.nq, ga.dbuf != 0, ga.replace_all != 0);
    /* [0] input set 0, [1] gather, [2] range state, [3] heavy hitters, [4] input set 1, [5] range runs */
    unsigned long long *bars = (unsigned long long *)(smem + L.bars);
    QDesc *D = (QDesc *)(smem + L.desc);
    int32_t *hkey = (int32_t *)(smem + L.hkey);
    int16_t *hidx = (int16_t *)(smem + L.hidx);
    int32_t *hlist = (int32_t *)(smem + L.hlist);
    int32_t *hcnt = (int32_t *)(smem + L.hcnt);
    int32_t *hsecond = (int32_t *)(smem + L.hw);   /* second list tier at kernel start (2 x kMaxHot words) */
    const Acc hacc{(int32_t *)(smem + L.hw), (long long *)(smem + L.h64), kMaxHot};
    int *cbase = (int *)(smem + L.qbase);
    int *rbase = cbase + (ga.nq + 1);
    __shared__ int s_nhot, s_top, s_skip, s_pre_err, s_pre_n1, s_pre_n2;
    __shared__ int s_nheavy;                 /* partitions of the chunk far above their share */
    __shared__ int s_gr;                     /* the key range drawn from the launch's counter */
    __shared__ uint32_t s_heavy[kHeavyList];
    __shared__ __align__(16) int32_t s_emkey[kEmSlots];   /* the query's keys found heavy within this push */
    __shared__ long long wtop_sum[kW];
    __shared__ int32_t wtop_i[kW][6];
    unsigned long long *trace = ga.trace ? ga.trace + (int64_t)blockIdx.x * 8 : nullptr;
    if (trace && tid == 0) trace[0] = globaltimer();

    /* A single-query launch knows its chunks' addresses from the kernel
       parameters: the inputs of its first chunk (and, double-buffered, of its
       second) are requested before anything else, as are the query's error
       flag and heavy-hitter list (CTAs with a phase-A chunk set the query up
       there). */
    const bool single = ga.nq == 1;
    const bool dbuf = ga.dbuf != 0;
    const bool prefetched = single && (int)blockIdx.x < ga.C_tot;
    const bool aligned1 = single && (ga.q0.flags & QF_ALIGNED);
    const int len4_0 = prefetched && aligned1 ? chunk_len4(ga.q0.S, ga.q0.n, blockIdx.x) : 0;
    const int len4_1 =
        dbuf && prefetched && aligned1 && (int)blockIdx.x + ga.grid < ga.C_tot ? chunk_len4(ga.q0.S, ga.q0.n, blockIdx.x + ga.grid) : 0;
    if (prefetched && tid == 32) {
        s_pre_err = *(volatile int *)ga.q0.err;
        s_pre_n1 = *(volatile int *)ga.q0.hot_cur_n;
        s_pre_n2 = *(volatile int *)(ga.q0.hot_cur_n + 1);
    }
    if (tid == 0) {
        for (int b = 0; b < 6; b++) mbar_init(&bars[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (prefetched) {
            /* both tiers of the list; the second lands in the heavy-hitter
               accumulators' space, which phase A initialises only later */
            mbar_expect(&bars[3], 16u * kMaxHot);
            tma_load(hlist, ga.q0.hot_cur, 4u * kMaxHot, &bars[3]);
            tma_load(hcnt, ga.q0.hot_cur_cnt, 4u * kMaxHot, &bars[3]);
            tma_load(hsecond, ga.q0.hot_cur + kMaxHot, 4u * kMaxHot, &bars[3]);
            tma_load(hsecond + kMaxHot, ga.q0.hot_cur_cnt + kMaxHot, 4u * kMaxHot, &bars[3]);
        }
        for (int set = 0; set < 2; set++) {
            const int len4 = set ? len4_1 : len4_0;
            if (len4 == 0) continue;
            const int64_t cbeg = (int64_t)(blockIdx.x + set * ga.grid) * ga.q0.S;
            int64_t s0 = ga.q0.slot0 + cbeg;
            if (s0 >= ga.q0.W) s0 -= ga.q0.W;
            issue_chunk_loads(ga.q0.keys, ga.q0.vals, ga.q0.ring_k, ga.q0.ring_v, ga.q0.W, cbeg, s0, len4,
                              ga.q0.old_len > 0, in_arr(smem, L, set, 0), in_arr(smem, L, set, 1),
                              in_arr(smem, L, set, 2), in_arr(smem, L, set, 3), set ? &bars[4] : &bars[0]);
        }
    }
    if (ga.nq > 1)
        for (int q = tid; q <= ga.nq; q += kT) {
            cbase[q] = ga.chunk_base[q];
            rbase[q] = ga.range_base[q];
        }
    /* a block resets each query's next heavy-hitter list before the barrier */
    for (int q = blockIdx.x * kT + tid; q < ga.nq; q += ga.grid * kT) {
        q_hot_next_n(ga, q)[0] = 0;
        q_hot_next_n(ga, q)[1] = 0;
    }
    __syncthreads();

    int cur_q = -1;
    /* ---------------- phase A ---------------- */
    uint8_t *flag = (uint8_t *)(smem + L.a_flag);
    uint32_t *cnt = (uint32_t *)(smem + L.a_cnt);
    uint32_t *cur = (uint32_t *)(smem + L.a_cur);
    Delta *stage_s = (Delta *)(smem + L.a_stage);
    bool timed_out = false;
    uint32_t par0 = 0, par1 = 0;   /* phases of the input sets' barriers */
    int it = 0;
    for (int gc = blockIdx.x; gc < ga.C_tot && !timed_out; gc += ga.grid, it++) {
        const int q = ga.nq == 1 ? 0 : find_query(cbase, ga.nq, gc);
        if (q != cur_q) {
            if (tid == 0) {
                if (ga.nq == 1) *D = ga.q0;
                else *D = ga.qs[q];
            }
            __syncthreads();
            if (prefetched)
                setup_query_prefetched(D, s_pre_err, s_pre_n1, s_pre_n2, &bars[3], hkey, hidx, hlist, hcnt, hsecond,
                                       &s_skip, &s_nhot, &s_top, &timed_out);
            else
                setup_query(D, true, hkey, hidx, hlist, &s_skip, &s_nhot, &s_top);
            cur_q = q;
        }
        const int c = gc - (ga.nq == 1 ? 0 : cbase[q]);
        const int set = dbuf ? (it & 1) : 0;
        unsigned long long *ibar = set ? &bars[4] : &bars[0];
        uint32_t &ipar = set ? par1 : par0;
        int32_t *sk = in_arr(smem, L, set, 0), *sv = in_arr(smem, L, set, 1);
        int32_t *srk = in_arr(smem, L, set, 2), *srv = in_arr(smem, L, set, 3);
        /* inputs already requested: at kernel start (first two chunks), or at
           the end of the chunk two before this one (double-buffered) */
        const bool issued = it == 0 ? len4_0 > 0
                          : it == 1 ? len4_1 > 0
                                    : dbuf && !s_skip && (D->flags & QF_ALIGNED) && chunk_len4(D->S, D->n, c) > 0;
        if (s_skip) {   /* a poisoned query: nothing of it is used or written */
            if (issued) {
                if (tid == 0 && !mbar_wait(ibar, ipar)) timed_out = true;
                ipar ^= 1u;
            }
            if (__syncthreads_or(timed_out)) {
                timed_out = true;
                break;
            }
            continue;
        }
        const int flags = D->flags;
        const bool minmax = flags & QF_MINMAX, front = (flags & QF_FRONT) != 0;
        const int P = D->P, rbits = D->rbits;
        const int64_t W = D->W, G = D->G;
        const int64_t cbeg = min((int64_t)c * D->S, D->n);
        const int len = (int)(min(cbeg + D->S, D->n) - cbeg);
        int64_t s0 = D->slot0 + cbeg;
        if (s0 >= W) s0 -= W;
        const bool tma = (flags & QF_ALIGNED) != 0;
        const int len4 = tma ? (len & ~3) : 0;
        const int n_hot = s_nhot, top = s_top;
        for (int p = tid; p <= P; p += kT) cnt[p] = 0;
        for (int h = tid; h < n_hot; h += kT) acc_init(hacc, h);
        if (tid == 0) s_nheavy = 0;
        if (tid == 0 && len4 > 0 && !issued)
            issue_chunk_loads(D->keys, D->vals, D->ring_k, D->ring_v, W, cbeg, s0, len4, D->old_len > 0, sk, sv,
                              srk, srv, ibar);
        /* unaligned batches and ragged tails: asynchronous copies, so that
           every element of a thread is in flight at once */
        for (int i = len4 + tid; i < len; i += kT) {
            int64_t sl = s0 + i;
            if (sl >= W) sl -= W;
            cp_async(sk + i, D->keys + cbeg + i);
            cp_async(sv + i, D->vals + cbeg + i);
            if (D->old_len > 0) {
                cp_async(srk + i, D->ring_k + sl);
                cp_async(srv + i, D->ring_v + sl);
            }
        }
        if (len4 < len) cp_async_wait_all();
        if (len4 > 0) {
            if (tid == 0 && !mbar_wait(ibar, ipar)) timed_out = true;
            ipar ^= 1u;
        }
        if (__syncthreads_or(timed_out)) {
            timed_out = true;
            break;
        }
        /* the new tuples go to the ring (their old occupants are in smem) */
        if (tid == 0 && len4 > 0) {
            fence_async_smem();
            ring_store(D->ring_k, sk, W, s0, len4);
            ring_store(D->ring_v, sv, W, s0, len4);
            tma_commit();
        }
        for (int i = len4 + tid; i < len; i += kT) {
            int64_t sl = s0 + i;
            if (sl >= W) sl -= W;
            D->ring_k[sl] = sk[i];
            D->ring_v[sl] = sv[i];
        }
        /* pass 1: heavy hitters into the private records (the heaviest in
           registers), the others counted per partition; flag bits: 1 insert
           exchanged, 2 retract exchanged, 4 the retract leaves the front */
        long long r_sum = 0;
        int32_t r_ins = 0, r_ret = 0;
        int32_t r_imin = INT32_MAX, r_imax = INT32_MIN, r_fdep = 0;
        bool bad = false;
        const uint32_t Wu = (uint32_t)W, hmod = (uint32_t)D->hmod;
        const int32_t old_len = (int32_t)D->old_len, fa = (int32_t)D->fa, fb = (int32_t)D->fb;
        for (int i = tid; i < len; i += kT) {
            uint32_t sl = (uint32_t)s0 + (uint32_t)i;
            if (sl >= Wu) sl -= Wu;
            int32_t rel = (int32_t)sl - (int32_t)hmod;
            if (rel < 0) rel += (int32_t)Wu;
            uint32_t f = 0;
            const int32_t k = sk[i];
            if ((uint32_t)k >= (uint32_t)G) {
                bad = true;
            } else {
                const int h = n_hot ? hot_find(hkey, hidx, k) : -1;
                if (h >= 0 && h == top) {
                    const int32_t v = sv[i];
                    r_sum += v;
                    r_ins++;
                    r_imin = min(r_imin, v);
                    r_imax = max(r_imax, v);
                } else if (h >= 0) {
                    acc_ins(hacc, h, sv[i], minmax);
                } else {
                    atomicAdd(&cnt[(uint32_t)k >> rbits], 1u);
                    f = 1;
                }
            }
            if (rel < old_len) {
                const int32_t ok = srk[i];
                if ((uint32_t)ok < (uint32_t)G) {
                    const bool fr = front && rel >= fa && rel < fb;
                    const int h = n_hot ? hot_find(hkey, hidx, ok) : -1;
                    if (h >= 0 && h == top) {
                        r_sum -= srv[i];
                        r_ret++;
                        r_fdep += fr ? 1 : 0;
                    } else if (h >= 0) {
                        acc_ret(hacc, h, srv[i], fr);
                    } else {
                        atomicAdd(&cnt[(uint32_t)ok >> rbits], 1u);
                        f |= fr ? 6u : 2u;
                    }
                }
            }
            flag[i] = (uint8_t)f;
        }
        if (bad) atomicOr(D->bad, 1);
        if (top >= 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                r_sum += __shfl_xor_sync(kFull, r_sum, o);
                r_ins += __shfl_xor_sync(kFull, r_ins, o);
                r_ret += __shfl_xor_sync(kFull, r_ret, o);
                r_imin = min(r_imin, __shfl_xor_sync(kFull, r_imin, o));
                r_imax = max(r_imax, __shfl_xor_sync(kFull, r_imax, o));
                r_fdep += __shfl_xor_sync(kFull, r_fdep, o);
            }
            if (lane == 0) {
                wtop_sum[warp] = r_sum;
                wtop_i[warp][0] = r_ins;
                wtop_i[warp][1] = r_ret;
                wtop_i[warp][2] = r_imin;
                wtop_i[warp][3] = r_imax;
                wtop_i[warp][4] = r_fdep;
            }
        }
        /* the previous chunk's bulk stores must have read the staging buffer */
        if (tid == 0) tma_wait_read();
        __syncthreads();
        /* partition runs (and the partitions far above their share: cq_heavy.cuh) */
        const uint32_t total = block_scan_even3<kT>(cnt, cur, cnt, P, D->heavy_bound, s_heavy, &s_nheavy, kHeavyList);
        {   /* each key range's run in this chunk: (begin, length), range-major */
            uint2 *pairs = (uint2 *)D->off;
            const int ppp = D->ppp, R = D->R, Cpad = (D->C + 1) & ~1;
            for (int r = tid; r < R; r += kT) {
                const int p0 = r * ppp, p1 = min(P, p0 + ppp);
                pairs[(int64_t)r * Cpad + c] = make_uint2(cnt[p0], cnt[p1] - cnt[p0]);
            }
        }
        /* the chunk's heavy-hitter updates, added to the query's accumulators */
        for (int h = tid; h < n_hot; h += kT) {
            acc_fold(hacc, h);
            HotAcc r;
            r.sum = hacc.acc64[h];
            r.ins = *hacc.f(A_INS, h);
            r.ret = *hacc.f(A_RET, h);
            r.imin = *hacc.f(A_IMIN, h);
            r.imax = *hacc.f(A_IMAX, h);
            r.fdep = *hacc.f(A_FDEP, h);
            if (h == top) {
                for (int w = 0; w < kW; w++) {
                    r.sum += wtop_sum[w];
                    r.ins += wtop_i[w][0];
                    r.ret += wtop_i[w][1];
                    r.imin = min(r.imin, wtop_i[w][2]);
                    r.imax = max(r.imax, wtop_i[w][3]);
                    r.fdep += wtop_i[w][4];
                }
            }
            HotAcc *a = D->hotacc + (int64_t)(c & (kHotRep - 1)) * kMaxHot + h;
            if (r.ins | r.ret) atomicAdd((unsigned long long *)&a->sum, (unsigned long long)r.sum);
            if (r.ins) {
                atomicAdd(&a->ins, r.ins);
                if (minmax) {
                    atomicMin(&a->imin, r.imin);
                    atomicMax(&a->imax, r.imax);
                }
            }
            if (r.ret) {
                atomicAdd(&a->ret, r.ret);
                if (r.fdep) atomicAdd(&a->fdep, r.fdep);
            }
        }
        /* pass 2: place the exchanged deltas at their partition's cursor */
        for (int i = tid; i < len; i += kT) {
            const uint32_t f = flag[i];
            if (f & 1u) {
                const int32_t k = sk[i];
                const uint32_t pos = atomicAdd(&cur[(uint32_t)k >> rbits], 1u);
                stage_s[pos] = DeltaIO::make((uint32_t)k, sv[i]);
            }
            if (f & 2u) {
                const int32_t ok = srk[i];
                const bool fr = (f & 4u) != 0;
                const uint32_t pos = atomicAdd(&cur[(uint32_t)ok >> rbits], 1u);
                stage_s[pos] = DeltaIO::make((uint32_t)ok | kRetract | (fr ? kFrontDep : 0u), srv[i]);
            }
        }
        __syncthreads();
        for (int p = tid; p < P; p += kT)
            if (cur[p] < cnt[p + 1]) stage_s[cur[p]] = DeltaIO::make(kDummy, 0);
        __syncthreads();
        /* runs far above their share: a key heavy within this push (cq_heavy.cuh) */
        const int n_heavy = min(s_nheavy, kHeavyList);
        if (n_heavy > 0) {
            for (int j = warp; j < n_heavy; j += kW) {
                const uint32_t p = s_heavy[j];
                fold_heavy_run(stage_s + cnt[p], cnt[p + 1] - cnt[p], D->heavy_min, c & (kHotRep - 1), D->emkey,
                                      D->emacc, D->emfolds, minmax);
            }
            __syncthreads();
        }
        if (tid == 0) {
            if (total) {
                fence_async_smem();
                tma_store((Delta *)D->stage + (int64_t)c * D->stride, stage_s, total * (uint32_t)DS);
                tma_commit();
            }
            tma_wait_read();   /* sk/sv (ring stores) and stage_s are free again */
            /* double-buffered: this set now takes the chunk two ahead */
            const int cn = c + 2 * ga.grid;
            if (dbuf && (flags & QF_ALIGNED) && cn < D->C) {
                const int len4n = chunk_len4(D->S, D->n, cn);
                if (len4n > 0) {
                    const int64_t cbn = (int64_t)cn * D->S;
                    int64_t sn = D->slot0 + cbn;
                    if (sn >= W) sn -= W;
                    issue_chunk_loads(D->keys, D->vals, D->ring_k, D->ring_v, W, cbn, sn, len4n, D->old_len > 0, sk,
                                      sv, srk, srv, ibar);
                }
            }
        }
        __syncthreads();
    }
    /* staging, ring and offset writes complete and visible before the barrier */
    if (tid == 0) {
        tma_wait_all();
        fence_async_global();
    }
    const Acc tab{(int32_t *)(smem + L.b_w), (long long *)(smem + L.b_acc64), ga.tcap};
    Delta *dstage = (Delta *)(smem + L.b_dstage);
    uint2 *pairs = (uint2 *)(smem + L.b_pairs);   /* per chunk: begin, then offset in the gather */
    unsigned long long *st_sum = (unsigned long long *)(smem + L.b_sum);
    int32_t *st_cnt = (int32_t *)(smem + L.b_cnt);
    unsigned long long *st_bmin = (unsigned long long *)(smem + L.b_bmin);
    unsigned long long *st_bmax = (unsigned long long *)(smem + L.b_bmax);
    unsigned long long *st_fmin = (unsigned long long *)(smem + L.b_fmin);
    unsigned long long *st_fmax = (unsigned long long *)(smem + L.b_fmax);
    /* a single query's first key range: its state is not written in phase A,
       so it is requested, and the table cleared, before the grid barrier */
    const bool pre_b = ga.nq == 1 && cur_q == 0 && !s_skip && !timed_out && (int)blockIdx.x < ga.R_tot;
    if (pre_b) {
        __syncthreads();   /* phase A's shared memory is free */
        const int q0 = (int)blockIdx.x * D->ppp, q1 = min(D->P, q0 + D->ppp);
        const int64_t g0 = (int64_t)q0 << D->rbits;
        const int range = (int)(min((int64_t)q1 << D->rbits, D->G) - g0);
        if (tid == 0)
            issue_range_state(D, g0, (range + 3) & ~3, (D->flags & QF_MINMAX) != 0,
                              (D->flags & QF_FRONT) != 0, st_sum, st_cnt, st_bmin, st_bmax, st_fmin, st_fmax,
                              &bars[2]);
        for (int l = tid; l < range; l += kT) acc_init(tab, l);
    }
    if (trace && tid == 0) trace[2] = globaltimer();
    const bool arrived = grid_barrier(ga.bar, timed_out ? 0ULL : ga.bar_target);   /* always arrive */
    if (timed_out || !arrived) {
        mark_timeout(ga);
        return;
    }
    fence_async_global();
    if (trace && tid == 0) trace[3] = globaltimer();
    if (blockIdx.x == 0)
        for (int q = tid; q < ga.nq; q += kT) {
            int *bad = q_bad(ga, q);
            if (*(volatile int *)bad) {
                *bad = 0;
                atomicOr(q_err(ga, q), 1);
                int *eh = q_err_host(ga, q);
                if (eh) *(volatile int *)eh = 1;
            }
        }

    /* ---------------- phase B ---------------- */
    uint32_t g_parity = 0, s_parity = 0, p_parity = 0;
    /* One query: CTA b takes ranges b, b + grid, ...  Several queries, whose
       ranges differ widely in cost: each CTA draws its next range from a
       counter (bar[1], zeroed with the barrier before the launch), so a CTA
       that drew expensive ranges takes fewer. */
    const bool drawn = ga.nq > 1;
    const auto next_range = [&](int gr) -> int {
        if (!drawn) return gr + ga.grid;
        __syncthreads();
        if (tid == 0) s_gr = (int)atomicAdd(ga.bar + 1, 1ull);
        __syncthreads();
        return s_gr;
    };
    /* cur_q carries over: a range of the query phase A ended with needs no
       new descriptor or heavy-hitter list */
    for (int gr = drawn ? next_range(0) : (int)blockIdx.x; gr < ga.R_tot; gr = next_range(gr)) {
        const int q = ga.nq == 1 ? 0 : find_query(rbase, ga.nq, gr);
        if (q != cur_q) {
            if (tid == 0) {
                if (ga.nq == 1) *D = ga.q0;
                else *D = ga.qs[q];
            }
            __syncthreads();
            setup_query(D, false, hkey, hidx, hlist, &s_skip, &s_nhot, &s_top);
            cur_q = q;
        }
        if (s_skip) continue;
        /* the keys found heavy within the push, needed after the range's
           deltas: copied now without waiting (warp 1), waited for below */
        if (warp == 1 && lane < kEmSlots / 4)
            cp_async((uint4 *)s_emkey + lane, (const uint4 *)D->emkey + lane);
        const int lr = gr - (ga.nq == 1 ? 0 : rbase[q]);
        const int flags = D->flags;
        const bool minmax = flags & QF_MINMAX, front = (flags & QF_FRONT) != 0;
        const int P = D->P, C = D->C;
        const uint32_t epoch = D->epoch;
        const int q0 = lr * D->ppp, q1 = min(P, q0 + D->ppp);
        const int64_t g0 = (int64_t)q0 << D->rbits;
        const int64_t g1 = min((int64_t)q1 << D->rbits, D->G);
        const int range = (int)(g1 - g0);
        const int range4 = (range + 3) & ~3;
        const Delta *stage = (const Delta *)D->stage;
        /* the range's state (already requested for a pre-barrier first range)
           and its runs' (begin, length) in every chunk */
        const int Cpad = (C + 1) & ~1;
        const bool first_pre = pre_b && gr == (int)blockIdx.x;
        if (tid == 0) {
            mbar_expect(&bars[5], 8u * (uint32_t)Cpad);
            tma_load(pairs, (const uint2 *)D->off + (int64_t)lr * Cpad, 8u * Cpad, &bars[5]);
            if (!first_pre)
                issue_range_state(D, g0, range4, minmax, front, st_sum, st_cnt, st_bmin, st_bmax, st_fmin, st_fmax,
                                  &bars[2]);
        }
        if (!first_pre)
            for (int l = tid; l < range; l += kT) acc_init(tab, l);
        if (tid == 0 && (!mbar_wait(&bars[2], s_parity) || !mbar_wait(&bars[5], p_parity))) timed_out = true;
        s_parity ^= 1u;
        p_parity ^= 1u;
        if (__syncthreads_or(timed_out)) {
            mark_timeout(ga);
            return;
        }
        const uint32_t total = block_scan_pairs<kT>(pairs, C);
        for (uint32_t b0 = 0; b0 < total && !timed_out; b0 += (uint32_t)ga.dcap) {
            const uint32_t b1 = min(total, b0 + (uint32_t)ga.dcap);
            if (tid == 0) mbar_expect(&bars[1], (b1 - b0) * (uint32_t)DS);
            __syncthreads();
            for (int c = tid; c < C; c += kT) {
                const uint32_t s0 = pairs[c].y, s1 = c + 1 < C ? pairs[c + 1].y : total;
                const uint32_t lo = max(s0, b0), hi = min(s1, b1);
                if (lo < hi)
                    tma_load(dstage + (lo - b0), stage + (int64_t)c * D->stride + pairs[c].x + (lo - s0),
                             (hi - lo) * (uint32_t)DS, &bars[1]);
            }
            if (tid == 0 && !mbar_wait(&bars[1], g_parity)) timed_out = true;
            g_parity ^= 1u;
            if (__syncthreads_or(timed_out)) {
                timed_out = true;
                break;
            }
            for (uint32_t i = tid; i < b1 - b0; i += kT) {
                uint32_t kf;
                int32_t dv;
                DeltaIO::get(dstage[i], kf, dv);
                const int l = (int)((int64_t)(kf & kKeyMask) - g0);
                if (l < 0 || l >= range) continue;   /* padding deltas and any out-of-range key */
                if (kf & kRetract) tab_ret(tab, l, dv, (kf & kFrontDep) != 0);
                else tab_ins(tab, l, dv, minmax);
            }
            __syncthreads();
            for (int l = tid; l < range; l += kT) acc_fold(tab, l);
            __syncthreads();
        }
        if (warp == 1 && lane < kEmSlots / 4) cp_async_wait_all();
        if (__syncthreads_or(timed_out)) {
            mark_timeout(ga);
            return;
        }
        /* heavy hitters of the range, then the keys found heavy within the
           push (slots n_hot ..): a warp per key sums its replicas (a lane
           each), adds them to the table and puts them back to identity */
        const int n_hot = s_nhot;
        for (int h = warp; h < n_hot + kEmSlots; h += kW) {
            const bool em = h >= n_hot;
            const int32_t key = em ? s_emkey[h - n_hot] : hlist[h];
            if ((int64_t)key < g0 || (int64_t)key >= g1) continue;   /* also a free slot (-1) */
            long long hs = 0;
            int32_t ins = 0, ret = 0, imin = INT32_MAX, imax = INT32_MIN, fdep = 0;
            HotAcc *const base = em ? D->emacc + (h - n_hot) : D->hotacc + h;
            const int stride = em ? kEmSlots : kMaxHot;
            for (int r = lane; r < kHotRep; r += 32) {
                HotAcc *a = base + (int64_t)r * stride;
                hs += __ldcg(&a->sum);
                ins += __ldcg(&a->ins);
                ret += __ldcg(&a->ret);
                imin = min(imin, __ldcg(&a->imin));
                imax = max(imax, __ldcg(&a->imax));
                fdep += __ldcg(&a->fdep);
                a->sum = 0;
                a->ins = 0;
                a->ret = 0;
                a->imin = INT32_MAX;
                a->imax = INT32_MIN;
                a->fdep = 0;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                hs += __shfl_xor_sync(kFull, hs, o);
                ins += __shfl_xor_sync(kFull, ins, o);
                ret += __shfl_xor_sync(kFull, ret, o);
                imin = min(imin, __shfl_xor_sync(kFull, imin, o));
                imax = max(imax, __shfl_xor_sync(kFull, imax, o));
                fdep += __shfl_xor_sync(kFull, fdep, o);
            }
            if (lane == 0) {
                const int l = (int)(key - g0);
                tab.acc64[l] += hs;
                *tab.f(A_INS, l) += ins;
                *tab.f(A_RET, l) += ret;
                *tab.f(A_IMIN, l) = min(*tab.f(A_IMIN, l), imin);
                *tab.f(A_IMAX, l) = max(*tab.f(A_IMAX, l), imax);
                *tab.f(A_FDEP, l) += fdep;
                if (em) D->emkey[h - n_hot] = -1;   /* only this range's owner frees it */
            }
        }
        __syncthreads();
        const bool avg = flags & QF_AVG;
        const bool replace = flags & QF_REPLACE;
        for (int l = tid; l < range; l += kT) {
            const int32_t ins = *tab.f(A_INS, l), ret = *tab.f(A_RET, l);
            /* a replaced window also empties the groups that had tuples */
            if (ins + ret == 0 && (!replace || st_cnt[l] == 0)) continue;
            const int64_t g = g0 + l;
            const long long s = (replace ? 0LL : (long long)st_sum[l]) + tab.acc64[l];
            const int32_t cn = (replace ? 0 : st_cnt[l]) + (ins - ret);
            D->sum[g] = (unsigned long long)s;
            D->cnt[g] = cn;
            if (minmax) {
                int32_t blo = untag_dn(st_bmin[l], epoch, INT32_MAX);
                int32_t bhi = untag_up(st_bmax[l], epoch, INT32_MIN);
                if (ins) {
                    blo = min(blo, *tab.f(A_IMIN, l));
                    bhi = max(bhi, *tab.f(A_IMAX, l));
                    D->bmin[g] = tag_dn(epoch, blo);
                    D->bmax[g] = tag_up(epoch, bhi);
                }
                /* the front has live tags only in pushes that expire front
                   tuples; otherwise it decodes empty */
                int32_t flo_v = INT32_MAX, fhi_v = INT32_MIN;
                if (front) {
                    const int32_t dep = *tab.f(A_FDEP, l);
                    const unsigned long long tf_lo = st_fmin[l], tf_hi = st_fmax[l];
                    flo_v = untag_up(tf_lo, epoch, INT32_MAX);
                    fhi_v = untag_dn(tf_hi, epoch, INT32_MIN);
                    if (dep > 0 && (uint32_t)(tf_lo >> 32) == epoch) {
                        const int2 x = front_next(D->fptr, D->sufs, g, dep);
                        flo_v = x.x;
                        fhi_v = x.y;
                        D->fmin[g] = tag_up(epoch, flo_v);
                        D->fmax[g] = tag_dn(epoch, fhi_v);
                    }
                }
                D->rmin[g] = cn > 0 ? min(blo, flo_v) : INT32_MAX;
                D->rmax[g] = cn > 0 ? max(bhi, fhi_v) : INT32_MIN;
            }
            if (avg) {
                D->ravg[g] = cn > 0 ? avg_rn(s, cn)
                                    : __longlong_as_double(0x7FF8000000000000LL);
            }
            if (D->hot_cap && (uint32_t)ins >= D->hot_threshold) {
                const int tier = (uint32_t)ins >= D->hot_gthr ? 0 : 1;
                const int idx = atomicAdd(D->hot_next_n + tier, 1);
                if (idx < D->hot_cap) {
                    D->hot_next[tier * kMaxHot + idx] = (int32_t)g;
                    D->hot_next_cnt[tier * kMaxHot + idx] = ins;
                }
            }
        }
        __syncthreads();
    }
    if (trace && tid == 0) trace[5] = globaltimer();
}

}  // namespace

int64_t group_smem_bytes(int maxP, int maxC, int maxS, int tcap, int dcap, bool front, int nq, bool dbuf,
                         bool replace_all) {
    (void)front;
    return GLayout(maxP, maxC, maxS, tcap, dcap, 8, nq, dbuf, replace_all).total();
}

const void *group_kernel_ptr(bool front) {
    (void)front;   /* one delta form for every push */
    return (const void *)group_kernel<8>;
}


}  // namespace cq
