/*
 * cq_stream.cu -- the persistent multi-batch push of one query (cq_stream.cuh).
 *
 * One cooperative launch of two CTAs per SM folds nb batches into the
 * query's window, in stream order.  Roles are taken at start-up by arrival on
 * each SM: the first CTA of an SM is a producer, the second a consumer, so
 * every SM runs one of each and the two overlap.
 *
 * Producer p, for every batch i (chunks p, p + nA, ... of the batch):
 *   - the chunk's keys and values arrive by bulk copy, requested two chunks
 *     ahead (they may belong to a later batch); the ring slots the chunk
 *     overwrites (and their suffix extrema) are read once the batch that
 *     last wrote them has been reported by every producer;
 *   - a delta of a heavy hitter -- a key listed by a batch kSSlots earlier
 *     (or, for the first batches, by the query's previous pushes) -- goes to
 *     a private record: the heaviest key in registers, the others in shared
 *     memory.  A heavy hitter's work is so split over every producer instead
 *     of landing on one consumer (the paper's remedy for skew, Section 4:
 *     load moves off an overloaded worker, decided on an earlier batch);
 *   - every other delta takes its rank in its key range's run from a shared
 *     counter (one atomic per delta), the runs are laid out by an exclusive
 *     scan (the paper's two-pass placement of a batch, Section 3.1, the
 *     second pass being a plain scatter by rank), written to the batch's
 *     scratch slot by one bulk store, and each range's (begin, length) run
 *     goes to a range-major run table (the paper's threadDataIndicator);
 *   - the new tuples go to the window ring (bulk store);
 *   - after the batch's chunks: the heavy-hitter records are stored as this
 *     producer's partials (plain stores, no atomics), the bulk stores are
 *     waited for, and the producer reports the batch (release add).
 * Consumer c owns key range c for the whole launch; its groups' SUM, COUNT
 * and MIN/MAX segment extrema stay in shared memory.  For every batch, once
 * every producer reported it:
 *   - the range's run-table row arrives by one bulk load; every chunk's run
 *     is gathered by one bulk copy per chunk, in rounds of dcap deltas;
 *   - the deltas are folded into a shared table with 32-bit shared atomics
 *     (a sum as the signed sums of its 16-bit halves, exact, folded into an
 *     int64 after every round);
 *   - one warp per heavy hitter of the range sums the producers' partials;
 *   - every touched group's state is updated and its SUM, COUNT, MIN, MAX and
 *     AVG are written (a batch that replaces the window restarts every group
 *     from the batch's tuples alone); groups whose insert count reached the
 *     threshold are listed as heavy hitters of batch i + kSSlots;
 *   - the consumer reports the batch, which frees the scratch slot.
 * At the end each consumer stores its groups' extrema back as epoch-tagged
 * words (cq_tags.cuh), so later pushes of any path continue from them.
 *
 * Every wait is bounded (SArgs::wait_ns).  A wait that gives up marks the
 * query timed out, raises the launch's abort word, and every CTA leaves once
 * its own copies in flight have landed.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "cq_internal.h"
#include "cq_push_dev.cuh"
#include "cq_stream.cuh"
#include "cq_tags.cuh"
#include "cq_tma.cuh"

namespace cq {

namespace {

using namespace pushdev;
using namespace tma;

constexpr int kT = kSThreads;
constexpr int kW = kT / 32;
constexpr uint32_t kPadKey = 0x7FFFFFFFu;   /* key of padding deltas: never a group (G <= 2^31 - 1) */
constexpr uint16_t kNone = 0xFFFF;          /* no delta exchanged */
constexpr int kMaxSmSlots = 512;            /* SC_SM words reserved for %smid values */

__device__ __forceinline__ uint32_t sm_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

/* Arrivals a slot's counter must reach for batch i to be reported by all n
 * CTAs of a role: slot i mod kSSlots counts n reports of every batch
 * i' = i mod kSSlots, i' <= i. */
__device__ __forceinline__ unsigned long long slot_target(int n, int i) {
    return (unsigned long long)n * (unsigned long long)(i / kSSlots + 1);
}

__device__ __noinline__ void raise_timeout(unsigned long long *ctl, int *err, int *err_host) {
    atomicExch(ctl + SC_ABORT, 1ULL);
    atomicOr(err, 2);
    if (err_host) *(volatile int *)err_host = 2;
}

/* One thread: wait until *ctr >= target.  False once the launch is aborted,
 * or after limit_ns (then it aborts the launch and marks the query timed
 * out). */
__device__ __noinline__ bool wait_ctr(const unsigned long long *ctr, unsigned long long target,
                                      unsigned long long *ctl, int *err, int *err_host,
                                      unsigned long long limit_ns) {
    unsigned long long t0 = 0;
    for (uint32_t it = 0;; it++) {
        if (ld_acquire(ctr) >= target) return true;
        if (*(volatile unsigned long long *)(ctl + SC_ABORT)) return false;
        __nanosleep(64);
        if ((it & 15) == 15) {
            const unsigned long long now = globaltimer();
            if (!t0) {
                t0 = now;
            } else if (now - t0 > limit_ns) {
                raise_timeout(ctl, err, err_host);
                return false;
            }
        }
    }
}

/* Producer shared memory: barriers, the heavy-hitter hash and records, two
 * input sets (keys, values and, for batches whose old tuples leave, ring
 * keys, ring values and suffix extrema pairs), the per-tuple ranks, the
 * range counts and offsets, and the staged deltas of a chunk. */
struct PLayout {
    int64_t bars, hkey, hidx, hlist, hcnt, hw, h64, in, arr, set, rank, cnt, off, stage, end;
    __host__ __device__ PLayout(int Smax, int R, bool ring, int ds) {
        bars = 0;
        hkey = 64;
        hidx = hkey + kHotSlots * 4;
        hlist = hidx + kHotSlots * 2;
        hcnt = hlist + kMaxHot * 4;
        hw = hcnt + kMaxHot * 4;
        h64 = hw + (int64_t)A_NUM * kMaxHot * 4;
        in = h64 + kMaxHot * 8;
        arr = pad16((int64_t)Smax * 4);
        set = arr * (ring ? (ds == 16 ? 6 : 4) : 2);
        rank = in + 2 * set;
        cnt = rank + pad16((int64_t)Smax * 2 * (ring ? 2 : 1));
        off = cnt + pad16((int64_t)(R + 1) * 4);
        stage = off + pad16((int64_t)(R + 1) * 4);
        end = stage + ((int64_t)(ring ? 2 : 1) * Smax + R + 2) * ds;
    }
};

/* Consumer shared memory: barriers, the batch's heavy-hitter keys, the run
 * table row, the fold table, the resident per-group state and the gathered
 * deltas. */
struct CLayout {
    int64_t bars, hl, pairs, tw, t64, ssum, scnt, sext, dstage, end;
    __host__ __device__ CLayout(int tcap, int Cpad, int dcap, int ds, bool minmax) {
        bars = 0;
        hl = 64;
        pairs = hl + kMaxHot * 4;
        tw = pairs + (int64_t)Cpad * 8;
        t64 = tw + pad16((int64_t)A_NUM * tcap * 4);
        ssum = t64 + pad16((int64_t)tcap * 8);
        scnt = ssum + pad16((int64_t)tcap * 8);
        sext = scnt + pad16((int64_t)tcap * 4);
        dstage = sext + (minmax ? pad16((int64_t)4 * tcap * 4) : 0);
        end = dstage + (int64_t)dcap * ds;
    }
};

/* Exclusive scan of the n counts, each rounded up to even, into off[0 .. n]
 * (off[n] = total); returns the total.  All threads of the CTA. */
__device__ __noinline__ uint32_t scan_even(const uint32_t *cnt, uint32_t *off, int n) {
    __shared__ uint32_t wsum[kW];
    __shared__ uint32_t tot;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + kT - 1) / kT;
    const int b0 = tid * per;
    uint32_t s = 0;
    for (int j = 0; j < per; j++)
        if (b0 + j < n) s += (cnt[b0 + j] + 1u) & ~1u;
    uint32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < kW ? wsum[lane] : 0;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kW) wsum[lane] = wi - w;
        if (lane == kW - 1) tot = wi;
    }
    __syncthreads();
    uint32_t run = wsum[warp] + incl - s;
    for (int j = 0; j < per; j++)
        if (b0 + j < n) {
            off[b0 + j] = run;
            run += (cnt[b0 + j] + 1u) & ~1u;
        }
    const uint32_t total = tot;
    if (tid == 0) off[n] = total;
    __syncthreads();
    return total;
}

/* Exclusive scan of the .y fields of p[0, n) in place; returns the total. */
__device__ __noinline__ uint32_t scan_pairs(uint2 *p, int n) {
    __shared__ uint32_t wsum[kW];
    __shared__ uint32_t tot;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + kT - 1) / kT;
    const int b0 = tid * per;
    uint32_t s = 0;
    for (int j = 0; j < per; j++)
        if (b0 + j < n) s += p[b0 + j].y;
    uint32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < kW ? wsum[lane] : 0;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kW) wsum[lane] = wi - w;
        if (lane == kW - 1) tot = wi;
    }
    __syncthreads();
    uint32_t run = wsum[warp] + incl - s;
    for (int j = 0; j < per; j++)
        if (b0 + j < n) {
            const uint32_t x = p[b0 + j].y;
            p[b0 + j].y = run;
            run += x;
        }
    const uint32_t total = tot;
    __syncthreads();
    return total;
}

/* The heavy-hitter list a batch privatises: batches i < kSSlots take the
 * query's list, later ones the list batch i - kSSlots found.  Fills the
 * tier counts; entry h is tier0[h] for h < n1, else tier1[h - n1]. */
struct HotList {
    const int32_t *keys, *cnts;   /* 2 tiers of kMaxHot */
    int n1, n_hot;
};

__device__ __forceinline__ HotList hot_list_of(const SArgs &a, int i) {
    HotList L;
    const int *n;
    if (i < kSSlots) {
        L.keys = a.q_hot;
        L.cnts = a.q_hot_cnt;
        n = a.q_hot_n;
    } else {
        const int s = i % kSListSlots;
        L.keys = a.lists + (int64_t)s * 2 * kMaxHot;
        L.cnts = a.list_cnt + (int64_t)s * 2 * kMaxHot;
        n = a.list_n + 2 * (int64_t)i;
    }
    const int cap = a.hot_cap;
    const int t0 = __ldcg(n), t1 = __ldcg(n + 1);
    L.n1 = cap > 0 ? min(t0, cap) : 0;
    L.n_hot = cap > 0 ? L.n1 + min(t1, cap - L.n1) : 0;
    return L;
}

__device__ __forceinline__ int hot_entry(const HotList &L, int h) {
    return h < L.n1 ? h : kMaxHot + (h - L.n1);
}

/* Runtime-flag forms of the private heavy-hitter record updates. */
__device__ __forceinline__ void rec_ins(const Acc &r, int h, int32_t v, bool minmax) {
    atomicAdd(r.f(A_LO, h), v & 0xFFFF);
    atomicAdd(r.f(A_HI, h), v >> 16);
    atomicAdd(r.f(A_INS, h), 1);
    if (minmax) {
        if (v < *(volatile int32_t *)r.f(A_IMIN, h)) atomicMin(r.f(A_IMIN, h), v);
        if (v > *(volatile int32_t *)r.f(A_IMAX, h)) atomicMax(r.f(A_IMAX, h), v);
    }
}

__device__ __forceinline__ void rec_ret(const Acc &r, int h, int32_t v, int32_t smin, int32_t smax) {
    atomicAdd(r.f(A_LO, h), -(v & 0xFFFF));
    atomicAdd(r.f(A_HI, h), -(v >> 16));
    atomicAdd(r.f(A_RET, h), 1);
    if (smin != INT32_MIN || smax != INT32_MAX) {
        if (smin > *(volatile int32_t *)r.f(A_FRAISE, h)) atomicMax(r.f(A_FRAISE, h), smin);
        if (smax < *(volatile int32_t *)r.f(A_FLOWER, h)) atomicMin(r.f(A_FLOWER, h), smax);
    }
}

/* Fold-table updates of a consumer: its groups see few deltas each (heavy
 * hitters are privatised by the producers), so the extrema are updated
 * unconditionally. */
__device__ __forceinline__ void tab_ins(const Acc &t, int l, int32_t v, bool minmax) {
    atomicAdd(t.f(A_LO, l), v & 0xFFFF);
    atomicAdd(t.f(A_HI, l), v >> 16);
    atomicAdd(t.f(A_INS, l), 1);
    if (minmax) {
        atomicMin(t.f(A_IMIN, l), v);
        atomicMax(t.f(A_IMAX, l), v);
    }
}

__device__ __forceinline__ void tab_ret(const Acc &t, int l, int32_t v, int32_t smin, int32_t smax) {
    atomicAdd(t.f(A_LO, l), -(v & 0xFFFF));
    atomicAdd(t.f(A_HI, l), -(v >> 16));
    atomicAdd(t.f(A_RET, l), 1);
    if (smin != INT32_MIN || smax != INT32_MAX) {
        atomicMax(t.f(A_FRAISE, l), smin);
        atomicMin(t.f(A_FLOWER, l), smax);
    }
}

/* ------------------------------------------------------------------------ */
/* producer                                                                  */
/* ------------------------------------------------------------------------ */

/* Position of a producer in the launch's flat list of its chunks: chunk c of
 * batch i (c = aid, aid + nA, ...), i = nb when the list is exhausted. */
struct Item {
    int i, c;
};

__device__ __forceinline__ Item first_item(const SArgs &a, int aid, int i) {
    while (i < a.nb && a.b[i].C <= aid) i++;
    return Item{i, aid};
}

__device__ __forceinline__ Item next_item(const SArgs &a, int aid, Item it) {
    const int c = it.c + a.nA;
    if (c < a.b[it.i].C) return Item{it.i, c};
    return first_item(a, aid, it.i + 1);
}

/* Phase stamp k of CTA `who` (producers 0 .. nA-1, consumers nA ..) for
 * batch i, when tracing. */
__device__ __forceinline__ void stamp(const SArgs &a, int who, int i, int k) {
    if (a.trace && threadIdx.x == 0) a.trace[((int64_t)who * a.nb + i) * 12 + k] = globaltimer();
}

template <int DS>
__device__ __forceinline__ void producer(const SArgs &a, const int aid, unsigned char *smem) {
    typedef typename std::conditional<DS == 16, uint4, uint2>::type Delta;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool ring_any = a.ring_any != 0;
    const PLayout L(a.Smax, a.R, ring_any, DS);
    unsigned long long *bars = (unsigned long long *)(smem + L.bars);   /* [0..1] keys/values of a set, [2..3] its ring */
    int32_t *hkey = (int32_t *)(smem + L.hkey);
    int16_t *hidx = (int16_t *)(smem + L.hidx);
    int32_t *hlist = (int32_t *)(smem + L.hlist);
    int32_t *hcnt = (int32_t *)(smem + L.hcnt);
    const Acc rec{(int32_t *)(smem + L.hw), (long long *)(smem + L.h64), kMaxHot};
    uint16_t *rank = (uint16_t *)(smem + L.rank);
    uint32_t *cnt = (uint32_t *)(smem + L.cnt);
    uint32_t *off = (uint32_t *)(smem + L.off);
    Delta *stage_s = (Delta *)(smem + L.stage);
    __shared__ int s_len4[2];        /* bulk-loaded prefix of each input set's chunk (0: none pending) */
    __shared__ int s_nhot, s_top, s_stop;
    __shared__ long long wtop_sum[kW];
    __shared__ int32_t wtop_i[kW][6];
    __shared__ SBatch s_b;
    const int R = a.R;
    const uint32_t M = a.M;
    const int64_t G = a.G, W = a.W;
    const bool minmax = a.minmax != 0;

    auto set_arr = [&](int set, int arr) -> int32_t * {
        return (int32_t *)(smem + L.in + (int64_t)set * L.set + (int64_t)arr * L.arr);
    };
    /* bulk loads of an item's keys and values (aligned batches only); one thread */
    auto issue_inputs = [&](int set, Item it) {
        s_len4[set] = 0;
        if (it.i >= a.nb) return;
        const SBatch &b = a.b[it.i];
        if (!(b.flags & SB_ALIGNED)) return;
        const int64_t cbeg = (int64_t)it.c * b.S;
        const int len = (int)min((int64_t)b.S, (int64_t)b.n - cbeg);
        const int len4 = len & ~3;
        if (len4 == 0) return;
        mbar_expect(&bars[set], 8u * (uint32_t)len4);
        tma_load(set_arr(set, 0), b.keys + cbeg, 4u * len4, &bars[set]);
        tma_load(set_arr(set, 1), b.vals + cbeg, 4u * len4, &bars[set]);
        s_len4[set] = len4;
    };

    if (tid == 0) {
        for (int j = 0; j < 4; j++) mbar_init(&bars[j], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t par[4] = {0, 0, 0, 0};
    Item issue = first_item(a, aid, 0);
    if (tid == 0) {
        s_stop = 0;
        for (int s = 0; s < 2; s++) {
            issue_inputs(s, issue);
            if (issue.i < a.nb) issue = next_item(a, aid, issue);
        }
    } else {
        for (int s = 0; s < 2 && issue.i < a.nb; s++) issue = next_item(a, aid, issue);
    }
    int set = 0;
    bool stop = false;

    for (int i = 0; i < a.nb && !stop; i++) {
        const int slot = i % kSSlots;
        /* the slot's previous batch (i - kSSlots) has been folded by every
           consumer: its scratch is free and its heavy-hitter list is final */
        if (tid == 0) {
            if (i >= kSSlots)
                stop = !wait_ctr(a.ctl + SC_B + slot, slot_target(a.nB, i - kSSlots), a.ctl, a.err, a.err_host,
                                 a.wait_ns);
            s_stop = stop;
            s_b = a.b[i];
            if (a.stamp_begin && aid < s_b.C) atomicMin(a.stamp_begin + i, globaltimer());
        }
        __syncthreads();
        if (s_stop) break;
        stamp(a, aid, i, 0);
        const SBatch &B = s_b;
        const bool mine = aid < B.C;
        const bool ring = (B.flags & SB_RING) != 0;
        const bool front = DS == 16 && (B.flags & SB_FRONT) != 0;
        long long r_sum = 0;
        int32_t r_ins = 0, r_ret = 0;
        int32_t r_imin = INT32_MAX, r_imax = INT32_MIN, r_fra = INT32_MIN, r_flo = INT32_MAX;
        if (mine) {
            /* the batch's heavy hitters: list, hash, the heaviest one */
            const HotList HL = hot_list_of(a, i);
            const int n_hot = HL.n_hot;
            for (int s = tid; s < kHotSlots; s += kT) hkey[s] = -1;
            __syncthreads();
            for (int h = tid; h < n_hot; h += kT) {
                const int e = hot_entry(HL, h);
                const int32_t k = __ldcg(HL.keys + e);
                hlist[h] = k;
                hcnt[h] = __ldcg(HL.cnts + e);
                uint32_t s = hot_hash(k);
                for (int probe = 0; probe < kHotSlots; probe++) {
                    const int prev = atomicCAS(&hkey[s], -1, k);
                    if (prev == -1 || prev == k) {
                        hidx[s] = (int16_t)h;
                        break;
                    }
                    s = (s + 1) & (kHotSlots - 1);
                }
                acc_init(rec, h);
            }
            __syncthreads();
            if (warp == 0) {
                int best = -1, bestc = -1;
                for (int h = lane; h < n_hot; h += 32) {
                    const int c = hcnt[h];
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
                if (lane == 0) {
                    s_top = best;
                    s_nhot = n_hot;
                }
            }
            __syncthreads();
        }
        const int n_hot = mine ? s_nhot : 0;
        const int top = mine ? s_top : -1;
        stamp(a, aid, i, 1);
        int nch = 0;

        for (int c = aid; c < B.C && !stop; c += a.nA) {
            const int64_t cbeg = (int64_t)c * B.S;
            const int len = (int)min((int64_t)B.S, (int64_t)B.n - cbeg);
            int64_t s064 = (int64_t)B.slot0 + cbeg;   /* ring slot of the chunk's first tuple */
            if (s064 >= W) s064 -= W;
            const int s0 = (int)s064;
            const int len4 = s_len4[set];
            int32_t *sk = set_arr(set, 0), *sv = set_arr(set, 1);
            int32_t *srk = set_arr(set, 2), *srv = set_arr(set, 3);
            int2 *ss = (int2 *)set_arr(set, 4);
            for (int r = tid; r <= R; r += kT) cnt[r] = 0;
            /* ring slots: only after the batch that last wrote them is out */
            if (ring) {
                if (tid == 0 && B.ring_dep >= 0) {
                    const bool ok = wait_ctr(a.ctl + SC_A + B.ring_dep % kSSlots, slot_target(a.nA, B.ring_dep),
                                             a.ctl, a.err, a.err_host, a.wait_ns);
                    if (!ok) s_stop = 1;
                    fence_async_global();
                }
                __syncthreads();
                if (s_stop) {
                    stop = true;
                    break;
                }
                if (tid == 0 && len4 > 0) {
                    const uint32_t bytes = 8u * len4 + (front ? 8u * len4 : 0u);
                    mbar_expect(&bars[2 + set], bytes);
                    const int64_t n1 = min((int64_t)len4, W - s064);
                    tma_load(srk, a.ring_k + s064, 4u * (uint32_t)n1, &bars[2 + set]);
                    tma_load(srv, a.ring_v + s064, 4u * (uint32_t)n1, &bars[2 + set]);
                    if (front) tma_load(ss, a.suf + s064, 8u * (uint32_t)n1, &bars[2 + set]);
                    if (len4 > n1) {
                        const uint32_t n2 = (uint32_t)(len4 - n1);
                        tma_load(srk + n1, a.ring_k, 4u * n2, &bars[2 + set]);
                        tma_load(srv + n1, a.ring_v, 4u * n2, &bars[2 + set]);
                        if (front) tma_load(ss + n1, a.suf, 8u * n2, &bars[2 + set]);
                    }
                }
            }
            /* unaligned batches and ragged tails: per-element asynchronous copies */
            bool any_cp = false;
            for (int j = len4 + tid; j < len; j += kT) {
                any_cp = true;
                cp_async(sk + j, B.keys + cbeg + j);
                cp_async(sv + j, B.vals + cbeg + j);
                if (ring) {
                    int64_t sl = s064 + j;
                    if (sl >= W) sl -= W;
                    cp_async(srk + j, a.ring_k + sl);
                    cp_async(srv + j, a.ring_v + sl);
                    if (front) cp_async(ss + j, a.suf + sl);
                }
            }
            if (any_cp) cp_async_wait_all();
            if (tid == 0 && len4 > 0) {
                bool ok = mbar_wait(&bars[set], par[set], a.wait_ns);
                par[set] ^= 1u;
                if (ring) {
                    ok = mbar_wait(&bars[2 + set], par[2 + set], a.wait_ns) && ok;
                    par[2 + set] ^= 1u;
                }
                if (!ok) {
                    raise_timeout(a.ctl, a.err, a.err_host);
                    s_stop = 1;
                }
            }
            __syncthreads();
            if (tid == 0) s_len4[set] = 0;   /* consumed (every thread has read len4) */
            if (s_stop) {
                stop = true;
                break;
            }
            stamp(a, aid, i, nch == 0 ? 2 : 7);
            /* pass 1: heavy hitters into the private records (the heaviest in
               registers), the rest ranked within their key range's run */
            bool bad = false;
            const uint32_t Wu = (uint32_t)W, hmod = (uint32_t)B.hmod;
            const int32_t old_len = B.old_len, fa = B.fa, fb = B.fb;
            for (int j = tid; j < len; j += kT) {
                const int32_t k = sk[j];
                uint16_t ri = kNone;
                if ((uint32_t)k >= (uint32_t)G) {
                    bad = true;
                } else {
                    const int h = n_hot ? hot_find(hkey, hidx, k) : -1;
                    if (h >= 0 && h == top) {
                        const int32_t v = sv[j];
                        r_sum += v;
                        r_ins++;
                        r_imin = min(r_imin, v);
                        r_imax = max(r_imax, v);
                    } else if (h >= 0) {
                        rec_ins(rec, h, sv[j], minmax);
                    } else {
                        ri = (uint16_t)atomicAdd(&cnt[__umulhi((uint32_t)k, M)], 1u);
                    }
                }
                rank[j] = ri;
                if (ring) {
                    uint32_t sl = (uint32_t)s0 + (uint32_t)j;
                    if (sl >= Wu) sl -= Wu;
                    int32_t rel = (int32_t)sl - (int32_t)hmod;
                    if (rel < 0) rel += (int32_t)Wu;
                    uint16_t rr = kNone;
                    if (rel < old_len) {
                        const int32_t ok = srk[j];
                        if ((uint32_t)ok < (uint32_t)G) {
                            const bool fr = front && rel >= fa && rel < fb;
                            const int h = n_hot ? hot_find(hkey, hidx, ok) : -1;
                            if (h >= 0 && h == top) {
                                r_sum -= srv[j];
                                r_ret++;
                                if (fr) {
                                    r_fra = max(r_fra, ss[j].x);
                                    r_flo = min(r_flo, ss[j].y);
                                }
                            } else if (h >= 0) {
                                rec_ret(rec, h, srv[j], fr ? ss[j].x : INT32_MIN, fr ? ss[j].y : INT32_MAX);
                            } else {
                                rr = (uint16_t)atomicAdd(&cnt[__umulhi((uint32_t)ok, M)], 1u);
                            }
                        }
                    }
                    rank[a.Smax + j] = rr;
                }
            }
            if (bad) {
                atomicOr(a.err, 1);
                if (a.err_host) *(volatile int *)a.err_host = 1;
            }
            /* the previous chunk's bulk stores must have read the staging area */
            if (tid == 0) tma_wait_read();
            __syncthreads();
            stamp(a, aid, i, nch == 0 ? 3 : 8);
            for (int h = tid; h < n_hot; h += kT) acc_fold(rec, h);
            const uint32_t total = scan_even(cnt, off, R);
            {   /* each range's run in this chunk: (begin, padded length), range-major */
                uint2 *row = a.pairs + (int64_t)slot * a.pairs_slot + c;
                for (int r = tid; r < R; r += kT)
                    row[(int64_t)r * a.Cpad] = make_uint2(off[r], (cnt[r] + 1u) & ~1u);
            }
            /* pass 2: place the exchanged deltas by rank */
            for (int j = tid; j < len; j += kT) {
                const uint16_t ri = rank[j];
                if (ri != kNone) {
                    const int32_t k = sk[j];
                    stage_s[off[__umulhi((uint32_t)k, M)] + ri] =
                        DeltaIO<Delta>::make((uint32_t)k, sv[j], INT32_MIN, INT32_MAX);
                }
                if (ring) {
                    const uint16_t rr = rank[a.Smax + j];
                    if (rr != kNone) {
                        const int32_t ok = srk[j];
                        bool fr = false;
                        if (front) {
                            uint32_t sl = (uint32_t)s0 + (uint32_t)j;
                            if (sl >= Wu) sl -= Wu;
                            int32_t rel = (int32_t)sl - (int32_t)hmod;
                            if (rel < 0) rel += (int32_t)Wu;
                            fr = rel >= fa && rel < fb;
                        }
                        stage_s[off[__umulhi((uint32_t)ok, M)] + rr] = DeltaIO<Delta>::make(
                            (uint32_t)ok | kRetract, srv[j], fr ? ss[j].x : INT32_MIN, fr ? ss[j].y : INT32_MAX);
                    }
                }
            }
            for (int r = tid; r < R; r += kT)
                if (cnt[r] & 1u) stage_s[off[r] + cnt[r]] = DeltaIO<Delta>::make(kPadKey, 0, INT32_MIN, INT32_MAX);
            __syncthreads();
            if (tid == 0 && total > 0) {
                fence_async_smem();
                tma_store((Delta *)a.stage + (int64_t)slot * a.stage_slot + (int64_t)c * a.stride, stage_s,
                          total * (uint32_t)DS);
                tma_commit();
            }
            if (nch == 0) stamp(a, aid, i, 4);
            /* the new tuples go to the ring once the batch that last wrote
               these slots is out (already waited for when the ring was read) */
            if (!ring && B.ring_dep >= 0) {
                if (tid == 0) {
                    const bool ok = wait_ctr(a.ctl + SC_A + B.ring_dep % kSSlots, slot_target(a.nA, B.ring_dep),
                                             a.ctl, a.err, a.err_host, a.wait_ns);
                    if (!ok) s_stop = 1;
                    fence_async_global();
                }
                __syncthreads();
                if (s_stop) {
                    stop = true;
                    break;
                }
            }
            if (nch == 0) stamp(a, aid, i, 5);
            if (tid == 0 && len4 > 0) {
                fence_async_smem();
                const int64_t n1 = min((int64_t)len4, W - s064);
                tma_store(a.ring_k + s064, sk, 4u * (uint32_t)n1);
                tma_store(a.ring_v + s064, sv, 4u * (uint32_t)n1);
                if (len4 > n1) {
                    tma_store(a.ring_k, sk + n1, 4u * (uint32_t)(len4 - n1));
                    tma_store(a.ring_v, sv + n1, 4u * (uint32_t)(len4 - n1));
                }
                tma_commit();
            }
            for (int j = len4 + tid; j < len; j += kT) {
                int64_t sl = s064 + j;
                if (sl >= W) sl -= W;
                a.ring_k[sl] = sk[j];
                a.ring_v[sl] = sv[j];
            }
            /* this input set is free once the ring stores have read it: it
               takes the item two ahead */
            if (tid == 0) {
                tma_wait_read();
                issue_inputs(set, issue);
            }
            if (issue.i < a.nb) issue = next_item(a, aid, issue);
            set ^= 1;
            __syncthreads();
            stamp(a, aid, i, nch == 0 ? 6 : 9);
            nch++;
        }
        if (stop) break;
        if (mine) {
            /* the batch's heavy-hitter partials of this producer */
            if (top >= 0) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    r_sum += __shfl_xor_sync(kFull, r_sum, o);
                    r_ins += __shfl_xor_sync(kFull, r_ins, o);
                    r_ret += __shfl_xor_sync(kFull, r_ret, o);
                    r_imin = min(r_imin, __shfl_xor_sync(kFull, r_imin, o));
                    r_imax = max(r_imax, __shfl_xor_sync(kFull, r_imax, o));
                    r_fra = max(r_fra, __shfl_xor_sync(kFull, r_fra, o));
                    r_flo = min(r_flo, __shfl_xor_sync(kFull, r_flo, o));
                }
                if (lane == 0) {
                    wtop_sum[warp] = r_sum;
                    wtop_i[warp][0] = r_ins;
                    wtop_i[warp][1] = r_ret;
                    wtop_i[warp][2] = r_imin;
                    wtop_i[warp][3] = r_imax;
                    wtop_i[warp][4] = r_fra;
                    wtop_i[warp][5] = r_flo;
                }
            }
            __syncthreads();
            HotAcc *dst = a.hotpart + ((int64_t)slot * a.nA + aid) * kMaxHot;
            for (int h = tid; h < n_hot; h += kT) {
                HotAcc r;
                r.sum = rec.acc64[h];
                r.ins = *rec.f(A_INS, h);
                r.ret = *rec.f(A_RET, h);
                r.imin = *rec.f(A_IMIN, h);
                r.imax = *rec.f(A_IMAX, h);
                r.fraise = *rec.f(A_FRAISE, h);
                r.flower = *rec.f(A_FLOWER, h);
                if (h == top) {
                    for (int w = 0; w < kW; w++) {
                        r.sum += wtop_sum[w];
                        r.ins += wtop_i[w][0];
                        r.ret += wtop_i[w][1];
                        r.imin = min(r.imin, wtop_i[w][2]);
                        r.imax = max(r.imax, wtop_i[w][3]);
                        r.fraise = max(r.fraise, wtop_i[w][4]);
                        r.flower = min(r.flower, wtop_i[w][5]);
                    }
                }
                dst[h] = r;
            }
        }
        /* every store of the batch (runs, ring, run table, partials) is out
           before the batch is reported */
        if (tid == 0) {
            tma_wait_all();
            fence_async_global();
        }
        __syncthreads();
        stamp(a, aid, i, 10);
        if (tid == 0 && !(aid == 0 && i == a.stall_batch)) red_release(a.ctl + SC_A + slot, 1ULL);
        stamp(a, aid, i, 11);
    }
    /* leave only once the copies this CTA requested have landed */
    if (tid == 0) {
        for (int s = 0; s < 2; s++)
            if (s_len4[s] > 0) {
                mbar_wait(&bars[s], par[s], a.wait_ns);
                par[s] ^= 1u;
            }
        tma_wait_all();
    }
    __syncthreads();
}

/* ------------------------------------------------------------------------ */
/* consumer                                                                  */
/* ------------------------------------------------------------------------ */

template <int DS>
__device__ __forceinline__ void consumer(const SArgs &a, const int bid, unsigned char *smem) {
    typedef typename std::conditional<DS == 16, uint4, uint2>::type Delta;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool minmax = a.minmax != 0, avg = a.avg != 0;
    const CLayout L(a.tcap, a.Cpad, a.dcap, DS, minmax);
    unsigned long long *bars = (unsigned long long *)(smem + L.bars);   /* [0] run-table row, [1] gather */
    int32_t *hl = (int32_t *)(smem + L.hl);
    uint2 *pairs = (uint2 *)(smem + L.pairs);
    const Acc tab{(int32_t *)(smem + L.tw), (long long *)(smem + L.t64), a.tcap};
    long long *st_sum = (long long *)(smem + L.ssum);
    int32_t *st_cnt = (int32_t *)(smem + L.scnt);
    int32_t *st_bmin = (int32_t *)(smem + L.sext);
    int32_t *st_bmax = st_bmin + a.tcap;
    int32_t *st_fmin = st_bmax + a.tcap;
    int32_t *st_fmax = st_fmin + a.tcap;
    Delta *dstage = (Delta *)(smem + L.dstage);
    __shared__ int s_stop, s_nhot, s_C;
    __shared__ uint32_t s_flags, s_thr, s_gthr;
    const bool has_range = bid < a.R;
    const int64_t lo = has_range ? stream_range_lo((uint32_t)bid, a.M, a.G) : 0;
    const int64_t hi = has_range ? stream_range_lo((uint32_t)bid + 1, a.M, a.G) : 0;
    const int rng = (int)(hi - lo);   /* <= tcap (the host sized tcap from the same bounds) */

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_stop = 0;
    }
    /* the range's state, resident for the whole launch */
    for (int l = tid; l < rng; l += kT) {
        const int64_t g = lo + l;
        st_sum[l] = (long long)a.sum[g];
        st_cnt[l] = a.cnt[g];
        if (minmax) {
            st_bmin[l] = untag_dn(a.bmin[g], a.epoch0, INT32_MAX);
            st_bmax[l] = untag_up(a.bmax[g], a.epoch0, INT32_MIN);
            st_fmin[l] = untag_up(a.fmin[g], a.epoch0, INT32_MAX);
            st_fmax[l] = untag_dn(a.fmax[g], a.epoch0, INT32_MIN);
        }
    }
    __syncthreads();
    uint32_t ppar = 0, gpar = 0;
    bool stop = false;
    for (int i = 0; i < a.nb && !stop; i++) {
        const int slot = i % kSSlots;
        if (tid == 0) {
            stop = !wait_ctr(a.ctl + SC_A + slot, slot_target(a.nA, i), a.ctl, a.err, a.err_host, a.wait_ns);
            fence_async_global();
            s_stop = stop;
            const SBatch &b = a.b[i];
            s_C = b.C;
            s_flags = (uint32_t)b.flags;
            s_thr = b.hot_threshold;
            s_gthr = b.hot_gthr;
            if (!stop && has_range && b.C > 0) {
                const int Cp = (b.C + 1) & ~1;
                mbar_expect(&bars[0], 8u * (uint32_t)Cp);
                tma_load(pairs, a.pairs + (int64_t)slot * a.pairs_slot + (int64_t)bid * a.Cpad, 8u * (uint32_t)Cp,
                         &bars[0]);
            }
        }
        __syncthreads();
        if (s_stop) {
            stop = true;
            break;
        }
        const int me = a.nA + bid;
        stamp(a, me, i, 0);
        if (has_range) {
            const int C = s_C;
            const uint32_t flags = s_flags;
            const bool replace = (flags & SB_REPLACE) != 0;
            /* the batch's heavy-hitter keys (their partials are merged below) */
            const HotList HL = hot_list_of(a, i);
            for (int h = tid; h < HL.n_hot; h += kT) hl[h] = __ldcg(HL.keys + hot_entry(HL, h));
            if (tid == 0) s_nhot = HL.n_hot;
            for (int l = tid; l < rng; l += kT) acc_init(tab, l);
            if (C > 0) {
                if (tid == 0 && !mbar_wait(&bars[0], ppar, a.wait_ns)) {
                    raise_timeout(a.ctl, a.err, a.err_host);
                    s_stop = 1;
                }
                ppar ^= 1u;
            }
            __syncthreads();
            if (s_stop) {
                stop = true;
                break;
            }
            stamp(a, me, i, 1);
            const uint32_t total = C > 0 ? scan_pairs(pairs, C) : 0u;
            stamp(a, me, i, 2);
            const Delta *stage = (const Delta *)a.stage + (int64_t)slot * a.stage_slot;
            for (uint32_t b0 = 0; b0 < total && !stop; b0 += (uint32_t)a.dcap) {
                const uint32_t b1 = min(total, b0 + (uint32_t)a.dcap);
                if (tid == 0) mbar_expect(&bars[1], (b1 - b0) * (uint32_t)DS);
                __syncthreads();
                for (int c = tid; c < C; c += kT) {
                    const uint32_t s0 = pairs[c].y, s1 = c + 1 < C ? pairs[c + 1].y : total;
                    const uint32_t x0 = max(s0, b0), x1 = min(s1, b1);
                    if (x0 < x1)
                        tma_load(dstage + (x0 - b0), stage + (int64_t)c * a.stride + pairs[c].x + (x0 - s0),
                                 (x1 - x0) * (uint32_t)DS, &bars[1]);
                }
                if (tid == 0 && !mbar_wait(&bars[1], gpar, a.wait_ns)) {
                    raise_timeout(a.ctl, a.err, a.err_host);
                    s_stop = 1;
                }
                gpar ^= 1u;
                __syncthreads();
                if (s_stop) {
                    stop = true;
                    break;
                }
                if (b0 == 0) stamp(a, me, i, 3);
                for (uint32_t j = tid; j < b1 - b0; j += kT) {
                    uint32_t kf;
                    int32_t dv, smin, smax;
                    DeltaIO<Delta>::get(dstage[j], kf, dv, smin, smax);
                    const int64_t l = (int64_t)(kf & kKeyMask) - lo;
                    if (l < 0 || l >= rng) continue;   /* padding deltas */
                    if (kf & kRetract) tab_ret(tab, (int)l, dv, smin, smax);
                    else tab_ins(tab, (int)l, dv, minmax);
                }
                __syncthreads();
                for (int l = tid; l < rng; l += kT) acc_fold(tab, l);
                __syncthreads();
            }
            if (stop) break;
            stamp(a, me, i, 4);
            /* heavy hitters of the range: a warp sums a key's partials over
               the producers that had chunks of the batch */
            const int n_hot = s_nhot;
            const int nparts = min(a.nA, C);
            const HotAcc *parts = a.hotpart + (int64_t)slot * a.nA * kMaxHot;
            for (int h = warp; h < n_hot; h += kW) {
                const int32_t key = hl[h];
                if ((int64_t)key < lo || (int64_t)key >= hi) continue;
                long long hs = 0;
                int32_t ins = 0, ret = 0, imin = INT32_MAX, imax = INT32_MIN, fra = INT32_MIN, flo = INT32_MAX;
                for (int p = lane; p < nparts; p += 32) {
                    const HotAcc *r = parts + (int64_t)p * kMaxHot + h;
                    hs += __ldcg(&r->sum);
                    ins += __ldcg(&r->ins);
                    ret += __ldcg(&r->ret);
                    imin = min(imin, __ldcg(&r->imin));
                    imax = max(imax, __ldcg(&r->imax));
                    fra = max(fra, __ldcg(&r->fraise));
                    flo = min(flo, __ldcg(&r->flower));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    hs += __shfl_xor_sync(kFull, hs, o);
                    ins += __shfl_xor_sync(kFull, ins, o);
                    ret += __shfl_xor_sync(kFull, ret, o);
                    imin = min(imin, __shfl_xor_sync(kFull, imin, o));
                    imax = max(imax, __shfl_xor_sync(kFull, imax, o));
                    fra = max(fra, __shfl_xor_sync(kFull, fra, o));
                    flo = min(flo, __shfl_xor_sync(kFull, flo, o));
                }
                if (lane == 0) {
                    const int l = (int)(key - lo);
                    tab.acc64[l] += hs;
                    *tab.f(A_INS, l) += ins;
                    *tab.f(A_RET, l) += ret;
                    *tab.f(A_IMIN, l) = min(*tab.f(A_IMIN, l), imin);
                    *tab.f(A_IMAX, l) = max(*tab.f(A_IMAX, l), imax);
                    *tab.f(A_FRAISE, l) = max(*tab.f(A_FRAISE, l), fra);
                    *tab.f(A_FLOWER, l) = min(*tab.f(A_FLOWER, l), flo);
                }
            }
            __syncthreads();
            stamp(a, me, i, 5);
            /* finalise: state, results of touched groups, next heavy hitters */
            const uint32_t thr = s_thr, gthr = s_gthr;
            const int ls = (i + kSSlots) % kSListSlots;
            int *next_n = a.list_n + 2 * (int64_t)(i + kSSlots);
            for (int l = tid; l < rng; l += kT) {
                const int32_t ins = *tab.f(A_INS, l), ret = *tab.f(A_RET, l);
                const int32_t oc = st_cnt[l];
                if (ins + ret == 0 && !(replace && oc > 0)) continue;
                const int64_t g = lo + l;
                const long long s = (replace ? 0LL : st_sum[l]) + tab.acc64[l];
                const int32_t cn = (replace ? 0 : oc) + (ins - ret);
                st_sum[l] = s;
                st_cnt[l] = cn;
                a.sum[g] = (unsigned long long)s;
                a.cnt[g] = cn;
                if (minmax) {
                    int32_t blo = replace ? INT32_MAX : st_bmin[l];
                    int32_t bhi = replace ? INT32_MIN : st_bmax[l];
                    int32_t flo = replace ? INT32_MAX : st_fmin[l];
                    int32_t fhi = replace ? INT32_MIN : st_fmax[l];
                    if (ins) {
                        blo = min(blo, *tab.f(A_IMIN, l));
                        bhi = max(bhi, *tab.f(A_IMAX, l));
                    }
                    /* a front tuple leaving raises the front minimum to the
                       least of the group's later front tuples (lowers the
                       maximum likewise); identity when none left */
                    flo = max(flo, *tab.f(A_FRAISE, l));
                    fhi = min(fhi, *tab.f(A_FLOWER, l));
                    st_bmin[l] = blo;
                    st_bmax[l] = bhi;
                    st_fmin[l] = flo;
                    st_fmax[l] = fhi;
                    a.rmin[g] = cn > 0 ? min(blo, flo) : INT32_MAX;
                    a.rmax[g] = cn > 0 ? max(bhi, fhi) : INT32_MIN;
                }
                if (avg)
                    a.ravg[g] = cn > 0 ? __ddiv_rn(__ll2double_rn(s), (double)cn)
                                       : __longlong_as_double(0x7FF8000000000000LL);
                if (a.hot_cap && (uint32_t)ins >= thr) {
                    const int tier = (uint32_t)ins >= gthr ? 0 : 1;
                    const int idx = atomicAdd(next_n + tier, 1);
                    if (idx < a.hot_cap) {
                        a.lists[((int64_t)ls * 2 + tier) * kMaxHot + idx] = (int32_t)g;
                        a.list_cnt[((int64_t)ls * 2 + tier) * kMaxHot + idx] = ins;
                    }
                }
            }
            if (a.snap_sum) {
                __syncthreads();
                const int64_t base = (int64_t)i * a.G;
                for (int l = tid; l < rng; l += kT) {
                    const int64_t g = lo + l;
                    const int32_t cn = st_cnt[l];
                    const long long s = st_sum[l];
                    a.snap_sum[base + g] = s;
                    a.snap_cnt[base + g] = cn;
                    a.snap_min[base + g] = minmax && cn > 0 ? min(st_bmin[l], st_fmin[l]) : INT32_MAX;
                    a.snap_max[base + g] = minmax && cn > 0 ? max(st_bmax[l], st_fmax[l]) : INT32_MIN;
                    a.snap_avg[base + g] = avg && cn > 0 ? __ddiv_rn(__ll2double_rn(s), (double)cn)
                                                         : __longlong_as_double(0x7FF8000000000000LL);
                }
            }
        }
        __syncthreads();
        stamp(a, me, i, 6);
        if (tid == 0) {
            if (a.stamp_end && has_range) atomicMax(a.stamp_end + i, globaltimer());
            red_release(a.ctl + SC_B + slot, 1ULL);
        }
        stamp(a, me, i, 7);
    }
    /* the range's extrema back as tagged words of the last batch's epoch */
    if (!stop && minmax && a.nb > 0) {
        const uint32_t e = a.b[a.nb - 1].epoch;
        for (int l = tid; l < rng; l += kT) {
            const int64_t g = lo + l;
            a.bmin[g] = tag_dn(e, st_bmin[l]);
            a.bmax[g] = tag_up(e, st_bmax[l]);
            a.fmin[g] = tag_up(e, st_fmin[l]);
            a.fmax[g] = tag_dn(e, st_fmax[l]);
        }
    }
}

template <int DS>
__global__ void __launch_bounds__(kT, 2) stream_kernel(const __grid_constant__ SArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_role, s_id;
    if (threadIdx.x == 0) {
        const uint32_t sm = sm_id();
        int role = -1, id = -1;
        if (sm < (uint32_t)kMaxSmSlots) {
            const unsigned long long k = atomicAdd(a.ctl + SC_SM + sm, 1ULL);
            role = k == 0 ? 0 : (k == 1 ? 1 : -1);
        }
        if (role >= 0) {
            id = (int)atomicAdd(a.ctl + (role == 0 ? SC_ROLE_A : SC_ROLE_B), 1ULL);
            if (id >= (role == 0 ? a.nA : a.nB)) role = -1;
        }
        /* a CTA the roles cannot place would leave a producer or consumer
           missing: the launch is abandoned as timed out */
        if (role < 0) raise_timeout(a.ctl, a.err, a.err_host);
        s_role = role;
        s_id = id;
    }
    __syncthreads();
    if (s_role == 0) producer<DS>(a, s_id, smem);
    else if (s_role == 1) consumer<DS>(a, s_id, smem);
}

}  // namespace

int64_t stream_smem_bytes(int Smax, int R, int tcap, int Cpad, int dcap, bool ring, int ds, bool minmax) {
    const int64_t p = PLayout(Smax, R, ring, ds).end;
    const int64_t c = CLayout(tcap, Cpad, dcap, ds, minmax).end;
    const int64_t m = p > c ? p : c;
    return m <= kSSmem ? kSSmem : -1;
}

int stream_max_chunk(int R, bool ring, int ds) {
    /* bytes of the producer layout that do not scale with the chunk, then
       the bytes per tuple */
    const int64_t fixed = PLayout(0, R, ring, ds).end + 16 * 8;
    const int64_t per = 2 * 4 * (ring ? (ds == 16 ? 6 : 4) : 2) + 2 * (ring ? 2 : 1) + (int64_t)(ring ? 2 : 1) * ds;
    int64_t s = (kSSmem - fixed) / per;
    s &= ~(int64_t)3;
    if (s > kSMaxChunk) s = kSMaxChunk;
    return (int)s;
}

int stream_max_range(int Cpad, int dcap, int ds, bool minmax) {
    const int64_t fixed = CLayout(0, Cpad, dcap, ds, minmax).end + 16 * 8;
    const int64_t per = (int64_t)A_NUM * 4 + 8 + 8 + 4 + (minmax ? 16 : 0);
    const int64_t t = (kSSmem - fixed) / per;
    return t > 0 ? (int)t : 0;
}

bool stream_launchable() {
    const void *fns[2] = {(const void *)stream_kernel<8>, (const void *)stream_kernel<16>};
    for (const void *fn : fns) {
        int occ = 0;
        if (raise_dyn_smem(fn, kSSmem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kT, (size_t)kSSmem) != cudaSuccess || occ != 2) {
            cudaGetLastError();
            return false;
        }
    }
    return true;
}

cudaError_t launch_stream(const SArgs &a, int ds, cudaStream_t s) {
    const void *fn = ds == 16 ? (const void *)stream_kernel<16> : (const void *)stream_kernel<8>;
    cudaError_t e = raise_dyn_smem(fn, kSSmem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kT, (size_t)kSSmem);
    if (e != cudaSuccess) return e;
    if (occ != 2) return cudaErrorInvalidConfiguration;   /* the roles need exactly two CTAs per SM */
    SArgs args = a;
    void *params[] = {&args};
    return cudaLaunchCooperativeKernel(fn, dim3(a.nA + a.nB), dim3(kT), params, (size_t)kSSmem, s);
}

}  // namespace cq
