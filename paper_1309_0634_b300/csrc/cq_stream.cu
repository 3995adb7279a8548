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
 *     overwrites are read once the batch that
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
#include "cq_avg.cuh"
#include "cq_tags.cuh"
#include "cq_tma.cuh"

namespace cq {

namespace {

using namespace pushdev;
using namespace tma;

constexpr int kT = kSThreads;
constexpr int kW = kT / 32;
constexpr uint32_t kPadKey = kPadWord;   /* key word of padding deltas: never a group */
constexpr int kMaxSmSlots = kSSmSlots;      /* SC_SM words reserved for %smid values */

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
        __nanosleep(128);
        if ((it & 7) == 7) {
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

/* Heavy-hitter updates of a producer: the RegTop<RING>::n heaviest keys of the list
 * (by their counts in the batch that found them) are summed in each thread's
 * registers and reduced once per batch; the other, lighter, heavy hitters go
 * to the CTA's shared records by atomics, which they seldom contend for. */
template <bool RING>
struct RegTop {
    static constexpr int n = 2;   /* four measured slower: each tuple then tests four keys */
};

/* Producer shared memory: barriers, the heavy-hitter hash and records, two
 * input sets (keys, values and, for batches whose old tuples leave, ring
 * keys and ring values), the per-tuple packed ranks
 * (insert and retract), the range counts and offsets, and the staged deltas
 * of a chunk. */
struct PLayout {
    int64_t bars, hkey, hidx, hcnt, htop, hw, h64, in, arr, set, rank, cnt, off, stage, end;
    __host__ __device__ PLayout(int Smax, int R, bool ring, int ds) {
        bars = 0;
        hkey = 64;
        hidx = hkey + kHotSlots * 4;
        hcnt = hidx + kHotSlots * 2;
        htop = hcnt + kMaxHot * 4;
        hw = htop + kMaxHot * 4;
        h64 = hw + (int64_t)A_NUM * kMaxHot * 4;
        in = h64 + kMaxHot * 8;
        arr = pad16((int64_t)Smax * 4);
        set = arr * (ring ? 4 : 2);
        rank = in + 2 * set;
        cnt = rank + (int64_t)(ring ? 2 : 1) * arr;
        off = cnt + pad16((int64_t)(R + 1) * 4);
        stage = off + pad16((int64_t)(R + 1) * 4);
        end = stage + ((int64_t)(ring ? 2 : 1) * Smax + R + 2) * ds;
    }
};

/* Consumer shared memory: barriers, the heavy-hitter keys, the run table
 * row, the fold table, the resident per-group state and the gathered
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
 * (off[n] = total); returns the total to every lane.  One warp: lane l
 * takes counts [l * per, (l + 1) * per).  A single warp needs no CTA barrier,
 * which a block-wide scan of a few hundred counts would spend most of its
 * time in. */
__device__ __forceinline__ uint32_t scan_even_warp(const uint32_t *cnt, uint32_t *off, int n, int lane) {
    const int per = (n + 31) >> 5;
    const int b0 = lane * per;
    uint32_t s = 0;
    for (int j = 0; j < per; j++)
        if (b0 + j < n) s += (cnt[b0 + j] + 1u) & ~1u;
    uint32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    uint32_t run = incl - s;
    for (int j = 0; j < per; j++)
        if (b0 + j < n) {
            off[b0 + j] = run;
            run += (cnt[b0 + j] + 1u) & ~1u;
        }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (lane == 0) off[n] = total;
    return total;
}

/* The heavy-hitter list of list epoch `le` (-1: the query's list): its key
 * and count arrays (2 tiers of kMaxHot) and the number of entries; entry h
 * is tier0[h] for h < n1, else tier1[h - n1]. */
struct HotList {
    const int32_t *keys, *cnts;
    int n1, n_hot;
};

/* List epoch of batch i: -1 for the first kSSlots batches, else the index of
 * the refresh whose list the batch privatises. */
__device__ __forceinline__ int list_epoch(int i) { return i < kSSlots ? -1 : (i - kSSlots) / kSRefresh; }

__device__ __forceinline__ HotList hot_list_of(const SArgs &a, int le) {
    HotList L;
    const int *n;
    if (le < 0) {
        L.keys = a.q_hot;
        L.cnts = a.q_hot_cnt;
        n = a.q_hot_n;
    } else {
        const int s = le & 1;
        L.keys = a.lists + (int64_t)s * 2 * kMaxHot;
        L.cnts = a.list_cnt + (int64_t)s * 2 * kMaxHot;
        n = a.list_n + 2 * (int64_t)le;
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

/* Fold-table update of a consumer by one delta (padding deltas fall outside
 * the range).  Field f of local group l is t.w[f * t.stride + l]. */
__device__ __forceinline__ void tab_apply(const Acc &t, uint32_t kf, int32_t v, uint32_t lo_key, uint32_t rng,
                                          bool minmax) {
    const uint32_t l = (kf & kKeyMask) - lo_key;
    if (l >= rng) return;
    int32_t *const p = t.w + l;
    const int st = t.stride;
    if (kf & kRetract) {
        atomicAdd(p + A_LO * st, -(v & 0xFFFF));
        atomicAdd(p + A_HI * st, -(v >> 16));
        atomicAdd(p + A_RET * st, 1);
        if (kf & kFrontDep) atomicAdd(p + A_FDEP * st, 1);
    } else {
        atomicAdd(p + A_LO * st, v & 0xFFFF);
        atomicAdd(p + A_HI * st, v >> 16);
        atomicAdd(p + A_INS * st, 1);
        if (minmax) {
            atomicMin(p + A_IMIN * st, v);
            atomicMax(p + A_IMAX * st, v);
        }
    }
}

/* Heavy-hitter indices h[0 .. U) of keys k[0 .. U) (-1: not listed, or
 * live[u] false).  The first probes of all U keys are issued together; a key
 * that meets another key in its first slot walks on alone. */
template <int U>
__device__ __forceinline__ void hot_find_n(const int32_t *hkey, const int16_t *hidx, const int32_t *k,
                                           const bool *live, int n_hot, int *h) {
    uint32_t s[U];
    int32_t x[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        s[u] = hot_hash(k[u]);
        x[u] = (live[u] && n_hot) ? hkey[s[u]] : -1;
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
        h[u] = -1;
        if (x[u] == k[u]) {
            h[u] = hidx[s[u]];
        } else if (x[u] != -1) {
            uint32_t t = s[u];
            for (int probe = 1; probe < kHotSlots; probe++) {
                t = (t + 1) & (kHotSlots - 1);
                const int32_t y = hkey[t];
                if (y == k[u]) {
                    h[u] = hidx[t];
                    break;
                }
                if (y == -1) break;
            }
        }
    }
}

/* Runtime-flag forms of the CTA heavy-hitter record updates. */
__device__ __forceinline__ void rec_ins(const Acc &r, int h, int32_t v, bool minmax) {
    atomicAdd(r.f(A_LO, h), v & 0xFFFF);
    atomicAdd(r.f(A_HI, h), v >> 16);
    atomicAdd(r.f(A_INS, h), 1);
    if (minmax) {
        if (v < *(volatile int32_t *)r.f(A_IMIN, h)) atomicMin(r.f(A_IMIN, h), v);
        if (v > *(volatile int32_t *)r.f(A_IMAX, h)) atomicMax(r.f(A_IMAX, h), v);
    }
}

__device__ __forceinline__ void rec_ret(const Acc &r, int h, int32_t v, bool front_dep) {
    atomicAdd(r.f(A_LO, h), -(v & 0xFFFF));
    atomicAdd(r.f(A_HI, h), -(v >> 16));
    atomicAdd(r.f(A_RET, h), 1);
    if (front_dep) atomicAdd(r.f(A_FDEP, h), 1);
}

/* Stamp k of CTA `who` (producers 0 .. nA-1, consumers nA ..) for batch i,
 * when tracing. */
__device__ __forceinline__ void stamp(const SArgs &a, int who, int i, int k) {
    if (a.trace && threadIdx.x == 0) a.trace[((int64_t)who * a.nb + i) * 12 + k] = globaltimer();
}

/* Batch descriptors of the next few batches, in shared memory: thread 0
 * copies batches 0 .. kDescAhead - 1 at the start, then batch i + kDescAhead
 * at the start of batch i (one cp.async group a batch) and waits for all
 * but that newest group, so batches i .. i + kDescAhead - 1 are in place for
 * every thread after the next CTA barrier (slot (i + kDescAhead) mod
 * kDescRing held batch i - 1, which no thread reads any more).
 * Descriptor reads from global memory would put an L2 round trip on the
 * critical path of every chunk. */
constexpr int kDescRing = 4;
constexpr int kDescAhead = kDescRing - 1;

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_but1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

/* One thread: start copying batch i's descriptor into its ring slot (an
 * empty group past the last batch keeps the group count uniform). */
__device__ __forceinline__ void desc_copy(const SArgs &a, SBatch *ring, int i) {
    if (i < a.nb) {
        const uint4 *src = (const uint4 *)(a.b + i);
        uint4 *dst = (uint4 *)(ring + (i & (kDescRing - 1)));
#pragma unroll
        for (int q = 0; q < (int)(sizeof(SBatch) / 16); q++) cp_async(dst + q, src + q);
    }
    cp_async_commit();
}

/* The descriptor of batch j when batch i is current (ring copy for j in
 * [i, i + kDescAhead), else global memory). */
__device__ __forceinline__ const SBatch &desc_of(const SArgs &a, const SBatch *ring, int i, int j) {
    return (j >= i && j < i + kDescAhead) ? ring[j & (kDescRing - 1)] : a.b[j];
}

/* ------------------------------------------------------------------------ */
/* producer                                                                  */
/* ------------------------------------------------------------------------ */

/* A chunk a producer claimed: chunk c of batch i (i = nb: none left). */
struct Item {
    int i, c;
};

/* One thread: claim the next free chunk of batch `from` or of a later batch
 * (per-batch counters; work stealing, so that a producer whose SM is busier
 * cuts fewer chunks). */
__device__ __forceinline__ Item claim_chunk(const SArgs &a, const SBatch *ring, int cur, int from) {
    for (int j = from; j < a.nb; j++) {
        const int C = desc_of(a, ring, cur, j).C;
        if (C <= 0) continue;
        const unsigned long long c = atomicAdd(a.ctl + SC_CLAIM + j, 1ULL);
        if (c < (unsigned long long)C) return Item{j, (int)c};
    }
    return Item{a.nb, 0};
}

constexpr int kU = 4;                       /* tuples a producer thread handles at once in pass 2 */
constexpr int kTinyList = 4;                /* heavy-hitter lists this short are compared key by key */
constexpr int kPrivMin = 256;               /* exchanged deltas a batch that make a consumer privatise a key */
constexpr int kRangeWords = 80;             /* bitmap words of a consumer's range (a range holds < 2560 groups) */
static_assert(kSSmem / (A_NUM * 4 + 20) < kRangeWords * 32, "a range fits the listed-key bitmap");
constexpr uint32_t kNoRank = 0xFFFFFFFFu;   /* packed rank of a tuple whose delta is not exchanged */
constexpr uint32_t kFrontBit = 0x8000u;     /* in a packed retract rank: the tuple leaves the front */

template <int DS, bool RING>
__device__ __forceinline__ void producer(const SArgs &a, const int aid, unsigned char *smem) {
    constexpr int NT = RegTop<RING>::n;
    constexpr int kU1 = RING ? 2 : 4;   /* tuples a thread handles at once in pass 1 */
    typedef uint2 Delta;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool ring_any = a.ring_any != 0;
    const PLayout L(a.Smax, a.R, ring_any, DS);
    unsigned long long *bars = (unsigned long long *)(smem + L.bars);   /* [0..1] keys/values of a set, [2..3] its ring */
    int32_t *hkey = (int32_t *)(smem + L.hkey);
    int16_t *hidx = (int16_t *)(smem + L.hidx);
    int32_t *hcnt = (int32_t *)(smem + L.hcnt);   /* the list's counts, then scratch of the top selection */
    int32_t *htop = (int32_t *)(smem + L.htop);   /* rank of each list entry among the NT heaviest, or -1 */
    int32_t *rw = (int32_t *)(smem + L.hw);   /* the CTA heavy-hitter records, A_NUM fields of kMaxHot */
    long long *r64 = (long long *)(smem + L.h64);
    const Acc rec{rw, r64, kMaxHot};
    uint32_t *pr_ins = (uint32_t *)(smem + L.rank);
    uint32_t *pr_ret = (uint32_t *)(smem + L.rank + L.arr);
    uint32_t *cnt = (uint32_t *)(smem + L.cnt);
    uint32_t *off = (uint32_t *)(smem + L.off);
    Delta *stage_s = (Delta *)(smem + L.stage);
    __shared__ int s_len4[2];        /* bulk-loaded prefix of each input set's chunk (0: none pending) */
    __shared__ int s_item_i[2], s_item_c[2];   /* the claimed chunk each input set holds or awaits */
    __shared__ int s_nx_i, s_nx_c;             /* the claim that follows them, made while a chunk is cut */
    __shared__ int s_nhot, s_stop;
    __shared__ uint32_t s_total;     /* deltas of a chunk's runs */
    __shared__ int s_sel[NT];        /* list index of the key ranked t by count, -1 none */
    __shared__ int32_t s_tiny[kTinyList];   /* the keys of a list of at most kTinyList entries */
    __shared__ long long wtop_sum[NT][kW];
    __shared__ int32_t wtop_i[NT][kW][6];
    __shared__ __align__(16) SBatch s_desc[kDescRing];
    int cur = 0;   /* the current batch (descriptor ring window) */
    const int R = a.R;
    const uint32_t M = a.M;
    const uint32_t G = (uint32_t)a.G;
    const int64_t W = a.W;
    const bool minmax = a.minmax != 0;

    auto set_arr = [&](int set, int arr) -> int32_t * {
        return (int32_t *)(smem + L.in + (int64_t)set * L.set + (int64_t)arr * L.arr);
    };
    /* bulk loads of an item's keys and values (aligned batches only); one thread */
    auto issue_inputs = [&](int set, Item it) {
        s_len4[set] = 0;
        if (it.i >= a.nb) return;
        const SBatch &b = desc_of(a, s_desc, cur, it.i);
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
        for (int j = 0; j < kDescAhead; j++) desc_copy(a, s_desc, j);
        cp_async_wait_all();
    }
    __syncthreads();
    uint32_t par[4] = {0, 0, 0, 0};
    if (tid == 0) {
        /* the first two claims, their inputs requested at once */
        s_stop = 0;
        Item it = claim_chunk(a, s_desc, 0, 0);
        for (int s = 0; s < 2; s++) {
            issue_inputs(s, it);
            s_item_i[s] = it.i;
            s_item_c[s] = it.c;
            if (s == 0) it = claim_chunk(a, s_desc, 0, it.i);
        }
    }
    int set = 0;
    bool stop = false;
    int cur_le = -2;   /* list epoch whose heavy hitters the hash holds */
    int n_hot = 0;
    int sel[NT];
#pragma unroll
    for (int t = 0; t < NT; t++) sel[t] = -1;

    for (int i = 0; i < a.nb && !stop; i++) {
        const int slot = i % kSSlots;
        /* the slot's previous batch (i - kSSlots) has been folded by every
           consumer: its scratch is free (and a list it found is final) */
        if (tid == 0) {
            /* descriptors: batch i + kDescAhead on its way, i .. i + kDescAhead - 1 in place */
            desc_copy(a, s_desc, i + kDescAhead);
            cp_async_wait_but1();
            if (i >= kSSlots)
                stop = !wait_ctr(a.ctl + SC_B + slot, slot_target(a.nB, i - kSSlots), a.ctl, a.err, a.err_host,
                                 a.wait_ns);
            s_stop = stop;
            if (a.stamp_begin && s_item_i[set] == i) atomicMin(a.stamp_begin + i, globaltimer());
        }
        __syncthreads();
        if (s_stop) break;
        cur = i;
        stamp(a, aid, i, 0);
        const SBatch &B = s_desc[i & (kDescRing - 1)];
        const bool mine = s_item_i[set] == i;   /* this producer claimed chunks of the batch */
        const bool ring = RING && (B.flags & SB_RING) != 0;
        const bool front = RING && (B.flags & SB_FRONT) != 0;
        bool dep_pending = B.ring_dep >= 0;
        if (mine) {
            const int le = list_epoch(i);
            if (le != cur_le) {   /* a new heavy-hitter list: rebuild the hash */
                const HotList HL = hot_list_of(a, le);
                for (int s = tid; s < kHotSlots; s += kT) hkey[s] = -1;
                __syncthreads();
                for (int h = tid; h < HL.n_hot; h += kT) {
                    const int e = hot_entry(HL, h);
                    const int32_t k = __ldcg(HL.keys + e);
                    if (h < kTinyList) s_tiny[h] = k;
                    hcnt[h] = __ldcg(HL.cnts + e);
                    htop[h] = -1;
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
                if (tid == 0) s_nhot = HL.n_hot;
                cur_le = le;
                __syncthreads();
                n_hot = s_nhot;
                /* warp 0: the NT heaviest entries (count, then index), in order */
                if (warp == 0) {
                    for (int t = 0; t < NT; t++) {
                        int best = -1, bestc = -1;
                        for (int h = lane; h < n_hot; h += 32)
                            if (htop[h] < 0 && (hcnt[h] > bestc || (hcnt[h] == bestc && h < best))) {
                                bestc = hcnt[h];
                                best = h;
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
                            if (best >= 0) htop[best] = t;
                            s_sel[t] = best;
                        }
                        __syncwarp();
                    }
                }
                __syncthreads();
#pragma unroll
                for (int t = 0; t < NT; t++) sel[t] = s_sel[t];
            }
            for (int h = tid; h < n_hot; h += kT) acc_init(rec, h);
            __syncthreads();
        }
        long long r_sum[NT];
        int32_t r_ins[NT], r_ret[NT], r_imin[NT], r_imax[NT], r_fdep[NT];
#pragma unroll
        for (int t = 0; t < NT; t++) {
            r_sum[t] = 0;
            r_ins[t] = r_ret[t] = 0;
            r_imin[t] = INT32_MAX;
            r_imax[t] = INT32_MIN;
            r_fdep[t] = 0;
        }
        stamp(a, aid, i, 1);
        int nch = 0;

        for (int c = s_item_c[set]; s_item_i[set] == i && !stop; c = s_item_c[set]) {
            const int64_t cbeg = (int64_t)c * B.S;
            const int len = (int)min((int64_t)B.S, (int64_t)B.n - cbeg);
            int64_t s064 = (int64_t)B.slot0 + cbeg;   /* ring slot of the chunk's first tuple */
            if (s064 >= W) s064 -= W;
            const uint32_t s0 = (uint32_t)s064, Wu = (uint32_t)W;
            const int len4 = s_len4[set];
            int32_t *sk = set_arr(set, 0), *sv = set_arr(set, 1);
            int32_t *srk = set_arr(set, 2), *srv = set_arr(set, 3);
            for (int r = tid; r <= R; r += kT) cnt[r] = 0;
            /* the ring is read or written only after the batch that last
               wrote these slots is out (once per batch) */
            if (dep_pending) {
                if (tid == 0) {
                    const bool ok = wait_ctr(a.ctl + SC_A + B.ring_dep % kSSlots, slot_target(a.nA, B.ring_dep),
                                             a.ctl, a.err, a.err_host, a.wait_ns);
                    if (!ok) s_stop = 1;
                    fence_async_global();
                }
                __syncthreads();
                dep_pending = false;
                if (s_stop) {
                    stop = true;
                    break;
                }
            }
            if (ring && tid == 0 && len4 > 0) {
                const uint32_t bytes = 8u * len4;
                mbar_expect(&bars[2 + set], bytes);
                const int64_t n1 = min((int64_t)len4, W - s064);
                tma_load(srk, a.ring_k + s064, 4u * (uint32_t)n1, &bars[2 + set]);
                tma_load(srv, a.ring_v + s064, 4u * (uint32_t)n1, &bars[2 + set]);
                if (len4 > n1) {
                    const uint32_t n2 = (uint32_t)(len4 - n1);
                    tma_load(srk + n1, a.ring_k, 4u * n2, &bars[2 + set]);
                    tma_load(srv + n1, a.ring_v, 4u * n2, &bars[2 + set]);
                }
            }
            /* unaligned batches and ragged tails: per-element asynchronous copies */
            bool any_cp = false;
            for (int j = len4 + tid; j < len; j += kT) {
                any_cp = true;
                cp_async(sk + j, B.keys + cbeg + j);
                cp_async(sv + j, B.vals + cbeg + j);
                if (ring) {
                    uint32_t sl = s0 + (uint32_t)j;
                    if (sl >= Wu) sl -= Wu;
                    cp_async(srk + j, a.ring_k + sl);
                    cp_async(srv + j, a.ring_v + sl);
                }
            }
            if (any_cp) cp_async_wait_all();
            if (nch == 0) stamp(a, aid, i, 4);
            if (tid == 0 && len4 > 0) {
                bool ok = mbar_wait(&bars[set], par[set], a.wait_ns);
                if (nch == 0) stamp(a, aid, i, 5);
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
            /* pass 1: the new tuples go to the ring (coalesced stores); the
               heaviest keys are summed in registers, the other heavy
               hitters in the shared records; every other delta takes a
               rank in its key range's run, packed with the range as
               (range << 16 | rank), the front bit marking a retract that
               leaves the front */
            bool bad = false;
            const uint32_t hmod = (uint32_t)B.hmod;
            const int32_t old_len = B.old_len, fa = B.fa, fb = B.fb;
            if (!ring && n_hot == 0) {
                /* no heavy hitters and no retracts: every tuple takes a rank,
                   one tuple at a time (four at once measured slower here) */
                for (int j = tid; j < len; j += kT) {
                    const int32_t k = sk[j], v = sv[j];
                    uint32_t sl = s0 + (uint32_t)j;
                    if (sl >= Wu) sl -= Wu;
                    a.ring_k[sl] = k;
                    a.ring_v[sl] = v;
                    uint32_t p = kNoRank;
                    if ((uint32_t)k >= G) {
                        bad = true;
                    } else {
                        const uint32_t r = __umulhi((uint32_t)k, M);
                        p = (r << 16) | atomicAdd(&cnt[r], 1u);
                    }
                    pr_ins[j] = p;
                }
            } else if (!ring && n_hot <= kTinyList) {
                /* a short heavy-hitter list and no retracts: each key is
                   compared with the listed keys in registers, no hash probe */
                int32_t tkey[kTinyList];   /* -1: no entry (keys are >= 0) */
#pragma unroll
                for (int t = 0; t < kTinyList; t++) tkey[t] = t < n_hot ? s_tiny[t] : -1;
                for (int j = tid; j < len; j += kT) {
                    const int32_t k = sk[j], v = sv[j];
                    uint32_t sl = s0 + (uint32_t)j;
                    if (sl >= Wu) sl -= Wu;
                    a.ring_k[sl] = k;
                    a.ring_v[sl] = v;
                    uint32_t p = kNoRank;
                    if ((uint32_t)k >= G) {
                        bad = true;
                    } else {
                        int h = -1;
#pragma unroll
                        for (int t = 0; t < kTinyList; t++)
                            if (k == tkey[t]) h = t;
                        if (h < 0) {
                            const uint32_t r = __umulhi((uint32_t)k, M);
                            p = (r << 16) | atomicAdd(&cnt[r], 1u);
                        } else {
                            bool reg = false;
#pragma unroll
                            for (int t = 0; t < NT; t++)
                                if (h == sel[t]) {
                                    r_sum[t] += v;
                                    r_ins[t]++;
                                    r_imin[t] = min(r_imin[t], v);
                                    r_imax[t] = max(r_imax[t], v);
                                    reg = true;
                                }
                            if (!reg) rec_ins(rec, h, v, minmax);
                        }
                    }
                    pr_ins[j] = p;
                }
            } else
            for (int j0 = tid; j0 < len; j0 += kU1 * kT) {
                int32_t kk[kU1], vv[kU1];
                bool live[kU1];
                int hh[kU1];
                uint32_t p[kU1];
#pragma unroll
                for (int u = 0; u < kU1; u++) {
                    const int j = j0 + u * kT;
                    const bool in = j < len;
                    kk[u] = in ? sk[j] : 0;
                    vv[u] = in ? sv[j] : 0;
                    if (in) {
                        uint32_t sl = s0 + (uint32_t)j;
                        if (sl >= Wu) sl -= Wu;
                        a.ring_k[sl] = kk[u];
                        a.ring_v[sl] = vv[u];
                    }
                    bad |= in && (uint32_t)kk[u] >= G;
                    live[u] = in && (uint32_t)kk[u] < G;
                }
                hot_find_n<kU1>(hkey, hidx, kk, live, n_hot, hh);
#pragma unroll
                for (int u = 0; u < kU1; u++) {
                    p[u] = kNoRank;
                    if (live[u] && hh[u] < 0) {
                        const uint32_t r = __umulhi((uint32_t)kk[u], M);
                        p[u] = (r << 16) | atomicAdd(&cnt[r], 1u);
                    }
                }
#pragma unroll
                for (int u = 0; u < kU1; u++) {
                    const int j = j0 + u * kT;
                    if (j < len) pr_ins[j] = p[u];
                    if (hh[u] >= 0) {
                        bool reg = false;
#pragma unroll
                        for (int t = 0; t < NT; t++)
                            if (hh[u] == sel[t]) {
                                r_sum[t] += vv[u];
                                r_ins[t]++;
                                r_imin[t] = min(r_imin[t], vv[u]);
                                r_imax[t] = max(r_imax[t], vv[u]);
                                reg = true;
                            }
                        if (!reg) rec_ins(rec, hh[u], vv[u], minmax);
                    }
                }
                if (ring) {
                    bool fr[kU1];
#pragma unroll
                    for (int u = 0; u < kU1; u++) {
                        const int j = j0 + u * kT;
                        const bool in = j < len;
                        uint32_t sl = s0 + (uint32_t)j;
                        if (sl >= Wu) sl -= Wu;
                        int32_t rel = (int32_t)sl - (int32_t)hmod;
                        if (rel < 0) rel += (int32_t)Wu;
                        kk[u] = in ? srk[j] : 0;
                        vv[u] = in ? srv[j] : 0;
                        live[u] = in && rel < old_len && (uint32_t)kk[u] < G;
                        fr[u] = live[u] && front && rel >= fa && rel < fb;
                    }
                    hot_find_n<kU1>(hkey, hidx, kk, live, n_hot, hh);
#pragma unroll
                    for (int u = 0; u < kU1; u++) {
                        p[u] = kNoRank;
                        if (live[u] && hh[u] < 0) {
                            const uint32_t r = __umulhi((uint32_t)kk[u], M);
                            p[u] = (r << 16) | atomicAdd(&cnt[r], 1u) | (fr[u] ? kFrontBit : 0u);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kU1; u++) {
                        const int j = j0 + u * kT;
                        if (j < len) pr_ret[j] = p[u];
                        if (hh[u] >= 0) {
                            bool reg = false;
#pragma unroll
                            for (int t = 0; t < NT; t++)
                                if (hh[u] == sel[t]) {
                                    r_sum[t] -= vv[u];
                                    r_ret[t]++;
                                    r_fdep[t] += fr[u] ? 1 : 0;
                                    reg = true;
                                }
                            if (!reg) rec_ret(rec, hh[u], vv[u], fr[u]);
                        }
                    }
                }
            }
            if (bad) {
                atomicOr(a.err, 1);
                if (a.err_host) *(volatile int *)a.err_host = 1;
            }
            /* the previous chunk's bulk store must have read the staging area */
            if (tid == 0) tma_wait_read();
            __syncthreads();
            stamp(a, aid, i, nch == 0 ? 3 : 8);
            for (int h = tid; h < n_hot; h += kT) acc_fold(rec, h);
            if (warp == 0) {
                /* the runs' offsets; each range's run in this chunk (begin,
                   padded length) to the range-major run table; the padding
                   delta of every odd run */
                const uint32_t t = scan_even_warp(cnt, off, R, lane);
                if (lane == 0) s_total = t;
                uint2 *row = a.pairs + (int64_t)slot * a.pairs_slot + c;
                for (int r = lane; r < R; r += 32) {
                    const uint32_t n = cnt[r], o = off[r];
                    row[(int64_t)r * a.Cpad] = make_uint2(o, (n + 1u) & ~1u);
                    if (n & 1u) stage_s[o + n] = DeltaIO::make(kPadKey, 0);
                }
            } else if (tid == 32) {
                /* the next claim, while warp 0 scans: its round trip stays
                   off the chunk's path (claims stay in batch order: after
                   the other input set's) */
                const Item nx = claim_chunk(a, s_desc, cur, s_item_i[set ^ 1]);
                s_nx_i = nx.i;
                s_nx_c = nx.c;
            }
            __syncthreads();
            const uint32_t total = s_total;
            /* pass 2: place the exchanged deltas by rank, kU tuples of a
               thread at a time (their loads issued before their stores) */
            for (int j0 = tid; j0 < len; j0 += kU * kT) {
                uint32_t p[kU];
                int32_t kk[kU], vv[kU];
#pragma unroll
                for (int u = 0; u < kU; u++) {
                    const int j = j0 + u * kT;
                    p[u] = j < len ? pr_ins[j] : kNoRank;
                    kk[u] = j < len ? sk[j] : 0;
                    vv[u] = j < len ? sv[j] : 0;
                }
                uint32_t o[kU];
#pragma unroll
                for (int u = 0; u < kU; u++) o[u] = p[u] != kNoRank ? off[p[u] >> 16] + (p[u] & 0x7FFFu) : 0u;
#pragma unroll
                for (int u = 0; u < kU; u++)
                    if (p[u] != kNoRank) stage_s[o[u]] = DeltaIO::make((uint32_t)kk[u], vv[u]);
                if (ring) {
#pragma unroll
                    for (int u = 0; u < kU; u++) {
                        const int j = j0 + u * kT;
                        p[u] = j < len ? pr_ret[j] : kNoRank;
                        kk[u] = j < len ? srk[j] : 0;
                        vv[u] = j < len ? srv[j] : 0;
                    }
#pragma unroll
                    for (int u = 0; u < kU; u++) o[u] = p[u] != kNoRank ? off[p[u] >> 16] + (p[u] & 0x7FFFu) : 0u;
#pragma unroll
                    for (int u = 0; u < kU; u++)
                        if (p[u] != kNoRank)
                            stage_s[o[u]] = DeltaIO::make((uint32_t)kk[u] | kRetract |
                                                              ((p[u] & kFrontBit) ? kFrontDep : 0u),
                                                          vv[u]);
                }
            }
            __syncthreads();
            /* the runs go out by one bulk store; the input set is free and
               takes the item two ahead */
            if (tid == 0) {
                if (total > 0) {
                    fence_async_smem();
                    tma_store((Delta *)a.stage + (int64_t)slot * a.stage_slot + (int64_t)c * a.stride, stage_s,
                              total * (uint32_t)DS);
                    tma_commit();
                }
                const Item nx{s_nx_i, s_nx_c};
                issue_inputs(set, nx);
                s_item_i[set] = nx.i;
                s_item_c[set] = nx.c;
            }
            set ^= 1;
            stamp(a, aid, i, nch == 0 ? 6 : 9);
            nch++;
        }
        if (stop) break;
        if (mine && n_hot) {
            /* this producer's heavy-hitter partials of the batch: the CTA
               records plus the threads' register sums of the heaviest keys */
#pragma unroll
            for (int t = 0; t < NT; t++) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    r_sum[t] += __shfl_xor_sync(kFull, r_sum[t], o);
                    r_ins[t] += __shfl_xor_sync(kFull, r_ins[t], o);
                    r_ret[t] += __shfl_xor_sync(kFull, r_ret[t], o);
                    r_imin[t] = min(r_imin[t], __shfl_xor_sync(kFull, r_imin[t], o));
                    r_imax[t] = max(r_imax[t], __shfl_xor_sync(kFull, r_imax[t], o));
                    r_fdep[t] += __shfl_xor_sync(kFull, r_fdep[t], o);
                }
                if (lane == 0) {
                    wtop_sum[t][warp] = r_sum[t];
                    wtop_i[t][warp][0] = r_ins[t];
                    wtop_i[t][warp][1] = r_ret[t];
                    wtop_i[t][warp][2] = r_imin[t];
                    wtop_i[t][warp][3] = r_imax[t];
                    wtop_i[t][warp][4] = r_fdep[t];
                }
            }
            __syncthreads();
            HotAcc *dst = a.hotpart + ((int64_t)slot * a.nA + aid) * kMaxHot;
            for (int h = tid; h < n_hot; h += kT) {
                HotAcc r;
                r.sum = r64[h];
                r.ins = *rec.f(A_INS, h);
                r.ret = *rec.f(A_RET, h);
                r.imin = *rec.f(A_IMIN, h);
                r.imax = *rec.f(A_IMAX, h);
                r.fdep = *rec.f(A_FDEP, h);
                r.pad_ = 0;
                const int t = htop[h];
                if (t >= 0)
                    for (int w = 0; w < kW; w++) {
                        r.sum += wtop_sum[t][w];
                        r.ins += wtop_i[t][w][0];
                        r.ret += wtop_i[t][w][1];
                        r.imin = min(r.imin, wtop_i[t][w][2]);
                        r.imax = max(r.imax, wtop_i[t][w][3]);
                        r.fdep += wtop_i[t][w][4];
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
        /* reported by another thread than 0, whose next batch starts meanwhile */
        if (tid == 32) {
            /* whether this producer's partials of the batch are to be read */
            *(volatile unsigned long long *)(a.ctl + SC_FLAG + slot * 1024 + aid) = (mine && n_hot) ? 1ULL : 0ULL;
            if (!(aid == 0 && i == a.stall_batch)) red_release(a.ctl + SC_A + slot, 1ULL);
        }
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
    typedef uint2 Delta;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool minmax = a.minmax != 0, avg = a.avg != 0;
    const int tcap = a.tcap;
    const CLayout L(tcap, a.Cpad, a.dcap, DS, minmax);
    unsigned long long *bars = (unsigned long long *)(smem + L.bars);   /* [0] run-table row, [1] gather */
    int32_t *hl = (int32_t *)(smem + L.hl);
    uint2 *pairs = (uint2 *)(smem + L.pairs);
    int32_t *tw = (int32_t *)(smem + L.tw);
    const Acc tab{tw, (long long *)(smem + L.t64), tcap};
    long long *st_sum = (long long *)(smem + L.ssum);
    int32_t *st_cnt = (int32_t *)(smem + L.scnt);
    int32_t *st_bmin = (int32_t *)(smem + L.sext);
    int32_t *st_bmax = st_bmin + tcap;
    int32_t *st_fmin = st_bmax + tcap;
    int32_t *st_fmax = st_fmin + tcap;
    Delta *dstage = (Delta *)(smem + L.dstage);
    __shared__ int s_stop, s_nhot;
    __shared__ uint32_t s_total;
    __shared__ __align__(16) SBatch s_desc[kDescRing];
    __shared__ uint32_t s_listed[kRangeWords];   /* the range's listed heavy hitters (batch's list) */
    __shared__ int s_ctop[2];                    /* the range's privatised keys (local index, -1 none) */
    /* scratch of the privatised keys' reduction and of their choice, over
       the gather area, which is free once a batch's deltas are applied */
    int *s_cand_v = (int *)dstage;                       /* [kW][2] */
    int *s_cand_l = s_cand_v + 2 * kW;                   /* [kW][2] */
    long long *s_csum = (long long *)(s_cand_l + 2 * kW);   /* [2][kW] */
    int32_t *s_cfield = (int32_t *)(s_csum + 2 * kW);    /* [2][kW][6] */
    const bool has_range = bid < a.R;
    const int64_t lo = has_range ? stream_range_lo((uint32_t)bid, a.M, a.G) : 0;
    const int64_t hi = has_range ? stream_range_lo((uint32_t)bid + 1, a.M, a.G) : 0;
    const int rng = (int)(hi - lo);   /* <= tcap (the host sized tcap from the same bounds) */
    const uint32_t lo32 = (uint32_t)lo;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_stop = 0;
        s_ctop[0] = s_ctop[1] = -1;
        for (int j = 0; j < kDescAhead; j++) desc_copy(a, s_desc, j);
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
    int cur_le = -2;
    for (int i = 0; i < a.nb && !stop; i++) {
        const int slot = i % kSSlots;
        if (tid == 0) {
            desc_copy(a, s_desc, i + kDescAhead);
            cp_async_wait_but1();
            stop = !wait_ctr(a.ctl + SC_A + slot, slot_target(a.nA, i), a.ctl, a.err, a.err_host, a.wait_ns);
            fence_async_global();
            s_stop = stop;
            const SBatch &b = s_desc[i & (kDescRing - 1)];
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
        const SBatch &B = s_desc[i & (kDescRing - 1)];
        if (has_range) {
            const int C = B.C;
            const uint32_t flags = (uint32_t)B.flags;
            const bool replace = (flags & SB_REPLACE) != 0;
            /* a new heavy-hitter list: its keys (their partials are merged below) */
            const int le = list_epoch(i);
            if (le != cur_le) {
                const HotList HL = hot_list_of(a, le);
                for (int h = tid; h < HL.n_hot; h += kT) hl[h] = __ldcg(HL.keys + hot_entry(HL, h));
                if (tid == 0) s_nhot = HL.n_hot;
                cur_le = le;
            }
            for (int l = tid; l < rng; l += kT) acc_init(tab, l);
            for (int w = tid; w < kRangeWords; w += kT) s_listed[w] = 0u;
            /* the two keys of the range with the most exchanged deltas in the
               previous batch: every thread sums theirs in registers */
            const int ct0 = s_ctop[0], ct1 = s_ctop[1];
            /* the privatised keys as local indices no delta of the range can
               miss-match when unset (a range's keys are 0 .. rng - 1) */
            const uint32_t cu0 = ct0 >= 0 ? (uint32_t)ct0 : 0xFFFFFFFFu, cu1 = ct1 >= 0 ? (uint32_t)ct1 : 0xFFFFFFFFu;
            long long c_sum[2] = {0, 0};
            int32_t c_ins[2] = {0, 0}, c_ret[2] = {0, 0}, c_imin[2] = {INT32_MAX, INT32_MAX},
                    c_imax[2] = {INT32_MIN, INT32_MIN}, c_fdep[2] = {0, 0};
            auto cpriv = [&](int t, uint32_t kf, int32_t dv) {
#pragma unroll
                for (int q = 0; q < 2; q++)   /* constant indices: the sums stay in registers */
                    if (q == t) {
                        if (kf & kRetract) {
                            c_sum[q] -= dv;
                            c_ret[q]++;
                            c_fdep[q] += (kf & kFrontDep) ? 1 : 0;
                        } else {
                            c_sum[q] += dv;
                            c_ins[q]++;
                            c_imin[q] = min(c_imin[q], dv);
                            c_imax[q] = max(c_imax[q], dv);
                        }
                    }
            };
            auto capply = [&](uint32_t kf, int32_t dv) {
                const uint32_t l = (kf & kKeyMask) - lo32;
                if (l == cu0) cpriv(0, kf, dv);
                else if (l == cu1) cpriv(1, kf, dv);
                else tab_apply(tab, kf, dv, lo32, (uint32_t)rng, minmax);
            };
            /* warp 0: the run-table row's exclusive scan (each lane a block of
               consecutive chunks), then the first round's copies */
            uint32_t total = 0;
            if (warp == 0 && C > 0) {
                if (lane == 0 && !mbar_wait(&bars[0], ppar, a.wait_ns)) {
                    raise_timeout(a.ctl, a.err, a.err_host);
                    s_stop = 1;
                }
                __syncwarp();
                const int per = (C + 31) >> 5;
                const int c0 = lane * per, c1 = min(C, c0 + per);
                uint32_t s = 0;
                for (int c = c0; c < c1; c++) s += pairs[c].y;
                uint32_t incl = s;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += y;
                }
                total = __shfl_sync(kFull, incl, 31);
                uint32_t run = incl - s;
                for (int c = c0; c < c1; c++) {
                    const uint32_t x = pairs[c].y;
                    pairs[c].y = run;
                    run += x;
                }
                if (lane == 0) s_total = total;
            }
            if (C > 0) ppar ^= 1u;
            __syncthreads();
            if (s_stop) {
                stop = true;
                break;
            }
            stamp(a, me, i, 1);
            total = C > 0 ? s_total : 0u;
            const Delta *stage = (const Delta *)a.stage + (int64_t)slot * a.stage_slot;
            /* the 16-bit half sums stay exact for 32767 deltas of one group:
               a larger batch folds them into the int64 sums every round */
            const bool fold_rounds = total > 32767u;
            for (uint32_t b0 = 0; b0 < total && !stop; b0 += (uint32_t)a.dcap) {
                const uint32_t b1 = min(total, b0 + (uint32_t)a.dcap);
                if (b0 > 0) {   /* the previous round's deltas are applied */
                    __syncthreads();
                    if (fold_rounds) {
                        for (int l = tid; l < rng; l += kT) acc_fold(tab, l);
                        __syncthreads();
                    }
                }
                if (tid == 0) mbar_expect(&bars[1], (b1 - b0) * (uint32_t)DS);
                __syncthreads();
                /* one bulk copy per chunk's run (part), issued by the threads side by side */
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
                if (b0 == 0) stamp(a, me, i, 2);
                const uint32_t nd = b1 - b0;
                {
                    const uint4 *d2 = (const uint4 *)dstage;   /* two deltas a load */
                    for (uint32_t j = tid; j < nd / 2; j += kT) {
                        const uint4 x = d2[j];
                        const uint32_t l0 = (x.x & kKeyMask) - lo32, l1 = (x.z & kKeyMask) - lo32;
                        if (l0 == cu0 || l0 == cu1) cpriv(l0 == cu0 ? 0 : 1, x.x, (int32_t)x.y);
                        else tab_apply(tab, x.x, (int32_t)x.y, lo32, (uint32_t)rng, minmax);
                        if (l1 == cu0 || l1 == cu1) cpriv(l1 == cu0 ? 0 : 1, x.z, (int32_t)x.w);
                        else tab_apply(tab, x.z, (int32_t)x.w, lo32, (uint32_t)rng, minmax);
                    }
                }
            }
            if (stop) break;
            __syncthreads();
            for (int l = tid; l < rng; l += kT) acc_fold(tab, l);
            __syncthreads();
            if (ct0 >= 0 || ct1 >= 0) {
                /* the privatised keys' register sums, over the CTA */
#pragma unroll
                for (int t = 0; t < 2; t++) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        c_sum[t] += __shfl_xor_sync(kFull, c_sum[t], o);
                        c_ins[t] += __shfl_xor_sync(kFull, c_ins[t], o);
                        c_ret[t] += __shfl_xor_sync(kFull, c_ret[t], o);
                        c_imin[t] = min(c_imin[t], __shfl_xor_sync(kFull, c_imin[t], o));
                        c_imax[t] = max(c_imax[t], __shfl_xor_sync(kFull, c_imax[t], o));
                        c_fdep[t] += __shfl_xor_sync(kFull, c_fdep[t], o);
                    }
                    if (lane == 0) {
                        int32_t *f = s_cfield + (t * kW + warp) * 6;
                        s_csum[t * kW + warp] = c_sum[t];
                        f[0] = c_ins[t];
                        f[1] = c_ret[t];
                        f[2] = c_imin[t];
                        f[3] = c_imax[t];
                        f[4] = c_fdep[t];
                        f[5] = 0;
                        fence_async_smem();   /* the gather area: the next batch's copies land there */
                    }
                }
                __syncthreads();
                if (tid < 2) {
                    const int l = tid == 0 ? ct0 : ct1;
                    if (l >= 0) {
                        long long sm = 0;
                        int32_t in = 0, rt = 0, mn = INT32_MAX, mx = INT32_MIN, fd = 0;
                        for (int w = 0; w < kW; w++) {
                            const int32_t *f = s_cfield + (tid * kW + w) * 6;
                            sm += s_csum[tid * kW + w];
                            in += f[0];
                            rt += f[1];
                            mn = min(mn, f[2]);
                            mx = max(mx, f[3]);
                            fd += f[4];
                        }
                        tab.acc64[l] += sm;
                        *tab.f(A_INS, l) += in;
                        *tab.f(A_RET, l) += rt;
                        *tab.f(A_IMIN, l) = min(*tab.f(A_IMIN, l), mn);
                        *tab.f(A_IMAX, l) = max(*tab.f(A_IMAX, l), mx);
                        *tab.f(A_FDEP, l) += fd;
                    }
                }
                __syncthreads();
            }
            stamp(a, me, i, 3);
            /* heavy hitters of the range: a warp sums a key's partials over
               the producers that cut chunks of the batch (flagged) */
            const int n_hot = s_nhot;
            const HotAcc *parts = a.hotpart + (int64_t)slot * a.nA * kMaxHot;
            const unsigned long long *pflag = a.ctl + SC_FLAG + slot * 1024;
            for (int h = warp; h < n_hot; h += kW) {
                const int32_t key = hl[h];
                if ((int64_t)key < lo || (int64_t)key >= hi) continue;
                long long hs = 0;
                int32_t ins = 0, ret = 0, imin = INT32_MAX, imax = INT32_MIN, fdep = 0;
                for (int p = lane; p < a.nA; p += 32) {
                    if (!__ldcg(pflag + p)) continue;
                    const HotAcc *r = parts + (int64_t)p * kMaxHot + h;
                    hs += __ldcg(&r->sum);
                    ins += __ldcg(&r->ins);
                    ret += __ldcg(&r->ret);
                    imin = min(imin, __ldcg(&r->imin));
                    imax = max(imax, __ldcg(&r->imax));
                    fdep += __ldcg(&r->fdep);
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
                    const int l = (int)(key - lo);
                    atomicOr(&s_listed[l >> 5], 1u << (l & 31));
                    tab.acc64[l] += hs;
                    *tab.f(A_INS, l) += ins;
                    *tab.f(A_RET, l) += ret;
                    *tab.f(A_IMIN, l) = min(*tab.f(A_IMIN, l), imin);
                    *tab.f(A_IMAX, l) = max(*tab.f(A_IMAX, l), imax);
                    *tab.f(A_FDEP, l) += fdep;
                }
            }
            __syncthreads();
            stamp(a, me, i, 4);
            /* finalise: state, results of touched groups; heavy hitters are
               listed by the batches whose lists are used later */
            const uint32_t thr = B.hot_threshold, gthr = B.hot_gthr;
            const bool detect = a.hot_cap > 0 && (i % kSRefresh == 0 || i == a.nb - 1);
            /* the privatised pair is picked every kSRefresh batches, like the lists */
            const bool cpick = i % kSRefresh == 0;
            int cv0 = -1, cl0 = -1, cv1 = -1, cl1 = -1;   /* this thread's two busiest unlisted groups */
            for (int l = tid; l < rng; l += kT) {
                const int32_t ins = *tab.f(A_INS, l), ret = *tab.f(A_RET, l);
                if (cpick && !((s_listed[l >> 5] >> (l & 31)) & 1u)) {
                    const int v = ins + ret;
                    if (v > cv0) {
                        cv1 = cv0;
                        cl1 = cl0;
                        cv0 = v;
                        cl0 = l;
                    } else if (v > cv1) {
                        cv1 = v;
                        cl1 = l;
                    }
                }
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
                    /* front tuples left: the group's front pointer moves on,
                       and the front's extrema are those of its later front
                       tuples (empty once none is left) */
                    const int32_t dep = *tab.f(A_FDEP, l);
                    if (dep > 0) {
                        const int2 x = front_next(a.fptr, a.sufs, g, dep);
                        flo = x.x;
                        fhi = x.y;
                    }
                    st_bmin[l] = blo;
                    st_bmax[l] = bhi;
                    st_fmin[l] = flo;
                    st_fmax[l] = fhi;
                    a.rmin[g] = cn > 0 ? min(blo, flo) : INT32_MAX;
                    a.rmax[g] = cn > 0 ? max(bhi, fhi) : INT32_MIN;
                }
                if (avg)
                    a.ravg[g] = cn > 0 ? avg_rn(s, cn)
                                       : __longlong_as_double(0x7FF8000000000000LL);
                if (detect && (uint32_t)ins >= thr) {
                    const int tier = (uint32_t)ins >= gthr ? 0 : 1;
                    /* the refresh list of this batch, and the query's list after the last batch */
                    for (int w = 0; w < 2; w++) {
                        int li;
                        if (w == 0) {
                            if (i % kSRefresh) continue;
                            li = i / kSRefresh;
                        } else {
                            if (i != a.nb - 1) continue;
                            li = kSListN - 1;
                        }
                        const int ls = w == 0 ? li & 1 : 2;
                        const int idx = atomicAdd(a.list_n + 2 * li + tier, 1);
                        if (idx < a.hot_cap) {
                            a.lists[((int64_t)ls * 2 + tier) * kMaxHot + idx] = (int32_t)g;
                            a.list_cnt[((int64_t)ls * 2 + tier) * kMaxHot + idx] = ins;
                        }
                    }
                }
            }
            /* the warp's two busiest: the range's pair is picked after the barrier */
            if (cpick) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const int ov0 = __shfl_xor_sync(kFull, cv0, o), ol0 = __shfl_xor_sync(kFull, cl0, o);
                    const int ov1 = __shfl_xor_sync(kFull, cv1, o), ol1 = __shfl_xor_sync(kFull, cl1, o);
                    if (ov0 > cv0) {
                        if (cv0 > ov1) {
                            cv1 = cv0;
                            cl1 = cl0;
                        } else {
                            cv1 = ov1;
                            cl1 = ol1;
                        }
                        cv0 = ov0;
                        cl0 = ol0;
                    } else if (ov0 > cv1) {
                        cv1 = ov0;
                        cl1 = ol0;
                    }
                }
                if (lane == 0) {
                    s_cand_v[2 * warp] = cv0;
                    s_cand_l[2 * warp] = cl0;
                    s_cand_v[2 * warp + 1] = cv1;
                    s_cand_l[2 * warp + 1] = cl1;
                    fence_async_smem();
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
                    a.snap_avg[base + g] = avg && cn > 0 ? avg_rn(s, cn)
                                                         : __longlong_as_double(0x7FF8000000000000LL);
                }
            }
        }
        __syncthreads();
        if (tid == 64 && has_range && i % kSRefresh == 0) {
            /* the range's two groups with the most exchanged deltas (listed
               heavy hitters aside), privatised in the next batch if busy; by
               a thread that neither polls nor reports */
            int v0 = -1, l0 = -1, v1 = -1, l1 = -1;
            for (int w = 0; w < kW; w++)
                for (int t = 0; t < 2; t++) {
                    const int v = s_cand_v[2 * w + t], l = s_cand_l[2 * w + t];
                    if (v > v0) {
                        v1 = v0;
                        l1 = l0;
                        v0 = v;
                        l0 = l;
                    } else if (v > v1) {
                        v1 = v;
                        l1 = l;
                    }
                }
            s_ctop[0] = v0 >= kPrivMin ? l0 : -1;
            s_ctop[1] = v1 >= kPrivMin ? l1 : -1;
        }
        stamp(a, me, i, 5);
        if (tid == 0 && a.stamp_end && has_range) atomicMax(a.stamp_end + i, globaltimer());
        /* reported by another thread than 0, whose wait for the next batch starts meanwhile */
        if (tid == 32) red_release(a.ctl + SC_B + slot, 1ULL);
        stamp(a, me, i, 6);
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

template <int DS, bool RING>
__global__ void __launch_bounds__(kT, 2) stream_kernel(const __grid_constant__ SArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_role, s_id;
    if (threadIdx.x == 0) {
        const uint32_t sm = sm_id();
        int role = -1, id = -1;
        if (sm < (uint32_t)kMaxSmSlots) {
            /* the first CTA on an SM produces; the second consumes, except on
               the first (nA - nB) / 2 SMs to place a second CTA, where it
               produces too */
            const unsigned long long k = atomicAdd(a.ctl + SC_SM + sm, 1ULL);
            role = k == 0 ? 0 : (k == 1 ? 1 : -1);
            if (role == 1 && atomicAdd(a.ctl + SC_PP, 1ULL) < (unsigned long long)((a.nA - a.nB) / 2)) role = 0;
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
    if (s_role == 0) producer<DS, RING>(a, s_id, smem);
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
    const int64_t per = 2 * 4 * (ring ? 4 : 2) + 4 * (ring ? 2 : 1) + (int64_t)(ring ? 2 : 1) * ds;
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

/* The kernel of a launch: retract code when some batch reads the ring. */
const void *stream_fn(int ds, bool ring) {
    (void)ds;   /* one delta form (8 bytes) for every batch */
    return ring ? (const void *)stream_kernel<8, true> : (const void *)stream_kernel<8, false>;
}

bool stream_launchable() {
    const void *fns[2] = {stream_fn(8, false), stream_fn(8, true)};
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
    const void *fn = stream_fn(ds, a.ring_any != 0);
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
