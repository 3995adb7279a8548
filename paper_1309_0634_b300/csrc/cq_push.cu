/*
 * cq_push.cu -- the partitioned push: one cooperative launch per batch that
 * reads the batch and the evicted ring slots once, exchanges the per-group
 * updates through L2 by key range, and lets the CTA that owns a key range
 * aggregate it in shared memory and rewrite its groups' state and results.
 *
 * Phase A (every CTA, one or more chunks of <= 4096 consecutive effective
 * tuples, equal sizes so every CTA has the same work):
 *   - read the new tuples (k, v) and the tuples (k', v') they evict from the
 *     window ring, write (k, v) into the ring (Section 3.2's ring with an
 *     overwritten oldest entry, here one global ring);
 *   - an insert delta (k, +v) and a retract delta (k', -v') per tuple;
 *   - a delta of a heavy hitter (hot key, chosen at the previous push) is
 *     folded into a CTA-private shared-memory record -- the heavy hitter's
 *     work is split over all CTAs instead of landing on one owner (the
 *     paper's remedy for skew, Section 4: move load off an overloaded
 *     worker; here decided per batch on the device);
 *   - every other delta is counted per key-range partition, the chunk's
 *     deltas are counting-sorted by partition in shared memory (the paper's
 *     two-pass reordering of a batch, Section 3.1, done per chunk on the
 *     GPU) and written out contiguously, with one offset row per chunk (the
 *     paper's threadDataIndicator).
 * Grid-wide barrier (bounded spin; the kernel is launched cooperatively).
 * Phase B (CTA b owns the contiguous partitions [P*b/grid, P*(b+1)/grid)):
 *   - gather the deltas of its contiguous key range from every chunk (one
 *     run per chunk, copied asynchronously into shared memory) and fold them
 *     into a shared-memory table of the range's groups with 32-bit shared
 *     atomics only: a 64-bit sum is accumulated as the signed sums of the
 *     high and low 16-bit halves of the values, which cannot overflow within
 *     a batch of at most 8192 deltas, and folded into an int64 after each
 *     batch;
 *   - add the heavy hitters' per-CTA partial records;
 *   - for every touched group: read-modify-write SUM/COUNT and the epoch-
 *     tagged MIN/MAX segments, write MIN/MAX/AVG;
 *   - groups whose insert count reached the threshold become the hot keys of
 *     the next push (exact counting sketch; the effect is applied one push
 *     later, as the paper's rebalancing is, Section 3.1).
 * No global atomics touch per-group state; every result is exact.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "cq_internal.h"
#include "cq_push.cuh"
#include "cq_tags.cuh"

namespace cq {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kRetract = 0x80000000u;
constexpr uint32_t kKeyMask = 0x7FFFFFFFu;
constexpr int kWarps = kPushThreads / 32;

/* ---- shared-memory accumulators (structure of arrays) ----
 * Per group: signed sums of the low and high 16-bit halves of the inserted
 * minus retracted values of the current batch (exact for <= 8192 deltas),
 * an int64 running sum they are folded into, insert and retract counts,
 * extrema of the inserted values, and the front raise / lower values. */
enum Field { A_LO = 0, A_HI, A_INS, A_RET, A_IMIN, A_IMAX, A_FRAISE, A_FLOWER, A_NUM };

struct Acc {
    int32_t *w;          /* A_NUM arrays of `stride` words */
    long long *acc64;    /* folded sums */
    int stride;
    __device__ __forceinline__ int32_t *f(int field, int i) const { return w + field * stride + i; }
};

__device__ __forceinline__ void acc_init(const Acc &a, int i) {
    *a.f(A_LO, i) = 0;
    *a.f(A_HI, i) = 0;
    *a.f(A_INS, i) = 0;
    *a.f(A_RET, i) = 0;
    *a.f(A_IMIN, i) = INT32_MAX;
    *a.f(A_IMAX, i) = INT32_MIN;
    *a.f(A_FRAISE, i) = INT32_MIN;
    *a.f(A_FLOWER, i) = INT32_MAX;
    a.acc64[i] = 0;
}

/* v = (v >> 16) * 65536 + (v & 0xFFFF) for every int32 v (arithmetic shift) */
template <bool MINMAX>
__device__ __forceinline__ void acc_insert(const Acc &a, int i, int32_t v) {
    atomicAdd(a.f(A_LO, i), v & 0xFFFF);
    atomicAdd(a.f(A_HI, i), v >> 16);
    atomicAdd(a.f(A_INS, i), 1);
    if (MINMAX) {
        atomicMin(a.f(A_IMIN, i), v);
        atomicMax(a.f(A_IMAX, i), v);
    }
}

template <bool FRONT>
__device__ __forceinline__ void acc_retract(const Acc &a, int i, int32_t v, int32_t smin, int32_t smax) {
    atomicAdd(a.f(A_LO, i), -(v & 0xFFFF));
    atomicAdd(a.f(A_HI, i), -(v >> 16));
    atomicAdd(a.f(A_RET, i), 1);
    if (FRONT && (smin != INT32_MIN || smax != INT32_MAX)) {
        atomicMax(a.f(A_FRAISE, i), smin);
        atomicMin(a.f(A_FLOWER, i), smax);
    }
}

/* fold the batch's half sums into the int64 sum (caller owns entry i) */
__device__ __forceinline__ void acc_fold(const Acc &a, int i) {
    a.acc64[i] += (long long)*a.f(A_HI, i) * 65536LL + (long long)*a.f(A_LO, i);
    *a.f(A_LO, i) = 0;
    *a.f(A_HI, i) = 0;
}

/* ---- hot-key hash (key -> index in the hot list) ---- */
constexpr int kHotSlots = 512;

__device__ __forceinline__ uint32_t hot_hash(int32_t k) {
    uint32_t x = (uint32_t)k * 0x9E3779B1u;
    return (x ^ (x >> 15)) & (kHotSlots - 1);
}

__device__ __forceinline__ int hot_find(const int32_t *hkey, const int16_t *hidx, int32_t k) {
    uint32_t s = hot_hash(k);
    for (int probe = 0; probe < kHotSlots; probe++) {
        int32_t x = hkey[s];
        if (x == k) return hidx[s];
        if (x == -1) return -1;
        s = (s + 1) & (kHotSlots - 1);
    }
    return -1;
}

/* ---- block-wide exclusive scan of an smem array of n words, in place;
 * a[n] receives the total, which is also returned ---- */
__device__ uint32_t block_scan_inplace(uint32_t *a, int n) {
    __shared__ uint32_t wsum[kWarps];
    __shared__ uint32_t tot;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + kPushThreads - 1) / kPushThreads;
    const int b0 = tid * per;
    uint32_t s = 0;
    for (int j = 0; j < per; j++)
        if (b0 + j < n) s += a[b0 + j];
    uint32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kWarps ? wsum[lane] : 0;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kWarps) wsum[lane] = wi - w;
        if (lane == kWarps - 1) tot = wi;
    }
    __syncthreads();
    uint32_t run = wsum[warp] + incl - s;
    for (int j = 0; j < per; j++)
        if (b0 + j < n) {
            uint32_t x = a[b0 + j];
            a[b0 + j] = run;
            run += x;
        }
    const uint32_t total = tot;
    __syncthreads();
    if (tid == 0) a[n] = total;
    __syncthreads();
    return total;
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

/* Grid barrier over a monotonic counter; gives up after ~2 s.  Thread 0 of
 * each CTA publishes its CTA's writes with a release add and polls with
 * acquire loads. */
__device__ bool grid_barrier(unsigned long long *bar, unsigned long long target) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(bar) : "memory");
        unsigned long long t0 = globaltimer();
        int good = 1;
        for (unsigned it = 0;; it++) {
            unsigned long long v;
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(bar) : "memory");
            if (v >= target) break;
            if ((it & 63) == 63) {
                if (globaltimer() - t0 > 2000000000ULL) {
                    good = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ void cp_async(uint2 *dst, const uint2 *src) {
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async(uint4 *dst, const uint4 *src) {
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

struct HotRec {
    long long sum;        /* inserted minus retracted values */
    int32_t ins, ret;
    int32_t imin, imax, fraise, flower;
};

template <typename D>
struct DeltaIO;

template <>
struct DeltaIO<uint2> {
    static __device__ __forceinline__ uint2 make(uint32_t kf, int32_t v, int32_t, int32_t) {
        return make_uint2(kf, (uint32_t)v);
    }
    static __device__ __forceinline__ void get(uint2 d, uint32_t &kf, int32_t &v, int32_t &smin, int32_t &smax) {
        kf = d.x;
        v = (int32_t)d.y;
        smin = INT32_MIN;
        smax = INT32_MAX;
    }
};

template <>
struct DeltaIO<uint4> {
    static __device__ __forceinline__ uint4 make(uint32_t kf, int32_t v, int32_t smin, int32_t smax) {
        return make_uint4(kf, (uint32_t)v, (uint32_t)smin, (uint32_t)smax);
    }
    static __device__ __forceinline__ void get(uint4 d, uint32_t &kf, int32_t &v, int32_t &smin, int32_t &smax) {
        kf = d.x;
        v = (int32_t)d.y;
        smin = (int32_t)d.z;
        smax = (int32_t)d.w;
    }
};

__host__ __device__ constexpr int64_t pad16(int64_t x) { return (x + 15) / 16 * 16; }

/* Shared-memory layout: a fixed region (hot-key hash and accumulators) and a
 * region used by phase A (partition histogram, sorted chunk deltas) and then
 * by phase B (group table, batch of gathered deltas, per-chunk runs). */
struct Layout {
    int64_t hkey = 0, hidx, hlist, hw, h64, uni;
    int64_t a_hist, a_stage, a_end;
    int64_t b_acc64, b_w, b_dstage, b_segbeg, b_segoff, b_end;
    __host__ __device__ Layout(int P, int C, int tcap, int dcap, int dsize) {
        hidx = hkey + kHotSlots * 4;
        hlist = hidx + kHotSlots * 2;
        hw = hlist + kMaxHot * 4;
        h64 = hw + (int64_t)A_NUM * kMaxHot * 4;
        uni = h64 + kMaxHot * 8;
        a_hist = uni;
        a_stage = a_hist + pad16((int64_t)(P + 1) * 4);
        a_end = a_stage + 2 * (int64_t)kChunkCap * dsize;
        b_acc64 = uni;
        b_w = b_acc64 + (int64_t)tcap * 8;
        b_dstage = b_w + pad16((int64_t)A_NUM * tcap * 4);
        b_segbeg = b_dstage + (int64_t)dcap * dsize;
        b_segoff = b_segbeg + pad16((int64_t)C * 4);
        b_end = b_segoff + pad16((int64_t)(C + 1) * 4);
    }
    __host__ __device__ int64_t total() const { return a_end > b_end ? a_end : b_end; }
};

template <bool MINMAX, bool FRONT>
__global__ void __launch_bounds__(kPushThreads, 1) push_kernel(PushArgs a) {
    typedef typename std::conditional<FRONT, uint4, uint2>::type Delta;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = a.P;
    const Layout L(P, a.C, a.tcap, a.dcap, (int)sizeof(Delta));
    int32_t *hkey = (int32_t *)(smem + L.hkey);
    int16_t *hidx = (int16_t *)(smem + L.hidx);
    int32_t *hlist = (int32_t *)(smem + L.hlist);
    const Acc hacc{(int32_t *)(smem + L.hw), (long long *)(smem + L.h64), kMaxHot};

    if (*(volatile int *)a.err) return;   /* only earlier launches write err before the barrier */
    unsigned long long *trace = a.trace ? a.trace + (int64_t)blockIdx.x * 8 : nullptr;
    if (trace && tid == 0) trace[0] = globaltimer();

    if (blockIdx.x == 0 && tid == 0) *a.hot_next_n = 0;
    const int n_hot = min(*a.hot_cur_n, a.hot_cap);
    for (int s = tid; s < kHotSlots; s += kPushThreads) hkey[s] = -1;
    __syncthreads();
    for (int h = tid; h < n_hot; h += kPushThreads) {
        const int32_t k = a.hot_cur[h];
        hlist[h] = k;
        acc_init(hacc, h);
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
    __syncthreads();
    if (trace && tid == 0) trace[1] = globaltimer();

    /* ---------------- phase A ---------------- */
    uint32_t *hist = (uint32_t *)(smem + L.a_hist);   /* P + 1 words */
    Delta *stage_s = (Delta *)(smem + L.a_stage);     /* 2 * kChunkCap deltas */
    int local_err = 0;
    for (int round = 0; round < a.rounds; round++) {
        const int c = round * a.grid + blockIdx.x;
        const int64_t cbeg = (int64_t)c * a.S;
        int64_t cend = cbeg + a.S;
        if (cend > a.n) cend = a.n;
        for (int p = tid; p <= P; p += kPushThreads) hist[p] = 0;
        __syncthreads();
        int32_t k[kTPT], v[kTPT], ok[kTPT], ov[kTPT], smn[kTPT], smx[kTPT];
        bool has[kTPT], old[kTPT];
#pragma unroll
        for (int j = 0; j < kTPT; j++) {
            const int64_t i = cbeg + j * kPushThreads + tid;
            has[j] = i < cend;
            int64_t sl = a.slot0 + i;
            if (sl >= a.W) sl -= a.W;
            int64_t rel = sl - a.hmod;
            if (rel < 0) rel += a.W;
            old[j] = has[j] && rel < a.old_len;
            const bool fr = FRONT && old[j] && rel >= a.fa && rel < a.fb;
            k[j] = has[j] ? __ldcs(a.keys + i) : 0;
            v[j] = has[j] ? __ldcs(a.vals + i) : 0;
            ok[j] = old[j] ? a.ring_k[sl] : 0;
            ov[j] = old[j] ? a.ring_v[sl] : 0;
            smn[j] = INT32_MIN;
            smx[j] = INT32_MAX;
            if (FRONT && fr) {
                smn[j] = a.sufmin[sl];
                smx[j] = a.sufmax[sl];
            }
        }
        uint32_t pr[2 * kTPT];   /* partition << 16 | rank, or ~0 when hot / absent */
#pragma unroll
        for (int j = 0; j < kTPT; j++) {
            pr[2 * j] = 0xFFFFFFFFu;
            pr[2 * j + 1] = 0xFFFFFFFFu;
            if (has[j]) {
                int64_t sl = a.slot0 + cbeg + j * kPushThreads + tid;
                if (sl >= a.W) sl -= a.W;
                a.ring_k[sl] = k[j];
                a.ring_v[sl] = v[j];
                if ((uint32_t)k[j] >= (uint32_t)a.G) {
                    local_err = 1;
                } else {
                    const int h = n_hot ? hot_find(hkey, hidx, k[j]) : -1;
                    if (h >= 0) {
                        acc_insert<MINMAX>(hacc, h, v[j]);
                    } else {
                        const uint32_t p = (uint32_t)k[j] >> a.rbits;
                        pr[2 * j] = (p << 16) | atomicAdd(&hist[p], 1u);
                    }
                }
            }
            if (old[j] && (uint32_t)ok[j] < (uint32_t)a.G) {
                const int h = n_hot ? hot_find(hkey, hidx, ok[j]) : -1;
                if (h >= 0) {
                    acc_retract<FRONT>(hacc, h, ov[j], smn[j], smx[j]);
                } else {
                    const uint32_t p = (uint32_t)ok[j] >> a.rbits;
                    pr[2 * j + 1] = (p << 16) | atomicAdd(&hist[p], 1u);
                }
            }
        }
        __syncthreads();
        for (int h = tid; h < n_hot; h += kPushThreads) acc_fold(hacc, h);
        const uint32_t total = block_scan_inplace(hist, P);
        uint32_t *off_row = a.off + (int64_t)c * (P + 1);
        for (int p = tid; p <= P; p += kPushThreads) off_row[p] = hist[p];
#pragma unroll
        for (int j = 0; j < kTPT; j++) {
            if (pr[2 * j] != 0xFFFFFFFFu) {
                const uint32_t p = pr[2 * j] >> 16;
                stage_s[hist[p] + (pr[2 * j] & 0xFFFFu)] = DeltaIO<Delta>::make((uint32_t)k[j], v[j], 0, 0);
            }
            if (pr[2 * j + 1] != 0xFFFFFFFFu) {
                const uint32_t p = pr[2 * j + 1] >> 16;
                stage_s[hist[p] + (pr[2 * j + 1] & 0xFFFFu)] =
                    DeltaIO<Delta>::make((uint32_t)ok[j] | kRetract, ov[j], smn[j], smx[j]);
            }
        }
        __syncthreads();
        Delta *stage_g = (Delta *)a.stage + (int64_t)c * (2 * a.S);
        for (uint32_t i = tid; i < total; i += kPushThreads) stage_g[i] = stage_s[i];
        __syncthreads();
    }
    if (trace && tid == 0) trace[2] = globaltimer();
    /* heavy hitters: one partial record per CTA */
    HotRec *hotpart = (HotRec *)a.hotpart;
    for (int h = tid; h < n_hot; h += kPushThreads) {
        HotRec r;
        r.sum = hacc.acc64[h];
        r.ins = *hacc.f(A_INS, h);
        r.ret = *hacc.f(A_RET, h);
        r.imin = *hacc.f(A_IMIN, h);
        r.imax = *hacc.f(A_IMAX, h);
        r.fraise = *hacc.f(A_FRAISE, h);
        r.flower = *hacc.f(A_FLOWER, h);
        hotpart[(int64_t)h * a.grid + blockIdx.x] = r;
    }

    if (!grid_barrier(a.bar, a.bar_target)) {
        if (tid == 0) {
            atomicOr(a.err, 2);
            if (a.err_host) *(volatile int *)a.err_host = 2;
        }
        return;
    }
    if (trace && tid == 0) trace[3] = globaltimer();
    if (__syncthreads_or(local_err) && tid == 0) {
        atomicOr(a.err, 1);
        if (a.err_host) *(volatile int *)a.err_host = 1;
    }
    /* Deltas of bad keys were dropped; a poisoned query's results are
       undefined, so phase B still runs to keep the launch uniform. */

    /* ---------------- phase B ---------------- */
    const Acc tab{(int32_t *)(smem + L.b_w), (long long *)(smem + L.b_acc64), a.tcap};
    Delta *dstage = (Delta *)(smem + L.b_dstage);
    uint32_t *segbeg = (uint32_t *)(smem + L.b_segbeg);   /* C */
    uint32_t *segoff = (uint32_t *)(smem + L.b_segoff);   /* C + 1 */
    const Delta *stage = (const Delta *)a.stage;
    const int pb = (int)((int64_t)P * blockIdx.x / a.grid);
    const int pe = (int)((int64_t)P * (blockIdx.x + 1) / a.grid);
    for (int q0 = pb; q0 < pe; q0 += a.ppp) {
        const int q1 = min(pe, q0 + a.ppp);
        const int64_t g0 = (int64_t)q0 << a.rbits;
        const int64_t g1 = min((int64_t)q1 << a.rbits, a.G);
        const int range = (int)(g1 - g0);
        for (int l = tid; l < range; l += kPushThreads) acc_init(tab, l);
        for (int c = tid; c < a.C; c += kPushThreads) {
            const uint32_t *row = a.off + (int64_t)c * (P + 1);
            const uint32_t lo = row[q0], hi = row[q1];
            segbeg[c] = lo;
            segoff[c] = hi - lo;
        }
        __syncthreads();
        const uint32_t total = block_scan_inplace(segoff, a.C);
        for (uint32_t b0 = 0; b0 < total; b0 += (uint32_t)a.dcap) {
            const uint32_t b1 = min(total, b0 + (uint32_t)a.dcap);
            /* gather the batch's deltas: warp per chunk run, lanes along the run */
            for (int c = warp; c < a.C; c += kWarps) {
                const uint32_t s0 = segoff[c], s1 = segoff[c + 1];
                const uint32_t lo = max(s0, b0), hi = min(s1, b1);
                const Delta *src = stage + (int64_t)c * (2 * a.S) + segbeg[c];
                for (uint32_t x = lo + lane; x < hi; x += 32) cp_async(dstage + (x - b0), src + (x - s0));
            }
            cp_async_wait_all();
            __syncthreads();
            for (uint32_t i = tid; i < b1 - b0; i += kPushThreads) {
                uint32_t kf;
                int32_t dv, smin, smax;
                DeltaIO<Delta>::get(dstage[i], kf, dv, smin, smax);
                const int l = (int)((int64_t)(kf & kKeyMask) - g0);
                if (l < 0 || l >= range) continue;   /* bounds guard; a valid run never triggers it */
                if (kf & kRetract) acc_retract<FRONT>(tab, l, dv, smin, smax);
                else acc_insert<MINMAX>(tab, l, dv);
            }
            __syncthreads();
            for (int l = tid; l < range; l += kPushThreads) acc_fold(tab, l);
            __syncthreads();
        }
        if (trace && tid == 0) trace[4] = globaltimer();
        /* heavy hitters of this range: fold in their per-CTA records */
        for (int h = warp; h < n_hot; h += kWarps) {
            const int32_t key = hlist[h];
            if ((int64_t)key < g0 || (int64_t)key >= g1) continue;
            long long s = 0;
            int32_t ins = 0, ret = 0;
            int32_t imin = INT32_MAX, imax = INT32_MIN, fra = INT32_MIN, flo = INT32_MAX;
            for (int c = lane; c < a.grid; c += 32) {
                const HotRec r = hotpart[(int64_t)h * a.grid + c];
                s += r.sum;
                ins += r.ins;
                ret += r.ret;
                imin = min(imin, r.imin);
                imax = max(imax, r.imax);
                fra = max(fra, r.fraise);
                flo = min(flo, r.flower);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                s += __shfl_xor_sync(kFull, s, o);
                ins += __shfl_xor_sync(kFull, ins, o);
                ret += __shfl_xor_sync(kFull, ret, o);
                imin = min(imin, __shfl_xor_sync(kFull, imin, o));
                imax = max(imax, __shfl_xor_sync(kFull, imax, o));
                fra = max(fra, __shfl_xor_sync(kFull, fra, o));
                flo = min(flo, __shfl_xor_sync(kFull, flo, o));
            }
            if (lane == 0) {
                const int l = (int)(key - g0);
                tab.acc64[l] += s;
                *tab.f(A_INS, l) += ins;
                *tab.f(A_RET, l) += ret;
                *tab.f(A_IMIN, l) = min(*tab.f(A_IMIN, l), imin);
                *tab.f(A_IMAX, l) = max(*tab.f(A_IMAX, l), imax);
                *tab.f(A_FRAISE, l) = max(*tab.f(A_FRAISE, l), fra);
                *tab.f(A_FLOWER, l) = min(*tab.f(A_FLOWER, l), flo);
            }
        }
        __syncthreads();
        /* finalise the range's groups */
        for (int l = tid; l < range; l += kPushThreads) {
            const int32_t ins = *tab.f(A_INS, l), ret = *tab.f(A_RET, l);
            if (ins + ret == 0) continue;
            const int64_t g = g0 + l;
            const long long s = (long long)a.sum[g] + tab.acc64[l];
            const int32_t cn = a.cnt[g] + (ins - ret);
            a.sum[g] = (unsigned long long)s;
            a.cnt[g] = cn;
            if (MINMAX) {
                const int32_t imin = *tab.f(A_IMIN, l), imax = *tab.f(A_IMAX, l);
                int32_t blo = untag_dn(a.bmin[g], a.epoch, INT32_MAX);
                int32_t bhi = untag_up(a.bmax[g], a.epoch, INT32_MIN);
                if (ins) {
                    blo = min(blo, imin);
                    bhi = max(bhi, imax);
                    a.bmin[g] = tag_dn(a.epoch, blo);
                    a.bmax[g] = tag_up(a.epoch, bhi);
                }
                /* A front with live tags exists only in pushes that expire
                   front tuples (FRONT); otherwise it decodes empty. */
                int32_t flo_v = INT32_MAX, fhi_v = INT32_MIN;
                if (FRONT) {
                    const int32_t fra = *tab.f(A_FRAISE, l), flo = *tab.f(A_FLOWER, l);
                    const unsigned long long tf_lo = a.fmin[g], tf_hi = a.fmax[g];
                    flo_v = untag_up(tf_lo, a.epoch, INT32_MAX);
                    fhi_v = untag_dn(tf_hi, a.epoch, INT32_MIN);
                    if ((uint32_t)(tf_lo >> 32) == a.epoch && fra > flo_v) {
                        flo_v = fra;
                        a.fmin[g] = tag_up(a.epoch, flo_v);
                    }
                    if ((uint32_t)(tf_hi >> 32) == ~a.epoch && flo < fhi_v) {
                        fhi_v = flo;
                        a.fmax[g] = tag_dn(a.epoch, fhi_v);
                    }
                }
                a.rmin[g] = cn > 0 ? min(blo, flo_v) : INT32_MAX;
                a.rmax[g] = cn > 0 ? max(bhi, fhi_v) : INT32_MIN;
            }
            if (a.avg) {
                a.ravg[g] = cn > 0 ? __ddiv_rn(__ll2double_rn(s), (double)cn)
                                   : __longlong_as_double(0x7FF8000000000000LL);
            }
            if (a.hot_cap && (uint32_t)ins >= a.hot_threshold) {
                const int idx = atomicAdd(a.hot_next_n, 1);
                if (idx < a.hot_cap) a.hot_next[idx] = (int32_t)g;
            }
        }
        __syncthreads();
    }
    if (trace && tid == 0) trace[5] = globaltimer();
}

}  // namespace

int64_t push_smem_bytes(const PushPlan &pl, bool front) {
    return Layout(pl.P, pl.C, pl.tcap, pl.dcap, front ? 16 : 8).total();
}

int push_delta_cap(bool front) { return front ? 4096 : 8192; }

const void *push_kernel_ptr(bool minmax, bool front) {
    if (front) return (const void *)push_kernel<true, true>;
    if (minmax) return (const void *)push_kernel<true, false>;
    return (const void *)push_kernel<false, false>;
}

int64_t hot_rec_bytes() { return sizeof(HotRec); }

}  // namespace cq
