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

#include "cq_heavy.cuh"
#include "cq_internal.h"
#include "cq_push.cuh"
#include "cq_push_dev.cuh"
#include "cq_avg.cuh"
#include "cq_tags.cuh"
#include "cq_tma.cuh"

namespace cq {

namespace {

using namespace pushdev;
constexpr int kWarps = kPushThreads / 32;

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
        a_end = a_stage + (2 * (int64_t)kChunkCap + P + 2) * dsize;   /* runs padded to even lengths */
        b_acc64 = uni;
        b_w = b_acc64 + pad16((int64_t)tcap * 8);   /* keeps the gather staging 16-byte aligned */
        b_dstage = b_w + pad16((int64_t)A_NUM * tcap * 4);
        b_segbeg = b_dstage + (int64_t)dcap * dsize;
        b_segoff = b_segbeg + pad16((int64_t)C * 4);
        b_end = b_segoff + pad16((int64_t)(C + 1) * 4);
    }
    __host__ __device__ int64_t total() const { return a_end > b_end ? a_end : b_end; }
};

template <bool MINMAX, bool FRONT>
__global__ void __launch_bounds__(kPushThreads, 1) push_kernel(PushArgs a) {
    typedef uint2 Delta;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = a.P;
    const Layout L(P, a.C, a.tcap, a.dcap, (int)sizeof(Delta));
    int32_t *hkey = (int32_t *)(smem + L.hkey);
    int16_t *hidx = (int16_t *)(smem + L.hidx);
    int32_t *hlist = (int32_t *)(smem + L.hlist);
    const Acc hacc{(int32_t *)(smem + L.hw), (long long *)(smem + L.h64), kMaxHot};
    __shared__ int s_nheavy;                 /* partitions of the chunk far above their share */
    __shared__ uint32_t s_heavy[kHeavyList];
    __shared__ int32_t s_emkey[kEmSlots];     /* the keys found heavy within this push */
    __shared__ unsigned long long s_gbar;     /* phase-B gathers (bulk copies) */
    __shared__ int s_gfail;
    __shared__ uint32_t s_odd[kMaxParts / 32];   /* partitions whose run has a padding delta */

    if (*(volatile int *)a.err) return;   /* only earlier launches write err before the barrier */
    unsigned long long *trace = a.trace ? a.trace + (int64_t)blockIdx.x * 8 : nullptr;
    if (trace && tid == 0) trace[0] = globaltimer();

    if (blockIdx.x == 0 && tid == 0) {
        a.hot_next_n[0] = 0;
        a.hot_next_n[1] = 0;
    }
    if (tid == 0) {
        tma::mbar_init(&s_gbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_gfail = 0;
    }
    /* the list's keys sure of a slot, then the others up to the cap */
    const int n1 = min(a.hot_cur_n[0], a.hot_cap);
    const int n_hot = n1 + min(a.hot_cur_n[1], a.hot_cap - n1);
    for (int s = tid; s < kHotSlots; s += kPushThreads) hkey[s] = -1;
    __syncthreads();
    for (int h = tid; h < n_hot; h += kPushThreads) {
        const int32_t k = a.hot_cur[h < n1 ? h : kMaxHot + (h - n1)];
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
    /* a chunk's new tuples and the ring slots they overwrite, loaded into
       registers; the next chunk's loads are issued once the current chunk's
       deltas are in shared memory, so they overlap its store */
    int32_t k[kTPT], v[kTPT], ok[kTPT], ov[kTPT];
    bool has[kTPT], old[kTPT], frd[kTPT];
    const auto load_chunk = [&](int round) {
        const int64_t cbeg = (int64_t)(round * a.grid + blockIdx.x) * a.S;
        const int64_t cend = min(cbeg + a.S, a.n);
#pragma unroll
        for (int j = 0; j < kTPT; j++) {
            const int64_t i = cbeg + j * kPushThreads + tid;
            has[j] = i < cend;
            int64_t sl = a.slot0 + i;
            if (sl >= a.W) sl -= a.W;
            int64_t rel = sl - a.hmod;
            if (rel < 0) rel += a.W;
            old[j] = has[j] && rel < a.old_len;
            frd[j] = FRONT && old[j] && rel >= a.fa && rel < a.fb;   /* leaves the front */
            k[j] = has[j] ? __ldcs(a.keys + i) : 0;
            v[j] = has[j] ? __ldcs(a.vals + i) : 0;
            ok[j] = old[j] ? a.ring_k[sl] : 0;
            ov[j] = old[j] ? a.ring_v[sl] : 0;
        }
    };
    if (a.rounds > 0) load_chunk(0);
    for (int round = 0; round < a.rounds; round++) {
        const int c = round * a.grid + blockIdx.x;
        const int64_t cbeg = (int64_t)c * a.S;
        for (int p = tid; p <= P; p += kPushThreads) hist[p] = 0;
        if (tid == 0) s_nheavy = 0;
        __syncthreads();
        const uint32_t heavy_t = a.heavy_bound;
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
                        const uint32_t o = atomicAdd(&hist[p], 1u);
                        if (o == heavy_t) note_heavy(s_heavy, &s_nheavy, p);
                        pr[2 * j] = (p << 16) | o;
                    }
                }
            }
            if (old[j] && (uint32_t)ok[j] < (uint32_t)a.G) {
                const int h = n_hot ? hot_find(hkey, hidx, ok[j]) : -1;
                if (h >= 0) {
                    acc_retract(hacc, h, ov[j], frd[j]);
                } else {
                    const uint32_t p = (uint32_t)ok[j] >> a.rbits;
                    const uint32_t o = atomicAdd(&hist[p], 1u);
                    if (o == heavy_t) note_heavy(s_heavy, &s_nheavy, p);
                    pr[2 * j + 1] = (p << 16) | o;
                }
            }
        }
        __syncthreads();
        for (int h = tid; h < n_hot; h += kPushThreads) acc_fold(hacc, h);
        /* every run padded to an even length, so that each starts on a
           16-byte boundary and phase B takes it by one bulk copy */
        for (int w = tid; w < kMaxParts / 32; w += kPushThreads) s_odd[w] = 0u;
        __syncthreads();
        for (int p = tid; p < P; p += kPushThreads)
            if (hist[p] & 1u) {
                hist[p] += 1u;
                atomicOr(&s_odd[p >> 5], 1u << (p & 31));
            }
        const uint32_t total = block_scan_inplace<kPushThreads>(hist, P);
        uint32_t *off_row = a.off + (int64_t)c * (P + 1);
        for (int p = tid; p <= P; p += kPushThreads) off_row[p] = hist[p];
#pragma unroll
        for (int j = 0; j < kTPT; j++) {
            if (pr[2 * j] != 0xFFFFFFFFu) {
                const uint32_t p = pr[2 * j] >> 16;
                stage_s[hist[p] + (pr[2 * j] & 0xFFFFu)] = DeltaIO::make((uint32_t)k[j], v[j]);
            }
            if (pr[2 * j + 1] != 0xFFFFFFFFu) {
                const uint32_t p = pr[2 * j + 1] >> 16;
                stage_s[hist[p] + (pr[2 * j + 1] & 0xFFFFu)] =
                    DeltaIO::make((uint32_t)ok[j] | kRetract | (frd[j] ? kFrontDep : 0u), ov[j]);
            }
        }
        for (int p = tid; p < P; p += kPushThreads)
            if ((s_odd[p >> 5] >> (p & 31)) & 1u) stage_s[hist[p + 1] - 1] = DeltaIO::make(kPadWord, 0);
        if (round + 1 < a.rounds) load_chunk(round + 1);
        __syncthreads();
        /* runs far above their share: a key heavy within this push (cq_heavy.cuh) */
        const int n_heavy = min(s_nheavy, kHeavyList);
        if (n_heavy > 0) {
            for (int j = warp; j < n_heavy; j += kWarps) {
                const uint32_t p = s_heavy[j];
                fold_heavy_run(stage_s + hist[p], hist[p + 1] - hist[p], a.heavy_min, c & (kHotRep - 1),
                                      a.emkey, (HotAcc *)a.emacc, a.emfolds, MINMAX);
            }
            __syncthreads();
        }
        Delta *stage_g = (Delta *)a.stage + (int64_t)c * a.stride;
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
        r.fdep = *hacc.f(A_FDEP, h);
        r.pad_ = 0;
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
    /* phase A's plain stores (staged runs) and shared-memory use come
       before the bulk copies of phase B */
    tma::fence_async_global();
    tma::fence_async_smem();
    uint32_t g_parity = 0;

    /* ---------------- phase B ---------------- */
    const Acc tab{(int32_t *)(smem + L.b_w), (long long *)(smem + L.b_acc64), a.tcap};
    Delta *dstage = (Delta *)(smem + L.b_dstage);
    uint32_t *segbeg = (uint32_t *)(smem + L.b_segbeg);   /* C */
    uint32_t *segoff = (uint32_t *)(smem + L.b_segoff);   /* C + 1 */
    const Delta *stage = (const Delta *)a.stage;
    /* key ranges of ppp partitions drawn from a counter, so that a CTA whose
       ranges hold many deltas takes fewer of them */
    __shared__ int s_draw;
    const int R = (P + a.ppp - 1) / a.ppp;
    const auto draw = [&]() -> int {
        __syncthreads();
        if (tid == 0) s_draw = (int)(atomicAdd(a.bar + 1, 1ULL) - a.draw_base);
        __syncthreads();
        return s_draw;
    };
    for (int r = draw(); r >= 0 && r < R; r = draw()) {   /* (r < 0 only after a launch that gave up) */
        const int q0 = r * a.ppp;
        const int q1 = min(P, q0 + a.ppp);
        const int64_t g0 = (int64_t)q0 << a.rbits;
        const int64_t g1 = min((int64_t)q1 << a.rbits, a.G);
        const int range = (int)(g1 - g0);
        for (int l = tid; l < range; l += kPushThreads) acc_init(tab, l);
        if (tid < kEmSlots) s_emkey[tid] = __ldcg(&a.emkey[tid]);   /* used after the range's deltas */
        for (int c = tid; c < a.C; c += kPushThreads) {
            const uint32_t *row = a.off + (int64_t)c * (P + 1);
            const uint32_t lo = row[q0], hi = row[q1];
            segbeg[c] = lo;
            segoff[c] = hi - lo;
        }
        __syncthreads();
        const uint32_t total = block_scan_inplace<kPushThreads>(segoff, a.C);
        for (uint32_t b0 = 0; b0 < total; b0 += (uint32_t)a.dcap) {
            const uint32_t b1 = min(total, b0 + (uint32_t)a.dcap);
            /* every run is padded to an even length (16-byte aligned), so
               each chunk's run comes in one bulk copy (a thread per chunk) */
            if (tid == 0) tma::mbar_expect(&s_gbar, (b1 - b0) * 8u);
            __syncthreads();
            for (int c = tid; c < a.C; c += kPushThreads) {
                const uint32_t s0 = segoff[c], s1 = segoff[c + 1];
                const uint32_t lo = max(s0, b0), hi = min(s1, b1);
                if (lo < hi)
                    tma::tma_load(dstage + (lo - b0), stage + (int64_t)c * a.stride + segbeg[c] + (lo - s0),
                                  (hi - lo) * 8u, &s_gbar);
            }
            if (tid == 0 && !tma::mbar_wait(&s_gbar, g_parity)) s_gfail = 1;
            g_parity ^= 1u;
            __syncthreads();
            if (s_gfail) {   /* a copy that never landed: the launch reports a timeout */
                if (tid == 0) {
                    atomicOr(a.err, 2);
                    if (a.err_host) *(volatile int *)a.err_host = 2;
                }
                return;
            }
            if (trace && tid == 0 && b0 == 0) trace[6] = globaltimer();
            for (uint32_t i = tid; i < b1 - b0; i += kPushThreads) {
                uint32_t kf;
                int32_t dv;
                DeltaIO::get(dstage[i], kf, dv);
                const int l = (int)((int64_t)(kf & kKeyMask) - g0);
                if (l < 0 || l >= range) continue;   /* padding, and a bounds guard */
                if (kf & kRetract) acc_retract(tab, l, dv, (kf & kFrontDep) != 0);
                else acc_insert<MINMAX>(tab, l, dv);
            }
            __syncthreads();
            if (trace && tid == 0 && b0 == 0) trace[7] = globaltimer();
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
            int32_t imin = INT32_MAX, imax = INT32_MIN, fdep = 0;
            for (int c = lane; c < a.grid; c += 32) {
                const HotRec r = hotpart[(int64_t)h * a.grid + c];
                s += r.sum;
                ins += r.ins;
                ret += r.ret;
                imin = min(imin, r.imin);
                imax = max(imax, r.imax);
                fdep += r.fdep;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                s += __shfl_xor_sync(kFull, s, o);
                ins += __shfl_xor_sync(kFull, ins, o);
                ret += __shfl_xor_sync(kFull, ret, o);
                imin = min(imin, __shfl_xor_sync(kFull, imin, o));
                imax = max(imax, __shfl_xor_sync(kFull, imax, o));
                fdep += __shfl_xor_sync(kFull, fdep, o);
            }
            if (lane == 0) {
                const int l = (int)(key - g0);
                tab.acc64[l] += s;
                *tab.f(A_INS, l) += ins;
                *tab.f(A_RET, l) += ret;
                *tab.f(A_IMIN, l) = min(*tab.f(A_IMIN, l), imin);
                *tab.f(A_IMAX, l) = max(*tab.f(A_IMAX, l), imax);
                *tab.f(A_FDEP, l) += fdep;
            }
        }
        /* keys found heavy within this push whose range this is */
        merge_heavy_slots(tab, g0, g1, s_emkey, a.emkey, (HotAcc *)a.emacc, warp, kWarps);
        __syncthreads();
        /* finalise the range's groups, two a thread at a time: every global
           load of both is issued before any is used (two round trips, the
           second only for the fronts' suffix extrema) */
        for (int l0 = tid; l0 < range; l0 += 2 * kPushThreads) {
            unsigned long long sum0[2], tb_lo[2], tb_hi[2], tf_lo[2], tf_hi[2];
            int32_t cnt0[2], dep[2], p_old[2], ins[2], ret[2];
            bool on[2];
#pragma unroll
            for (int u = 0; u < 2; u++) {
                const int l = l0 + u * kPushThreads;
                const int64_t g = g0 + l;
                on[u] = false;
                sum0[u] = tb_lo[u] = tb_hi[u] = tf_lo[u] = tf_hi[u] = 0;
                cnt0[u] = dep[u] = p_old[u] = ins[u] = ret[u] = 0;
                if (l < range) {
                    ins[u] = *tab.f(A_INS, l);
                    ret[u] = *tab.f(A_RET, l);
                    on[u] = ins[u] + ret[u] != 0;
                }
                if (on[u]) {
                    sum0[u] = a.sum[g];
                    cnt0[u] = a.cnt[g];
                    if (MINMAX) {
                        tb_lo[u] = a.bmin[g];
                        tb_hi[u] = a.bmax[g];
                    }
                    if (FRONT) {
                        dep[u] = *tab.f(A_FDEP, l);
                        tf_lo[u] = a.fmin[g];
                        tf_hi[u] = a.fmax[g];
                        if (dep[u] > 0) p_old[u] = a.fptr[g];
                    }
                }
            }
            /* the fronts that shrink: pointers moved, survivors' extrema requested */
            int2 nx[2];
#pragma unroll
            for (int u = 0; u < 2; u++) {
                nx[u] = make_int2(INT32_MAX, INT32_MIN);
                if (FRONT && on[u] && dep[u] > 0 && (uint32_t)(tf_lo[u] >> 32) == a.epoch)
                    nx[u] = front_advance(a.fptr, a.sufs, g0 + l0 + u * kPushThreads, p_old[u], dep[u]);
            }
#pragma unroll
            for (int u = 0; u < 2; u++) {
                if (!on[u]) continue;
                const int l = l0 + u * kPushThreads;
                const int64_t g = g0 + l;
                const long long s = (long long)sum0[u] + tab.acc64[l];
                const int32_t cn = cnt0[u] + (ins[u] - ret[u]);
                a.sum[g] = (unsigned long long)s;
                a.cnt[g] = cn;
                if (MINMAX) {
                    const int32_t imin = *tab.f(A_IMIN, l), imax = *tab.f(A_IMAX, l);
                    int32_t blo = untag_dn(tb_lo[u], a.epoch, INT32_MAX);
                    int32_t bhi = untag_up(tb_hi[u], a.epoch, INT32_MIN);
                    if (ins[u]) {
                        blo = min(blo, imin);
                        bhi = max(bhi, imax);
                        a.bmin[g] = tag_dn(a.epoch, blo);
                        a.bmax[g] = tag_up(a.epoch, bhi);
                    }
                    /* A front with live tags exists only in pushes that expire
                       front tuples (FRONT); otherwise it decodes empty. */
                    int32_t flo_v = INT32_MAX, fhi_v = INT32_MIN;
                    if (FRONT) {
                        flo_v = untag_up(tf_lo[u], a.epoch, INT32_MAX);
                        fhi_v = untag_dn(tf_hi[u], a.epoch, INT32_MIN);
                        if (dep[u] > 0 && (uint32_t)(tf_lo[u] >> 32) == a.epoch) {
                            flo_v = nx[u].x;
                            fhi_v = nx[u].y;
                            a.fmin[g] = tag_up(a.epoch, flo_v);
                            a.fmax[g] = tag_dn(a.epoch, fhi_v);
                        }
                    }
                    a.rmin[g] = cn > 0 ? min(blo, flo_v) : INT32_MAX;
                    a.rmax[g] = cn > 0 ? max(bhi, fhi_v) : INT32_MIN;
                }
                if (a.avg) {
                    a.ravg[g] = cn > 0 ? avg_rn(s, cn)
                                       : __longlong_as_double(0x7FF8000000000000LL);
                }
                if (a.hot_cap && (uint32_t)ins[u] >= a.hot_threshold) {
                    const int tier = (uint32_t)ins[u] >= a.hot_gthr ? 0 : 1;
                    const int idx = atomicAdd(a.hot_next_n + tier, 1);
                    if (idx < a.hot_cap) {
                        a.hot_next[tier * kMaxHot + idx] = (int32_t)g;
                        a.hot_next_cnt[tier * kMaxHot + idx] = ins[u];
                    }
                }
            }
        }
        __syncthreads();
    }
    if (trace && tid == 0) trace[5] = globaltimer();
}

}  // namespace

int64_t push_smem_bytes(const PushPlan &pl, bool front) {
    (void)front;
    return Layout(pl.P, pl.C, pl.tcap, pl.dcap, 8).total();
}

int push_delta_cap(bool front) {
    (void)front;
    return 8192;
}

const void *push_kernel_ptr(bool minmax, bool front) {
    if (front) return (const void *)push_kernel<true, true>;
    if (minmax) return (const void *)push_kernel<true, false>;
    return (const void *)push_kernel<false, false>;
}

int64_t hot_rec_bytes() { return sizeof(HotRec); }

}  // namespace cq
