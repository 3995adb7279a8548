/*
 * cq_push_tma.cu -- the partitioned push with TMA-staged data movement.
 *
 * Same algorithm as cq_push.cu (phase A: fold heavy hitters privately and
 * counting-sort every other update of a chunk by key-range partition; grid
 * barrier; phase B: each CTA aggregates its key range in shared memory and
 * finalises its groups), with the bulk data moved by the Tensor Memory
 * Accelerator instead of per-thread loads:
 *   - a chunk's new keys and values and the ring slots they overwrite (and,
 *     when the front shrinks, the slots' suffix extrema) arrive in shared
 *     memory by cp.async.bulk, completed on an mbarrier;
 *   - the new tuples go back to the ring by a bulk store from shared memory;
 *   - the chunk's partition-sorted updates leave by one bulk store; every
 *     partition's run is padded to 16 bytes with an inert delta so that
 *   - phase B gathers each chunk's run of its key range with one bulk load;
 *   - the state of the key range (SUM, COUNT, epoch-tagged extrema) is
 *     prefetched by bulk loads while the updates are gathered.
 * Two CTAs of 512 threads share an SM, so one streams while the other
 * computes.  The launch requires 16-byte aligned batch pointers, a ring slot
 * of the first tuple that is a multiple of 4 and a window that is a multiple
 * of 4 (the host falls back to cq_push.cu otherwise).
 *
 * Every wait is bounded; a wait that gives up sets the query's error word
 * (timeout) and the CTA leaves after its own copies have drained.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "cq_internal.h"
#include "cq_push.cuh"
#include "cq_push_dev.cuh"
#include "cq_tags.cuh"

namespace cq {

namespace {

using namespace pushdev;

constexpr int kT = kTmaThreads;
constexpr int kW = kT / 32;
constexpr int kSCap = kTmaChunkCap;
constexpr uint32_t kDummy = 0x7FFFFFFFu;   /* key of padding deltas: never a group (G <= 2^31 - 1) */

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect(unsigned long long *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

/* Wait until the barrier's phase of the given parity completes; false after ~1 s. */
__device__ bool mbar_wait(unsigned long long *bar, uint32_t parity) {
    const uint32_t addr = smem_u32(bar);
    unsigned long long t0 = 0;
    for (uint32_t it = 0;; it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255) == 255) {
            const unsigned long long now = globaltimer();
            if (!t0) t0 = now;
            else if (now - t0 > 1000000000ULL) return false;
        }
    }
}

__device__ __forceinline__ void tma_load(void *dst, const void *src, uint32_t bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tma_store(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void tma_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void tma_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

/* Load elements [s, s + n) of a ring of W slots (n and s multiples of 4,
 * W a multiple of 4) into dst, in at most two bulk copies; returns bytes. */
template <typename T>
__device__ __forceinline__ uint32_t ring_load(T *dst, const T *ring, int64_t W, int64_t s, int64_t n,
                                              unsigned long long *bar) {
    if (n <= 0) return 0;
    const int64_t n1 = min(n, W - s);
    tma_load(dst, ring + s, (uint32_t)(n1 * sizeof(T)), bar);
    if (n > n1) tma_load(dst + n1, ring, (uint32_t)((n - n1) * sizeof(T)), bar);
    return (uint32_t)(n * sizeof(T));
}

template <typename T>
__device__ __forceinline__ void ring_store(T *ring, const T *src, int64_t W, int64_t s, int64_t n) {
    if (n <= 0) return;
    const int64_t n1 = min(n, W - s);
    tma_store(ring + s, src, (uint32_t)(n1 * sizeof(T)));
    if (n > n1) tma_store(ring, src + n1, (uint32_t)((n - n1) * sizeof(T)));
}

/* Shared-memory layout: fixed region (barriers, hot-key hash and
 * accumulators), then phase A (chunk inputs, partition counts and cursors,
 * sorted deltas) or phase B (group table, gathered deltas, per-chunk runs,
 * prefetched group state). */
struct TmaLayout {
    int64_t bars = 0, hkey, hidx, hlist, hw, h64, uni;
    int64_t a_k, a_v, a_rk, a_rv, a_smin, a_smax, a_flag, a_cnt, a_cur, a_stage, a_end;
    int64_t b_acc64, b_w, b_dstage, b_segbeg, b_segoff, b_sum, b_cnt, b_bmin, b_bmax, b_fmin, b_fmax, b_end;
    __host__ __device__ TmaLayout(int P, int C, int tcap, int dcap, int dsize, bool front) {
        hkey = bars + 64;
        hidx = hkey + kHotSlots * 4;
        hlist = hidx + kHotSlots * 2;
        hw = hlist + kMaxHot * 4;
        h64 = hw + (int64_t)A_NUM * kMaxHot * 4;
        uni = h64 + kMaxHot * 8;
        a_k = uni;
        a_v = a_k + kSCap * 4;
        a_rk = a_v + kSCap * 4;
        a_rv = a_rk + kSCap * 4;
        a_smin = a_rv + kSCap * 4;
        a_smax = a_smin + (front ? kSCap * 4 : 0);
        a_flag = a_smax + (front ? kSCap * 4 : 0);
        a_cnt = a_flag + kSCap;
        a_cur = a_cnt + pad16((int64_t)(P + 1) * 4);
        a_stage = a_cur + pad16((int64_t)(P + 1) * 4);
        a_end = a_stage + (int64_t)(2 * kSCap + P + 1) * dsize;
        b_acc64 = uni;
        b_w = b_acc64 + (int64_t)tcap * 8;
        b_dstage = b_w + pad16((int64_t)A_NUM * tcap * 4);
        b_segbeg = b_dstage + (int64_t)dcap * dsize;
        b_segoff = b_segbeg + pad16((int64_t)C * 4);
        b_sum = b_segoff + pad16((int64_t)(C + 1) * 4);
        b_cnt = b_sum + (int64_t)tcap * 8;
        b_bmin = b_cnt + pad16((int64_t)tcap * 4);
        b_bmax = b_bmin + (int64_t)tcap * 8;
        b_fmin = b_bmax + (int64_t)tcap * 8;
        b_fmax = b_fmin + (front ? (int64_t)tcap * 8 : 0);
        b_end = b_fmax + (front ? (int64_t)tcap * 8 : 0);
    }
    __host__ __device__ int64_t total() const { return a_end > b_end ? a_end : b_end; }
};

template <bool MINMAX, bool FRONT>
__global__ void __launch_bounds__(kT, 2) push_tma_kernel(PushArgs a) {
    typedef typename std::conditional<FRONT, uint4, uint2>::type Delta;
    constexpr int DS = (int)sizeof(Delta);
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = a.P;
    const TmaLayout L(P, a.C, a.tcap, a.dcap, DS, FRONT);
    unsigned long long *bars = (unsigned long long *)(smem + L.bars);   /* [0] inputs, [1] gather, [2] state */
    int32_t *hkey = (int32_t *)(smem + L.hkey);
    int16_t *hidx = (int16_t *)(smem + L.hidx);
    int32_t *hlist = (int32_t *)(smem + L.hlist);
    const Acc hacc{(int32_t *)(smem + L.hw), (long long *)(smem + L.h64), kMaxHot};

    if (*(volatile int *)a.err) return;   /* only earlier launches write err before the barrier */
    unsigned long long *trace = a.trace ? a.trace + (int64_t)blockIdx.x * 8 : nullptr;
    if (trace && tid == 0) trace[0] = globaltimer();

    int32_t *sk = (int32_t *)(smem + L.a_k);
    int32_t *sv = (int32_t *)(smem + L.a_v);
    int32_t *srk = (int32_t *)(smem + L.a_rk);
    int32_t *srv = (int32_t *)(smem + L.a_rv);
    int32_t *ssmin = (int32_t *)(smem + L.a_smin);
    int32_t *ssmax = (int32_t *)(smem + L.a_smax);
    /* bulk loads of chunk c's inputs (its first len4 tuples), issued by one thread */
    auto issue_chunk = [&](int c) {
        const int64_t cbeg = min((int64_t)c * a.S, a.n);
        const int64_t cend = min(cbeg + a.S, a.n);
        const int len4 = (int)(cend - cbeg) & ~3;
        if (len4 <= 0) return;
        int64_t s0 = a.slot0 + cbeg;
        if (s0 >= a.W) s0 -= a.W;
        mbar_expect(&bars[0], 16u * (uint32_t)len4 + (FRONT ? 8u * (uint32_t)len4 : 0u));
        tma_load(sk, a.keys + cbeg, 4u * len4, &bars[0]);
        tma_load(sv, a.vals + cbeg, 4u * len4, &bars[0]);
        ring_load(srk, a.ring_k, a.W, s0, len4, &bars[0]);
        ring_load(srv, a.ring_v, a.W, s0, len4, &bars[0]);
        if (FRONT) {
            ring_load(ssmin, a.sufmin, a.W, s0, len4, &bars[0]);
            ring_load(ssmax, a.sufmax, a.W, s0, len4, &bars[0]);
        }
    };
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (a.rounds > 0) issue_chunk(blockIdx.x);   /* chunk 0 streams in while the hot set loads */
    }
    if (blockIdx.x == 0 && tid == 0) *a.hot_next_n = 0;
    const int n_hot = min(*a.hot_cur_n, a.hot_cap);
    for (int s = tid; s < kHotSlots; s += kT) hkey[s] = -1;
    __syncthreads();
    for (int h = tid; h < n_hot; h += kT) {
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
    /* the heaviest hitter is accumulated in registers, the rest in shared memory */
    __shared__ int top_h;
    __shared__ long long wtop_sum[kW];
    __shared__ int32_t wtop_i[kW][6];   /* ins, ret, imin, imax, fraise, flower */
    if (warp == 0) {
        int best = -1, bestc = -1;
        for (int h = lane; h < n_hot; h += 32) {
            const int c = a.hot_cur_cnt[h];
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
        if (lane == 0) top_h = best;
    }
    __syncthreads();
    const int top = top_h;
    if (trace && tid == 0) trace[1] = globaltimer();

    /* ---------------- phase A ---------------- */
    uint8_t *flag = (uint8_t *)(smem + L.a_flag);
    uint32_t *cnt = (uint32_t *)(smem + L.a_cnt);
    uint32_t *cur = (uint32_t *)(smem + L.a_cur);
    Delta *stage_s = (Delta *)(smem + L.a_stage);
    int local_err = 0;
    bool timed_out = false;
    uint32_t in_parity = 0;
    for (int round = 0; round < a.rounds && !timed_out; round++) {
        const int c = round * a.grid + blockIdx.x;
        const int64_t cbeg = min((int64_t)c * a.S, a.n);
        const int64_t cend = min(cbeg + a.S, a.n);
        const int len = (int)(cend - cbeg);
        const int len4 = len & ~3;
        int64_t s0 = a.slot0 + cbeg;
        if (s0 >= a.W) s0 -= a.W;
        for (int p = tid; p <= P; p += kT) cnt[p] = 0;
        if (tid == 0 && round > 0) issue_chunk(c);   /* chunk 0 was issued in the prologue */
        if (tid < len - len4) {   /* ragged tail of the batch: plain loads */
            const int i = len4 + tid;
            int64_t sl = s0 + i;
            if (sl >= a.W) sl -= a.W;
            sk[i] = a.keys[cbeg + i];
            sv[i] = a.vals[cbeg + i];
            srk[i] = a.ring_k[sl];
            srv[i] = a.ring_v[sl];
            if (FRONT) {
                ssmin[i] = a.sufmin[sl];
                ssmax[i] = a.sufmax[sl];
            }
        }
        if (len4 > 0) {
            if (!mbar_wait(&bars[0], in_parity) && !mbar_wait(&bars[0], in_parity)) timed_out = true;
            in_parity ^= 1u;
        }
        __syncthreads();
        if (__syncthreads_or(timed_out)) {
            timed_out = true;
            break;
        }
        /* the new tuples go to the ring (their old occupants are in smem) */
        if (tid == 0 && len4 > 0) {
            fence_async_smem();
            ring_store(a.ring_k, sk, a.W, s0, len4);
            ring_store(a.ring_v, sv, a.W, s0, len4);
            tma_commit();
        }
        if (tid < len - len4) {
            const int i = len4 + tid;
            int64_t sl = s0 + i;
            if (sl >= a.W) sl -= a.W;
            a.ring_k[sl] = sk[i];
            a.ring_v[sl] = sv[i];
        }
        /* pass 1: heavy hitters into the private records, the others
           counted per partition; flag[i] remembers which of tuple i's two
           updates go through the partition exchange (bit 0: insert,
           bit 1: retract, bit 2: the retract leaves the front) */
        long long r_sum = 0;                 /* heaviest hitter: inserted minus retracted */
        int32_t r_ins = 0, r_ret = 0;
        int32_t r_imin = INT32_MAX, r_imax = INT32_MIN, r_fra = INT32_MIN, r_flo = INT32_MAX;
        for (int i = tid; i < len; i += kT) {
            uint32_t sl = (uint32_t)s0 + (uint32_t)i;
            if (sl >= (uint32_t)a.W) sl -= (uint32_t)a.W;
            int32_t rel = (int32_t)sl - (int32_t)a.hmod;
            if (rel < 0) rel += (int32_t)a.W;
            uint32_t f = 0;
            const int32_t k = sk[i];
            if ((uint32_t)k >= (uint32_t)a.G) {
                local_err = 1;
            } else {
                const int h = n_hot ? hot_find(hkey, hidx, k) : -1;
                if (h == top && h >= 0) {
                    const int32_t v = sv[i];
                    r_sum += v;
                    r_ins++;
                    r_imin = min(r_imin, v);
                    r_imax = max(r_imax, v);
                } else if (h >= 0) {
                    acc_insert<MINMAX>(hacc, h, sv[i]);
                } else {
                    atomicAdd(&cnt[(uint32_t)k >> a.rbits], 1u);
                    f = 1;
                }
            }
            if (rel < (int32_t)a.old_len) {
                const int32_t ok = srk[i];
                if ((uint32_t)ok < (uint32_t)a.G) {
                    const bool fr = FRONT && rel >= (int32_t)a.fa && rel < (int32_t)a.fb;
                    const int h = n_hot ? hot_find(hkey, hidx, ok) : -1;
                    if (h == top && h >= 0) {
                        r_sum -= srv[i];
                        r_ret++;
                        if (fr) {
                            r_fra = max(r_fra, ssmin[i]);
                            r_flo = min(r_flo, ssmax[i]);
                        }
                    } else if (h >= 0) {
                        acc_retract<FRONT>(hacc, h, srv[i], fr ? ssmin[i] : INT32_MIN, fr ? ssmax[i] : INT32_MAX);
                    } else {
                        atomicAdd(&cnt[(uint32_t)ok >> a.rbits], 1u);
                        f |= fr ? 6u : 2u;
                    }
                }
            }
            flag[i] = (uint8_t)f;
        }
        if (top >= 0) {   /* warp partials of the heaviest hitter */
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
        /* the previous chunk's bulk stores must have read the staging buffer */
        if (tid == 0) tma_wait_read();
        __syncthreads();
        /* partition runs padded to an even number of deltas (16 bytes) */
        uint32_t *off_row = a.off + (int64_t)c * (P + 1);
        const uint32_t total = block_scan_even3<kT>(cnt, cur, cnt, P);
        for (int p = tid; p <= P; p += kT) off_row[p] = cnt[p];
        for (int h = tid; h < n_hot; h += kT) {
            acc_fold(hacc, h);
            if (h == top) {
                long long ws = 0;
                int32_t wi = 0, wr = 0, wmn = INT32_MAX, wmx = INT32_MIN, wfr = INT32_MIN, wfl = INT32_MAX;
                for (int w = 0; w < kW; w++) {
                    ws += wtop_sum[w];
                    wi += wtop_i[w][0];
                    wr += wtop_i[w][1];
                    wmn = min(wmn, wtop_i[w][2]);
                    wmx = max(wmx, wtop_i[w][3]);
                    wfr = max(wfr, wtop_i[w][4]);
                    wfl = min(wfl, wtop_i[w][5]);
                }
                hacc.acc64[h] += ws;
                *hacc.f(A_INS, h) += wi;
                *hacc.f(A_RET, h) += wr;
                *hacc.f(A_IMIN, h) = min(*hacc.f(A_IMIN, h), wmn);
                *hacc.f(A_IMAX, h) = max(*hacc.f(A_IMAX, h), wmx);
                *hacc.f(A_FRAISE, h) = max(*hacc.f(A_FRAISE, h), wfr);
                *hacc.f(A_FLOWER, h) = min(*hacc.f(A_FLOWER, h), wfl);
            }
        }
        /* pass 2: place the exchanged deltas at their partition's cursor */
        for (int i = tid; i < len; i += kT) {
            const uint32_t f = flag[i];
            if (f & 1u) {
                const int32_t k = sk[i];
                const uint32_t pos = atomicAdd(&cur[(uint32_t)k >> a.rbits], 1u);
                stage_s[pos] = DeltaIO<Delta>::make((uint32_t)k, sv[i], 0, 0);
            }
            if (f & 2u) {
                const int32_t ok = srk[i];
                const bool fr = FRONT && (f & 4u);
                const uint32_t pos = atomicAdd(&cur[(uint32_t)ok >> a.rbits], 1u);
                stage_s[pos] = DeltaIO<Delta>::make((uint32_t)ok | kRetract, srv[i], fr ? ssmin[i] : INT32_MIN,
                                                    fr ? ssmax[i] : INT32_MAX);
            }
        }
        __syncthreads();
        for (int p = tid; p < P; p += kT)
            if (cur[p] < cnt[p + 1]) stage_s[cur[p]] = DeltaIO<Delta>::make(kDummy, 0, INT32_MIN, INT32_MAX);
        __syncthreads();
        if (tid == 0) {
            if (total) {
                fence_async_smem();
                tma_store((Delta *)a.stage + (int64_t)c * a.stride, stage_s, total * (uint32_t)DS);
                tma_commit();
            }
            /* the ring stores read sk/sv: drain before the next chunk lands there */
            tma_wait_read();
        }
        __syncthreads();
    }
    /* staging and ring writes complete and visible before the barrier */
    if (tid == 0) {
        tma_wait_all();
        fence_async_global();
    }
    if (trace && tid == 0) trace[2] = globaltimer();
    HotRec *hotpart = (HotRec *)a.hotpart;
    for (int h = tid; h < n_hot; h += kT) {
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
    const bool arrived = grid_barrier(a.bar, timed_out ? 0ULL : a.bar_target);   /* always arrive */
    if (timed_out || !arrived) {
        if (tid == 0) {
            atomicOr(a.err, 2);
            if (a.err_host) *(volatile int *)a.err_host = 2;
        }
        return;
    }
    fence_async_global();
    if (trace && tid == 0) trace[3] = globaltimer();
    if (__syncthreads_or(local_err) && tid == 0) {
        atomicOr(a.err, 1);
        if (a.err_host) *(volatile int *)a.err_host = 1;
    }

    /* ---------------- phase B ---------------- */
    const Acc tab{(int32_t *)(smem + L.b_w), (long long *)(smem + L.b_acc64), a.tcap};
    Delta *dstage = (Delta *)(smem + L.b_dstage);
    uint32_t *segbeg = (uint32_t *)(smem + L.b_segbeg);
    uint32_t *segoff = (uint32_t *)(smem + L.b_segoff);
    unsigned long long *st_sum = (unsigned long long *)(smem + L.b_sum);
    int32_t *st_cnt = (int32_t *)(smem + L.b_cnt);
    unsigned long long *st_bmin = (unsigned long long *)(smem + L.b_bmin);
    unsigned long long *st_bmax = (unsigned long long *)(smem + L.b_bmax);
    unsigned long long *st_fmin = (unsigned long long *)(smem + L.b_fmin);
    unsigned long long *st_fmax = (unsigned long long *)(smem + L.b_fmax);
    const Delta *stage = (const Delta *)a.stage;
    const int pb = (int)((int64_t)P * blockIdx.x / a.grid);
    const int pe = (int)((int64_t)P * (blockIdx.x + 1) / a.grid);
    uint32_t g_parity = 0, s_parity = 0;
    for (int q0 = pb; q0 < pe; q0 += a.ppp) {
        const int q1 = min(pe, q0 + a.ppp);
        const int64_t g0 = (int64_t)q0 << a.rbits;
        const int64_t g1 = min((int64_t)q1 << a.rbits, a.G);
        const int range = (int)(g1 - g0);
        const int range4 = (range + 3) & ~3;
        /* prefetch the range's state while the updates are gathered */
        if (tid == 0) {
            uint32_t bytes = 12u * range4 + (MINMAX ? 16u * range4 : 0u) + (FRONT ? 16u * range4 : 0u);
            mbar_expect(&bars[2], bytes);
            tma_load(st_sum, a.sum + g0, 8u * range4, &bars[2]);
            tma_load(st_cnt, a.cnt + g0, 4u * range4, &bars[2]);
            if (MINMAX) {
                tma_load(st_bmin, a.bmin + g0, 8u * range4, &bars[2]);
                tma_load(st_bmax, a.bmax + g0, 8u * range4, &bars[2]);
            }
            if (FRONT) {
                tma_load(st_fmin, a.fmin + g0, 8u * range4, &bars[2]);
                tma_load(st_fmax, a.fmax + g0, 8u * range4, &bars[2]);
            }
        }
        for (int l = tid; l < range; l += kT) acc_init(tab, l);
        for (int c = tid; c < a.C; c += kT) {
            const uint32_t *row = a.off + (int64_t)c * (P + 1);
            const uint32_t lo = row[q0], hi = row[q1];
            segbeg[c] = lo;
            segoff[c] = hi - lo;
        }
        __syncthreads();
        const uint32_t total = block_scan_inplace<kT>(segoff, a.C);
        for (uint32_t b0 = 0; b0 < total && !timed_out; b0 += (uint32_t)a.dcap) {
            const uint32_t b1 = min(total, b0 + (uint32_t)a.dcap);
            if (tid == 0) mbar_expect(&bars[1], (b1 - b0) * (uint32_t)DS);
            __syncthreads();
            for (int c = tid; c < a.C; c += kT) {
                const uint32_t s0 = segoff[c], s1 = segoff[c + 1];
                const uint32_t lo = max(s0, b0), hi = min(s1, b1);
                if (lo < hi)
                    tma_load(dstage + (lo - b0), stage + (int64_t)c * a.stride + segbeg[c] + (lo - s0),
                             (hi - lo) * (uint32_t)DS, &bars[1]);
            }
            if (!mbar_wait(&bars[1], g_parity) && !mbar_wait(&bars[1], g_parity)) timed_out = true;
            g_parity ^= 1u;
            if (__syncthreads_or(timed_out)) {
                timed_out = true;
                break;
            }
            if (trace && tid == 0 && b0 == 0) trace[6] = globaltimer();
            for (uint32_t i = tid; i < b1 - b0; i += kT) {
                uint32_t kf;
                int32_t dv, smin, smax;
                DeltaIO<Delta>::get(dstage[i], kf, dv, smin, smax);
                const int l = (int)((int64_t)(kf & kKeyMask) - g0);
                if (l < 0 || l >= range) continue;   /* padding deltas and any out-of-range key */
                if (kf & kRetract) acc_retract<FRONT>(tab, l, dv, smin, smax);
                else acc_insert<MINMAX>(tab, l, dv);
            }
            __syncthreads();
            if (trace && tid == 0 && b0 == 0) trace[7] = globaltimer();
            for (int l = tid; l < range; l += kT) acc_fold(tab, l);
            __syncthreads();
        }
        if (!mbar_wait(&bars[2], s_parity) && !mbar_wait(&bars[2], s_parity)) timed_out = true;
        s_parity ^= 1u;
        if (__syncthreads_or(timed_out)) {
            if (tid == 0) {
                atomicOr(a.err, 2);
                if (a.err_host) *(volatile int *)a.err_host = 2;
            }
            return;
        }
        if (trace && tid == 0) trace[4] = globaltimer();
        for (int h = warp; h < n_hot; h += kW) {
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
        for (int l = tid; l < range; l += kT) {
            const int32_t ins = *tab.f(A_INS, l), ret = *tab.f(A_RET, l);
            if (ins + ret == 0) continue;
            const int64_t g = g0 + l;
            const long long s = (long long)st_sum[l] + tab.acc64[l];
            const int32_t cn = st_cnt[l] + (ins - ret);
            a.sum[g] = (unsigned long long)s;
            a.cnt[g] = cn;
            if (MINMAX) {
                const int32_t imin = *tab.f(A_IMIN, l), imax = *tab.f(A_IMAX, l);
                int32_t blo = untag_dn(st_bmin[l], a.epoch, INT32_MAX);
                int32_t bhi = untag_up(st_bmax[l], a.epoch, INT32_MIN);
                if (ins) {
                    blo = min(blo, imin);
                    bhi = max(bhi, imax);
                    a.bmin[g] = tag_dn(a.epoch, blo);
                    a.bmax[g] = tag_up(a.epoch, bhi);
                }
                int32_t flo_v = INT32_MAX, fhi_v = INT32_MIN;
                if (FRONT) {
                    const int32_t fra = *tab.f(A_FRAISE, l), flo = *tab.f(A_FLOWER, l);
                    const unsigned long long tf_lo = st_fmin[l], tf_hi = st_fmax[l];
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
                if (idx < a.hot_cap) {
                    a.hot_next[idx] = (int32_t)g;
                    a.hot_next_cnt[idx] = ins;
                }
            }
        }
        __syncthreads();
    }
    if (trace && tid == 0) trace[5] = globaltimer();
}

}  // namespace

int64_t push_tma_smem_bytes(const PushPlan &pl, bool front) {
    return TmaLayout(pl.P, pl.C, pl.tcap, pl.dcap, front ? 16 : 8, front).total();
}

const void *push_tma_kernel_ptr(bool minmax, bool front) {
    if (front) return (const void *)push_tma_kernel<true, true>;
    if (minmax) return (const void *)push_tma_kernel<true, false>;
    return (const void *)push_tma_kernel<false, false>;
}

}  // namespace cq
