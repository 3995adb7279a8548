/*
 * cq_kernels.cu -- the per-push hot path: fused ingest/expire and finalise.
 *
 * One push of n tuples (Section 3.1: one iteration of a batch) does, for the
 * n_eff = min(n, W) tuples that can enter the window:
 *   1. read the new tuple (k, v) from the batch and the tuple (k', v') it
 *      evicts from the same ring slot (the paper's window ring whose oldest
 *      entry is overwritten, Section 3.2, here one global ring);
 *   2. write (k, v) into the slot;
 *   3. fold +v into group k (SUM, COUNT, back extrema) and retract v' from
 *      group k' (SUM, COUNT, and -- if k' leaves the front segment -- count
 *      one more front departure of k'; the finalise pass moves k''s front
 *      pointer by its departures and reads the extrema of the survivors
 *      from the sorted suffix array built at the last flip);
 *   4. mark k and k' as touched.
 * The finalise pass then rewrites MIN/MAX/AVG of every touched group.
 *
 * Skew (Section 4): equal keys inside a warp are combined with
 * __match_any_sync before any global atomic, so a heavy hitter costs one
 * atomic per warp instead of one per tuple.
 *
 * All combines are commutative integer atomics (add, min, max), so the
 * results are exact and independent of scheduling.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "cq_internal.h"
#include "cq_avg.cuh"
#include "cq_tags.cuh"

namespace cq {

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 4;          /* elements per thread per step */
constexpr unsigned kFull = 0xFFFFFFFFu;

struct Ptrs {
    int32_t *ring_k, *ring_v;
    unsigned long long *sum;
    int32_t *cnt;
    unsigned long long *bmin, *bmax, *fmin, *fmax;
    const int2 *sufs;           /* the front sorted by group: extrema of the group's later front tuples */
    int32_t *fptr;              /* per group: position in sufs of its oldest front tuple still in */
    int32_t *fdep;              /* per group: front tuples that left in this push (0 between pushes) */
    uint8_t *touched;
    int *err, *err_host;
    int64_t G, W;
};

__device__ __forceinline__ void flag_error(const Ptrs &p, int code) {
    atomicOr(p.err, code);
    if (p.err_host) *(volatile int *)p.err_host = code;
}

/* Insert side of one tuple, optionally combined across the warp. */
template <bool WARP_AGG, bool MINMAX>
__device__ __forceinline__ void apply_insert(const Ptrs &p, bool has, int32_t k, int32_t v, uint32_t epoch) {
    if (WARP_AGG) {
        int32_t key = has ? k : -1;
        unsigned peers = __match_any_sync(kFull, key);
        if (!has) return;
        int leader = __ffs(peers) - 1;
        long long s = peer_sum64(peers, v);
        int c = __popc(peers);
        int32_t lo = 0, hi = 0;
        if (MINMAX) {
            lo = __reduce_min_sync(peers, v);
            hi = __reduce_max_sync(peers, v);
        }
        if ((int)(threadIdx.x & 31) == leader) {
            red_add_u64(&p.sum[k], s);
            atomicAdd(&p.cnt[k], c);
            if (MINMAX) {
                atomicMin(&p.bmin[k], tag_dn(epoch, lo));
                atomicMax(&p.bmax[k], tag_up(epoch, hi));
            }
            p.touched[k] = 1;
        }
    } else {
        if (!has) return;
        red_add_u64(&p.sum[k], (long long)v);
        atomicAdd(&p.cnt[k], 1);
        if (MINMAX) {
            atomicMin(&p.bmin[k], tag_dn(epoch, v));
            atomicMax(&p.bmax[k], tag_up(epoch, v));
        }
        p.touched[k] = 1;
    }
}

/* Retract side of one evicted tuple (k', v'); `front` says whether it
 * leaves the front segment (counted; the finalise step moves the group's
 * front pointer by the count). */
template <bool WARP_AGG, bool MINMAX>
__device__ __forceinline__ void apply_retract(const Ptrs &p, bool has, int32_t k, int32_t v, bool front) {
    if (WARP_AGG) {
        int32_t key = has ? k : -1;
        unsigned peers = __match_any_sync(kFull, key);
        if (!has) return;
        int leader = __ffs(peers) - 1;
        long long s = peer_sum64(peers, v);
        int c = __popc(peers);
        unsigned fmask = 0;
        if (MINMAX) fmask = __ballot_sync(peers, front);
        if ((int)(threadIdx.x & 31) == leader) {
            red_add_u64(&p.sum[k], -s);
            atomicSub(&p.cnt[k], c);
            if (MINMAX && fmask) atomicAdd(&p.fdep[k], __popc(fmask));
            p.touched[k] = 1;
        }
    } else {
        if (!has) return;
        red_add_u64(&p.sum[k], -(long long)v);
        atomicSub(&p.cnt[k], 1);
        if (MINMAX && front) atomicAdd(&p.fdep[k], 1);
        p.touched[k] = 1;
    }
}

/* Fused ingest/expire.  Each warp walks chunks of 32 * kUnroll consecutive
 * effective tuples; lane l handles tuples chunk + j*32 + l, so every load
 * and store of the batch and of the ring is a coalesced 128-byte access. */
template <bool WARP_AGG, bool MINMAX>
__global__ void __launch_bounds__(kThreads) ingest_kernel(Ptrs p, IngestArgs a) {
    if (*(volatile int *)p.err) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
    const int64_t chunk = 32 * kUnroll;
    for (int64_t base = warp * chunk; base < a.n; base += nwarps * chunk) {
        int32_t k[kUnroll], v[kUnroll], ok[kUnroll], ov[kUnroll];
        bool has[kUnroll], old[kUnroll], fr[kUnroll];
        int64_t slot[kUnroll];
#pragma unroll
        for (int j = 0; j < kUnroll; j++) {
            int64_t i = base + j * 32 + lane;
            has[j] = i < a.n;
            int64_t sl = a.slot0 + i;
            if (sl >= p.W) sl -= p.W;
            slot[j] = sl;
            int64_t rel = sl - a.hmod;
            if (rel < 0) rel += p.W;
            old[j] = has[j] && rel < a.old_len;
            fr[j] = old[j] && rel >= a.fa && rel < a.fb;
            k[j] = has[j] ? __ldcs(a.keys + i) : 0;
            v[j] = has[j] ? __ldcs(a.vals + i) : 0;
            ok[j] = old[j] ? p.ring_k[sl] : 0;
            ov[j] = old[j] ? p.ring_v[sl] : 0;
        }
#pragma unroll
        for (int j = 0; j < kUnroll; j++) {
            if (has[j]) {
                p.ring_k[slot[j]] = k[j];
                p.ring_v[slot[j]] = v[j];
            }
            bool kin = has[j] && (uint32_t)k[j] < (uint32_t)p.G;
            if (has[j] && !kin) flag_error(p, 1);
            bool kout = old[j] && (uint32_t)ok[j] < (uint32_t)p.G;
            apply_insert<WARP_AGG, MINMAX>(p, kin, k[j], v[j], a.epoch);
            apply_retract<WARP_AGG, MINMAX>(p, kout, ok[j], ov[j], MINMAX && fr[j] && kout);
        }
    }
}

/* Finalise: every group flagged in touched[] gets MIN/MAX/AVG rewritten
 * from its state; flags are cleared for the next push.  One thread scans
 * 16 flags (one 16-byte load). */
template <bool MINMAX, bool AVG>
__global__ void __launch_bounds__(kThreads) finalize_kernel(Ptrs p, int32_t *rmin, int32_t *rmax, double *ravg,
                                                            uint32_t epoch, int64_t nwords) {
    if (*(volatile int *)p.err) return;
    for (int64_t w = (int64_t)blockIdx.x * kThreads + threadIdx.x; w < nwords; w += (int64_t)gridDim.x * kThreads) {
        uint4 f = reinterpret_cast<uint4 *>(p.touched)[w];
        if ((f.x | f.y | f.z | f.w) == 0) continue;
        reinterpret_cast<uint4 *>(p.touched)[w] = make_uint4(0, 0, 0, 0);
        uint32_t words[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            uint32_t m = words[q];
            while (m) {
                int byte = (__ffs(m) - 1) >> 3;
                m &= ~(0xFFu << (byte * 8));
                int64_t g = w * 16 + q * 4 + byte;
                if (g >= p.G) continue;
                int c = p.cnt[g];
                if (MINMAX) {
                    const int32_t dep = p.fdep[g];
                    if (dep > 0) {   /* front tuples left: the pointer moves, the front shrinks */
                        p.fdep[g] = 0;
                        if ((uint32_t)(p.fmin[g] >> 32) == epoch) {
                            const int2 x = front_next(p.fptr, p.sufs, g, dep);
                            p.fmin[g] = tag_up(epoch, x.x);
                            p.fmax[g] = tag_dn(epoch, x.y);
                        }
                    }
                    int32_t lo = INT32_MAX, hi = INT32_MIN;
                    if (c > 0) {
                        lo = min(untag_dn(p.bmin[g], epoch, INT32_MAX), untag_up(p.fmin[g], epoch, INT32_MAX));
                        hi = max(untag_up(p.bmax[g], epoch, INT32_MIN), untag_dn(p.fmax[g], epoch, INT32_MIN));
                    }
                    rmin[g] = lo;
                    rmax[g] = hi;
                }
                if (AVG) {
                    double a;
                    if (c > 0) {
                        long long s = (long long)p.sum[g];
                        a = avg_rn(s, c);
                    } else {
                        a = __longlong_as_double(0x7FF8000000000000LL);
                    }
                    ravg[g] = a;
                }
            }
        }
    }
}

__global__ void init_state_kernel(Ptrs p, int32_t *rmin, int32_t *rmax, double *ravg, int minmax) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < p.G; g += (int64_t)gridDim.x * blockDim.x) {
        p.sum[g] = 0ULL;
        p.cnt[g] = 0;
        rmin[g] = INT32_MAX;
        rmax[g] = INT32_MIN;
        ravg[g] = __longlong_as_double(0x7FF8000000000000LL);
        if (minmax) {
            p.bmin[g] = ~0ULL;
            p.bmax[g] = 0ULL;
            p.fmin[g] = 0ULL;
            p.fmax[g] = ~0ULL;
        }
    }
}

__global__ void reset_tags_kernel(Ptrs p) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < p.G; g += (int64_t)gridDim.x * blockDim.x) {
        p.bmin[g] = ~0ULL;
        p.bmax[g] = 0ULL;
        p.fmin[g] = 0ULL;
        p.fmax[g] = ~0ULL;
    }
}

Ptrs make_ptrs(const DeviceState &d) {
    Ptrs p;
    p.ring_k = d.ring_k;
    p.ring_v = d.ring_v;
    p.sum = d.sum;
    p.cnt = d.cnt;
    p.bmin = d.bmin;
    p.bmax = d.bmax;
    p.fmin = d.fmin;
    p.fmax = d.fmax;
    p.sufs = d.sufs;
    p.fptr = d.fptr;
    p.fdep = d.fdep;
    p.touched = d.touched;
    p.err = d.err;
    p.err_host = d.err_host;
    p.G = d.G;
    p.W = d.W;
    return p;
}

int grid_for(int64_t work, int per_block, int num_sms, int per_sm) {
    int64_t want = (work + per_block - 1) / per_block;
    int64_t cap = (int64_t)num_sms * per_sm;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (int)want;
}

}  // namespace

cudaError_t launch_ingest(const DeviceState &d, const IngestArgs &a, const Options &o, int num_sms,
                          cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    Ptrs p = make_ptrs(d);
    int grid = grid_for(a.n, kThreads * kUnroll, num_sms, 8);
    if (o.warp_agg) {
        if (a.minmax) ingest_kernel<true, true><<<grid, kThreads, 0, s>>>(p, a);
        else ingest_kernel<true, false><<<grid, kThreads, 0, s>>>(p, a);
    } else {
        if (a.minmax) ingest_kernel<false, true><<<grid, kThreads, 0, s>>>(p, a);
        else ingest_kernel<false, false><<<grid, kThreads, 0, s>>>(p, a);
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize(const DeviceState &d, uint32_t epoch, int minmax, int avg, int num_sms,
                            cudaStream_t s) {
    Ptrs p = make_ptrs(d);
    int64_t nwords = d.Gpad / 16;
    int grid = grid_for(nwords, kThreads, num_sms, 8);
    if (minmax && avg) finalize_kernel<true, true><<<grid, kThreads, 0, s>>>(p, d.rmin, d.rmax, d.ravg, epoch, nwords);
    else if (minmax) finalize_kernel<true, false><<<grid, kThreads, 0, s>>>(p, d.rmin, d.rmax, d.ravg, epoch, nwords);
    else if (avg) finalize_kernel<false, true><<<grid, kThreads, 0, s>>>(p, d.rmin, d.rmax, d.ravg, epoch, nwords);
    else finalize_kernel<false, false><<<grid, kThreads, 0, s>>>(p, d.rmin, d.rmax, d.ravg, epoch, nwords);
    return cudaGetLastError();
}

cudaError_t launch_init_state(const DeviceState &d, int minmax, cudaStream_t s) {
    Ptrs p = make_ptrs(d);
    int grid = grid_for(d.G, 256, 148, 8);
    init_state_kernel<<<grid, 256, 0, s>>>(p, d.rmin, d.rmax, d.ravg, minmax);
    return cudaGetLastError();
}

cudaError_t launch_reset_tags(const DeviceState &d, cudaStream_t s) {
    Ptrs p = make_ptrs(d);
    int grid = grid_for(d.G, 256, 148, 8);
    reset_tags_kernel<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace cq
