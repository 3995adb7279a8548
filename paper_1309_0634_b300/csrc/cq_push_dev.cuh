/*
 * cq_push_dev.cuh -- device helpers shared by the push kernels
 * (cq_push.cu: register-staged chunks of one query; cq_group.cu: shared-memory
 * staged chunks of one or many queries).
 */
#ifndef CQ_PUSH_DEV_CUH
#define CQ_PUSH_DEV_CUH

#include <cuda_runtime.h>
#include <stdint.h>

#include "cq_internal.h"
#include "cq_push.cuh"

namespace cq {
namespace pushdev {

constexpr unsigned kFull = 0xFFFFFFFFu;
/* A delta is (key word, value).  The key word holds the group (30 bits:
 * groups < 2^30 - 1), kRetract for a tuple that leaves the window and
 * kFrontDep for one that, leaving, shrinks the MIN/MAX front. */
constexpr uint32_t kRetract = 0x80000000u;
constexpr uint32_t kFrontDep = 0x40000000u;
constexpr uint32_t kKeyMask = 0x3FFFFFFFu;
constexpr uint32_t kPadWord = 0x3FFFFFFFu;   /* key word of padding deltas: no group (G <= 2^30 - 2) */


/* ---- shared-memory accumulators (structure of arrays) ----
 * Per group: signed sums of the low and high 16-bit halves of the inserted
 * minus retracted values of the current batch (exact for <= 8192 deltas),
 * an int64 running sum they are folded into, insert and retract counts,
 * extrema of the inserted values, and the count of its front tuples that
 * left (the group's front pointer advances by it). */
enum Field { A_LO = 0, A_HI, A_INS, A_RET, A_IMIN, A_IMAX, A_FDEP, A_NUM };

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
    *a.f(A_FDEP, i) = 0;
    a.acc64[i] = 0;
}

/* v = (v >> 16) * 65536 + (v & 0xFFFF) for every int32 v (arithmetic shift) */
template <bool MINMAX>
__device__ __forceinline__ void acc_insert(const Acc &a, int i, int32_t v) {
    atomicAdd(a.f(A_LO, i), v & 0xFFFF);
    atomicAdd(a.f(A_HI, i), v >> 16);
    atomicAdd(a.f(A_INS, i), 1);
    if (MINMAX) {
        /* a plain read first: most updates of a busy group cannot move its
           extrema, and a contended atomicMin/Max is far dearer than a load */
        if (v < *(volatile int32_t *)a.f(A_IMIN, i)) atomicMin(a.f(A_IMIN, i), v);
        if (v > *(volatile int32_t *)a.f(A_IMAX, i)) atomicMax(a.f(A_IMAX, i), v);
    }
}

__device__ __forceinline__ void acc_retract(const Acc &a, int i, int32_t v, bool front_dep) {
    atomicAdd(a.f(A_LO, i), -(v & 0xFFFF));
    atomicAdd(a.f(A_HI, i), -(v >> 16));
    atomicAdd(a.f(A_RET, i), 1);
    if (front_dep) atomicAdd(a.f(A_FDEP, i), 1);
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

/* ---- block-wide exclusive scan of an smem array of n words, in place, by
 * a CTA of NT threads; a[n] receives the total, which is also returned ---- */
template <int NT>
__device__ __noinline__ uint32_t block_scan_inplace(uint32_t *a, int n) {
    constexpr int kWarps = NT / 32;
    __shared__ uint32_t wsum[kWarps];
    __shared__ uint32_t tot;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + NT - 1) / NT;
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

/* Exclusive scan of the n counts in a, each first rounded up to an even
 * number; the offsets (and a[n] = total) are written to a, b and c.  The
 * indices of counts above mark_above go to marks (the first max_marks of
 * them; *n_marks counts them all). */
template <int NT>
__device__ __noinline__ uint32_t block_scan_even3(uint32_t *a, uint32_t *b, uint32_t *c, int n, uint32_t mark_above,
                                                  uint32_t *marks, int *n_marks, int max_marks) {
    constexpr int kWarps = NT / 32;
    __shared__ uint32_t wsum[kWarps];
    __shared__ uint32_t tot;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + NT - 1) / NT;
    const int b0 = tid * per;
    uint32_t s = 0;
    for (int j = 0; j < per; j++)
        if (b0 + j < n) {
            const uint32_t x = a[b0 + j];
            if (x > mark_above) {   /* a count far above its share: recorded for a later look */
                const int m = atomicAdd(n_marks, 1);
                if (m < max_marks) marks[m] = (uint32_t)(b0 + j);
            }
            s += (x + 1u) & ~1u;
        }
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
            const uint32_t x = (a[b0 + j] + 1u) & ~1u;
            a[b0 + j] = run;
            b[b0 + j] = run;
            c[b0 + j] = run;
            run += x;
        }
    const uint32_t total = tot;
    if (tid == 0) {
        a[n] = total;
        b[n] = total;
        c[n] = total;
    }
    __syncthreads();
    return total;
}

/* Grid barrier over a monotonic counter; gives up after ~2 s.  Thread 0 of
 * each CTA publishes its CTA's writes with a release add and polls with
 * acquire loads. */
static __device__ __noinline__ bool grid_barrier(unsigned long long *bar, unsigned long long target) {
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
            /* back off so that hundreds of pollers do not starve the arrivals */
            __nanosleep(96);
            if ((it & 63) == 63 && globaltimer() - t0 > 2000000000ULL) {
                good = 0;
                break;
            }
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ void cp_async(int32_t *dst, const int32_t *src) {
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async(int2 *dst, const int2 *src) {
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(src) : "memory");
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
    int32_t imin, imax, fdep, pad_;
};

/* A delta in memory: (key word, value). */
struct DeltaIO {
    static __device__ __forceinline__ uint2 make(uint32_t kf, int32_t v) { return make_uint2(kf, (uint32_t)v); }
    static __device__ __forceinline__ void get(uint2 d, uint32_t &kf, int32_t &v) {
        kf = d.x;
        v = (int32_t)d.y;
    }
};

__host__ __device__ constexpr int64_t pad16(int64_t x) { return (x + 15) / 16 * 16; }


}  // namespace pushdev
}  // namespace cq

#endif
