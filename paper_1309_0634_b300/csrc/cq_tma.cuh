/*
 * cq_tma.cuh -- inline-PTX helpers of the kernels that stage data through
 * shared memory with the bulk-copy (TMA) engine: mbarrier set-up and bounded
 * waits, cp.async.bulk loads and stores between global and shared memory,
 * bulk-group commits and waits, proxy fences, and ring-buffer copies that
 * wrap around the end of the window.
 *
 * Alignment: every bulk copy needs 16-byte aligned addresses and a size that
 * is a multiple of 16 bytes; callers guarantee it (ring copies: slot, length
 * and window multiples of 4 int32 words).
 */
#ifndef CQ_TMA_CUH
#define CQ_TMA_CUH

#include <cuda_runtime.h>
#include <stdint.h>

#include "cq_push_dev.cuh"

namespace cq {
namespace tma {

using pushdev::globaltimer;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect(unsigned long long *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

/* Wait until the barrier's phase of the given parity completes; false after
 * `limit_ns` (default ~2 s).  Each try suspends the thread for up to 20 us
 * (it resumes as soon as the phase completes), so a waiting thread takes no
 * issue slots from the SM's other warps.  One thread waits and a CTA barrier
 * follows: the other threads see the copied data through that barrier. */
static __device__ bool mbar_wait(unsigned long long *bar, uint32_t parity,
                                 unsigned long long limit_ns = 2000000000ULL) {
    const uint32_t addr = smem_u32(bar);
    unsigned long long t0 = 0;
    for (uint32_t it = 0;; it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity), "r"(20000u)
            : "memory");
        if (done) return true;
        if ((it & 7) == 7) {
            const unsigned long long now = globaltimer();
            if (!t0) t0 = now;
            else if (now - t0 > limit_ns) return false;
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

/* Bulk-load ring slots [s, s + n) (s, n, W multiples of 4), in at most two copies. */
template <typename T>
__device__ __forceinline__ void ring_load(T *dst, const T *ring, int64_t W, int64_t s, int64_t n,
                                          unsigned long long *bar) {
    const int64_t n1 = min(n, W - s);
    tma_load(dst, ring + s, (uint32_t)(n1 * sizeof(T)), bar);
    if (n > n1) tma_load(dst + n1, ring, (uint32_t)((n - n1) * sizeof(T)), bar);
}

/* Bulk-store n elements to ring slots [s, s + n) (s, n, W multiples of 4). */
template <typename T>
__device__ __forceinline__ void ring_store(T *ring, const T *src, int64_t W, int64_t s, int64_t n) {
    const int64_t n1 = min(n, W - s);
    tma_store(ring + s, src, (uint32_t)(n1 * sizeof(T)));
    if (n > n1) tma_store(ring, src + n1, (uint32_t)((n - n1) * sizeof(T)));
}

}  // namespace tma
}  // namespace cq

#endif
