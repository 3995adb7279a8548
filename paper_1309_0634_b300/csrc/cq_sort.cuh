/*
 * cq_sort.cuh -- device side of the decoupled look-back shared by the radix
 * sort passes (cq_sort.cu) and the flip's reverse segmented scan
 * (cq_flip.cu).
 *
 * A look-back word is 64 bits: the high half is a tag, the low half the
 * payload.  A tag has its top bit set (so cleared memory never matches), 28
 * bits of the sort's sequence number (SortCtl::seq, advanced once per sort
 * on the device, so a replayed graph gets fresh tags too) and a 3-bit stage
 * (0..2 = the count scan of a radix pass, 3 = the scan that follows a
 * sort).  Words published under another tag are stale and read as "not yet
 * published".
 */
#ifndef CQ_SORT_CUH
#define CQ_SORT_CUH

#include <stdint.h>

#include "cq_internal.h"

namespace cq {

__device__ __forceinline__ uint32_t lb_tag(const SortCtl *ctl, int stage) {
    const uint32_t seq = *(const volatile uint32_t *)&ctl->seq;
    return 0x80000000u | ((seq & 0x0FFFFFFFu) << 3) | (uint32_t)stage;
}

__device__ __forceinline__ unsigned long long lb_load(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

/* Relaxed load: several may be in flight at once.  Words whose payload sits
 * elsewhere need a fence (lb_fence) between this load and the payload's. */
__device__ __forceinline__ unsigned long long lb_peek(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void lb_fence() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ void lb_store(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

/* Relaxed store, for words that carry their whole payload. */
__device__ __forceinline__ void lb_put(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long lb_clock() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

/* Whether a CTA waiting in a look-back gives up (checked every 64 polls):
 * after about a second, or once another CTA has recorded a timeout (bit 2
 * of the error word).  Tiles are claimed in order from a counter, so the
 * tiles waited for belong to CTAs already running and the wait ends; the
 * limit only guards against a fault elsewhere. */
__device__ __forceinline__ bool lb_give_up(unsigned it, unsigned long long t0, const int *err) {
    if ((it & 63u) != 63u) return false;
    return (*(const volatile int *)err & 2) != 0 || lb_clock() - t0 > 1000000000ULL;
}

}  // namespace cq

#endif
