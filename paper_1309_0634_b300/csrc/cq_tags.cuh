/*
 * cq_tags.cuh -- epoch-tagged extrema and small warp helpers.
 *
 * MIN/MAX under retraction keep, per group, the extrema of two segments of
 * the window (the "front", which only shrinks, and the "back", which only
 * grows; the two-stacks sliding-window aggregation folklore).  Each extremum
 * is a 64-bit word: the high half is an epoch, the low half the int32 value
 * with its sign bit flipped so that unsigned order equals signed order.
 *
 *   up tag  (epoch << 32 | biased v), combined with atomicMax
 *   down tag (~epoch << 32 | biased v), combined with atomicMin
 *
 * A word written in an older epoch always loses against a current one, and
 * decodes to the identity (INT32_MAX for a minimum, INT32_MIN for a
 * maximum), so advancing the epoch empties a segment for every group at once.
 * Epoch 0 is never current: zero-filled up words and all-ones down words are
 * empty from the start.
 */
#ifndef CQ_TAGS_CUH
#define CQ_TAGS_CUH

#include <stdint.h>

namespace cq {

__device__ __forceinline__ uint32_t biased(int32_t v) { return (uint32_t)v ^ 0x80000000u; }
__device__ __forceinline__ int32_t unbiased(uint32_t u) { return (int32_t)(u ^ 0x80000000u); }

__device__ __forceinline__ unsigned long long tag_up(uint32_t e, int32_t v) {
    return ((unsigned long long)e << 32) | biased(v);
}
__device__ __forceinline__ unsigned long long tag_dn(uint32_t e, int32_t v) {
    return ((unsigned long long)(~e) << 32) | biased(v);
}
__device__ __forceinline__ int32_t untag_up(unsigned long long t, uint32_t e, int32_t empty) {
    return (uint32_t)(t >> 32) == e ? unbiased((uint32_t)t) : empty;
}
__device__ __forceinline__ int32_t untag_dn(unsigned long long t, uint32_t e, int32_t empty) {
    return (uint32_t)(t >> 32) == ~e ? unbiased((uint32_t)t) : empty;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

/* Exact int64 sum of the int32 values of the lanes in `peers` (all lanes of
 * `peers` must call it with the same mask): the values are split into a
 * signed high half and an unsigned low half so that both 32-bit warp sums
 * are exact. */
__device__ __forceinline__ long long peer_sum64(unsigned peers, int32_t v) {
    int hi = __reduce_add_sync(peers, v >> 16);
    unsigned lo = __reduce_add_sync(peers, (unsigned)(v & 0xFFFF));
    return (long long)hi * 65536LL + (long long)lo;
}

__device__ __forceinline__ void red_add_u64(unsigned long long *p, long long v) {
    atomicAdd(p, (unsigned long long)v);
}

/* The front extrema of group g once `dep` (> 0) more of its front tuples
 * have left, given its pointer p_old: the front, sorted by group, holds g's tuples from position
 * fptr[g] on in stream order, and sufs[p] holds the extrema of g's front
 * tuples after position p, so the pointer moves by dep and the survivors'
 * extrema are sufs[new pointer - 1] (empty once none is left).  Only the
 * owner of g's key range calls it in a push. */
__device__ __forceinline__ int2 front_advance(int32_t *fptr, const int2 *sufs, int64_t g, int32_t p_old,
                                              int32_t dep) {
    const int32_t p = p_old + dep;
    fptr[g] = p;
    return sufs[p - 1];
}
/* The same, with the pointer p_old = fptr[g] loaded beforehand. */
__device__ __forceinline__ int2 front_next(int32_t *fptr, const int2 *sufs, int64_t g, int32_t dep) {
    return front_advance(fptr, sufs, g, fptr[g], dep);
}

}  // namespace cq

#endif
