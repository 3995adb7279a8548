/*
 * cq_heavy.cuh -- keys that turn heavy within a push.
 *
 * The heavy hitters a push privatises are the previous push's (skew handling
 * one batch later, Section 4 of the paper).  A key that turns heavy within
 * the push -- a new stream, a re-drawn skew, the retraction of keys that
 * were heavy a window ago -- is not on that list; its deltas would all land
 * in one key range and serialise on the CTA that owns it.  Phase A notices
 * it almost for free: once a chunk's deltas are counted per partition, a
 * partition whose count is over a bound (several times the chunk's fair
 * share) is recorded.  After the chunk's deltas are
 * sorted by partition, one warp looks at each such run:
 *   - the most frequent key among 32 evenly spaced deltas of the run is the
 *     candidate; it must hold at least a quarter of them;
 *   - the candidate takes a slot of the query's small table of such keys
 *     (atomicCAS, so every CTA that finds it gets the same slot);
 *   - its deltas in the run are summed into one of kHotRep replicated
 *     accumulators of that slot and replaced by padding deltas.
 * Phase B's owner of the key's range merges the slot's replicas into its
 * table, puts them back to identity and frees the slot.  The finalise step
 * counts the key's inserts as usual, so the next push privatises it from the
 * start.  A push without such keys pays one comparison per counted delta.
 */
#ifndef CQ_HEAVY_CUH
#define CQ_HEAVY_CUH

#include <stdint.h>

#include "cq_group.cuh"
#include "cq_internal.h"
#include "cq_push_dev.cuh"

namespace cq {

constexpr uint32_t kHeavyMin = 128;   /* least run length that marks a partition */
constexpr int kHeavyList = 8;         /* marked partitions handled per chunk */
constexpr uint32_t kHeavyPad = pushdev::kPadWord;   /* key word of padding deltas (never a group) */

/* Both are computed once per push on the host, for full chunks (a ragged
 * last chunk is held to the same, higher, bound).
 *
 * A chunk of `len` of the push's n tuples: the least count of one key in one
 * of its runs that makes the key heavy here, four times the chunk's share of
 * the push's detection threshold `thr`.  Keys at the threshold's rate are on
 * the next push's list; the factor keeps the chance swings of a chunk's
 * count from registering them again and again in a steady stream. */
__host__ __device__ inline uint32_t heavy_key_min(int64_t len, int64_t n, uint32_t thr) {
    const int64_t m = 4 * (int64_t)thr * len / (n > 0 ? n : 1);
    return m > 16 ? (uint32_t)m : 16u;
}

/* Count above which a partition's run in a chunk of `deltas` deltas over P
 * partitions is looked at: four times its fair share, twice the least count
 * of a heavy key, and at least kHeavyMin. */
__host__ __device__ inline uint32_t heavy_bound(int64_t deltas, int P, uint32_t key_min) {
    int64_t b = 4 * deltas / (P > 0 ? P : 1);
    if (b < 2 * (int64_t)key_min) b = 2 * (int64_t)key_min;
    return b > kHeavyMin ? (uint32_t)b : kHeavyMin;
}

/* Record partition p (its count is over the bound) for a later look. */
__device__ __forceinline__ void note_heavy(uint32_t *list, int *n, uint32_t p) {
    const int j = atomicAdd(n, 1);
    if (j < kHeavyList) list[j] = p;
}

/* One warp: fold the dominant key of `run` (if it has key_min deltas there)
 * into the emergency accumulators of replica `rep`, leaving padding in its
 * place.  Not inlined: it runs rarely, and inlined it costs the kernels'
 * hot loops registers. */
static __device__ __noinline__ void fold_heavy_run(uint2 *run, uint32_t len, uint32_t key_min, int rep, int32_t *emkey, HotAcc *emacc,
                                            unsigned long long *folds, bool minmax) {
    using pushdev::DeltaIO;
    using pushdev::kFrontDep;
    using pushdev::kKeyMask;
    using pushdev::kRetract;
    const unsigned full = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    uint32_t kf;
    int32_t v;
    DeltaIO::get(run[(uint64_t)lane * len / 32], kf, v);
    int32_t key = (kf & kKeyMask) == kHeavyPad ? -1 : (int32_t)(kf & kKeyMask);
    const unsigned peers = __match_any_sync(full, key);
    int score = key >= 0 ? __popc(peers) : 0, best = key;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int os = __shfl_xor_sync(full, score, o), ob = __shfl_xor_sync(full, best, o);
        if (os > score || (os == score && ob < best)) {
            score = os;
            best = ob;
        }
    }
    if (score < 8 || best < 0) return;   /* no key holds a quarter of the run */
    uint32_t count = 0;
    for (uint32_t i = lane; i < len; i += 32) {
        DeltaIO::get(run[i], kf, v);
        count += (int32_t)(kf & kKeyMask) == best;
    }
    if (__reduce_add_sync(full, count) < key_min) return;   /* not heavy at the list's rate */
    int slot = -1;
    if (lane == 0)
        for (int s = 0; s < kEmSlots; s++) {
            const int prev = atomicCAS(&emkey[s], -1, best);
            if (prev == -1 || prev == best) {
                slot = s;
                break;
            }
        }
    slot = __shfl_sync(full, slot, 0);
    if (slot < 0) return;   /* the table is full: the run is left as it is */
    long long sum = 0;
    int32_t ins = 0, ret = 0, imin = INT32_MAX, imax = INT32_MIN, fdep = 0;
    for (uint32_t i = lane; i < len; i += 32) {
        DeltaIO::get(run[i], kf, v);
        if ((int32_t)(kf & kKeyMask) != best) continue;
        if (kf & kRetract) {
            sum -= v;
            ret++;
            fdep += (kf & kFrontDep) ? 1 : 0;
        } else {
            sum += v;
            ins++;
            imin = min(imin, v);
            imax = max(imax, v);
        }
        run[i] = DeltaIO::make(kHeavyPad, 0);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(full, sum, o);
        ins += __shfl_xor_sync(full, ins, o);
        ret += __shfl_xor_sync(full, ret, o);
        imin = min(imin, __shfl_xor_sync(full, imin, o));
        imax = max(imax, __shfl_xor_sync(full, imax, o));
        fdep += __shfl_xor_sync(full, fdep, o);
    }
    if (lane == 0) {
        atomicAdd(folds, 1ULL);
        HotAcc *a = emacc + (int64_t)rep * kEmSlots + slot;
        atomicAdd((unsigned long long *)&a->sum, (unsigned long long)sum);
        if (ins) {
            atomicAdd(&a->ins, ins);
            if (minmax) {
                atomicMin(&a->imin, imin);
                atomicMax(&a->imax, imax);
            }
        }
        if (ret) {
            atomicAdd(&a->ret, ret);
            if (fdep) atomicAdd(&a->fdep, fdep);
        }
    }
}

/* Phase B: warps `warp`, `warp + nwarps`, ... merge the emergency slots whose
 * key lies in [g0, g1) into the range's table (entry key - g0), put their
 * replicas back to identity and free the slots.  `seen` is a shared-memory
 * copy of the slots' keys, read early in the range so that its latency is
 * hidden; only the owner of a key's range frees the slot. */
__device__ __forceinline__ void merge_heavy_slots(const pushdev::Acc &tab, int64_t g0, int64_t g1,
                                                  const int32_t *seen, int32_t *emkey, HotAcc *emacc, int warp,
                                                  int nwarps) {
    using namespace pushdev;
    const unsigned full = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    for (int s = warp; s < kEmSlots; s += nwarps) {
        const int32_t key = seen[s];
        if (key < 0 || (int64_t)key < g0 || (int64_t)key >= g1) continue;
        long long hs = 0;
        int32_t ins = 0, ret = 0, imin = INT32_MAX, imax = INT32_MIN, fdep = 0;
        for (int r = lane; r < kHotRep; r += 32) {
            HotAcc *a = emacc + (int64_t)r * kEmSlots + s;
            hs += __ldcg(&a->sum);
            ins += __ldcg(&a->ins);
            ret += __ldcg(&a->ret);
            imin = min(imin, __ldcg(&a->imin));
            imax = max(imax, __ldcg(&a->imax));
            fdep += __ldcg(&a->fdep);
            a->sum = 0;
            a->ins = 0;
            a->ret = 0;
            a->imin = INT32_MAX;
            a->imax = INT32_MIN;
            a->fdep = 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            hs += __shfl_xor_sync(full, hs, o);
            ins += __shfl_xor_sync(full, ins, o);
            ret += __shfl_xor_sync(full, ret, o);
            imin = min(imin, __shfl_xor_sync(full, imin, o));
            imax = max(imax, __shfl_xor_sync(full, imax, o));
            fdep += __shfl_xor_sync(full, fdep, o);
        }
        if (lane == 0) {
            const int l = (int)(key - g0);
            tab.acc64[l] += hs;
            *tab.f(A_INS, l) += ins;
            *tab.f(A_RET, l) += ret;
            *tab.f(A_IMIN, l) = min(*tab.f(A_IMIN, l), imin);
            *tab.f(A_IMAX, l) = max(*tab.f(A_IMAX, l), imax);
            *tab.f(A_FDEP, l) += fdep;
            emkey[s] = -1;
        }
    }
}

}  // namespace cq

#endif
