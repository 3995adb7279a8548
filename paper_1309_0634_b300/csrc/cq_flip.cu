/*
 * cq_flip.cu -- rebuild the "front" of the MIN/MAX structure.
 *
 * Exact MIN/MAX over a sliding window cannot be retracted like a sum.  The
 * window is kept as two segments of stream indices: the front [H, F), whose
 * tuples only leave, and the back [F, N), to which tuples are only added
 * (the two-stacks sliding-window aggregation folklore).  The back keeps
 * insert-only extrema per group.  The front is kept sorted by group, in
 * stream order within a group (sufs), with, at every position, the extrema
 * of the same group's front tuples after it, and per group a pointer to its
 * oldest front tuple still in the window (fptr).  Front tuples leave in
 * stream order, so when d of a group's front tuples leave in a push its
 * pointer moves by d and the survivors' extrema are read at the position
 * before the new pointer: one read per touched group, and the flip writes
 * every array in sorted order (one scattered word per group, not per slot).

 * When the front is used up, the back becomes the front: a flip.  The flip
 * needs, per group, a reverse scan over its tuples in stream order, so the
 * segment [F, F + len) is sorted by key, straight out of the ring, with the
 * stable radix sort of cq_sort.cu (tuple order within a key is preserved),
 * and one reverse segmented scan over the sorted runs yields every
 * position's suffix extrema, each group's whole-segment extrema and the
 * position of each group's run.  The scan is a
 * single kernel: tiles are taken from the end of the sorted array towards
 * its start, and each tile finds the scan state of everything after it by
 * decoupled look-back.  A flip costs O(len) and happens at most once per W
 * tuples pushed; a push that replaces the whole window needs none.
 *
 * (The paper recomputes its aggregate from scratch over each group's window
 * after every tuple, Section 5.1; this structure replaces that rescan.)
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "cq_internal.h"
#include "cq_sort.cuh"
#include "cq_tags.cuh"

namespace cq {

namespace {

constexpr int kT = 256;                       /* threads per CTA */
constexpr int kWarps = kT / 32;
constexpr int kItems = 16;                    /* consecutive items per thread */
constexpr int kTile = kT * kItems;            /* 4096 */
constexpr int kPadTile = kTile + kTile / 32;  /* shared arrays, one pad word per 32 */
constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kScanSmem = 2 * kPadTile * 4;

/* Thread t reads items 16t .. 16t + 15: one pad word per 32 keeps the 32
 * lanes of a warp on 32 different banks. */
__device__ __forceinline__ int padded(int i) { return i + (i >> 5); }

/* State of the scan in decreasing index order: f = a run boundary was
 * crossed (the value no longer depends on later items), lo/hi = extrema. */
struct Seg {
    int f;
    int32_t lo, hi;
};

__device__ __forceinline__ Seg seg_id() { return Seg{0, INT32_MAX, INT32_MIN}; }

/* a = state accumulated from higher indices, b = next (lower-index) item or block */
__device__ __forceinline__ Seg seg_op(Seg a, Seg b) {
    Seg r;
    r.f = a.f | b.f;
    r.lo = b.f ? b.lo : min(a.lo, b.lo);
    r.hi = b.f ? b.hi : max(a.hi, b.hi);
    return r;
}

__device__ __forceinline__ Seg shfl_down_seg(Seg s, int o) {
    return Seg{__shfl_down_sync(kFull, s.f, o), __shfl_down_sync(kFull, s.lo, o), __shfl_down_sync(kFull, s.hi, o)};
}

__device__ __forceinline__ int2 ld_pay(const int2 *p) {
    int2 v;
    asm volatile("ld.relaxed.gpu.global.v2.s32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p) : "memory");
    return v;
}

/* Look-back word of the scan: low half = 2 * inclusive + f, payload (lo, hi)
 * in pay[2 tile + inclusive]. */
__global__ void __launch_bounds__(kT, 5) seg_scan_kernel(const uint32_t *key, const int32_t *val, int64_t len, int64_t G,
                                                      int2 *sufs, int32_t *fptr, unsigned long long *fmin,
                                                      unsigned long long *fmax, uint32_t epoch, SortCtl *ctl,
                                                      unsigned long long *status, int2 *pay, int *err) {
    extern __shared__ __align__(16) uint32_t fsm[];
    uint32_t *sk = fsm;
    int32_t *sv = (int32_t *)(fsm + kPadTile);
    __shared__ int64_t s_tile;
    __shared__ uint32_t s_tag, s_prev, s_next;
    __shared__ int s_fail;
    __shared__ Seg s_warp[kWarps], s_carry;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (*(volatile int *)err) return;
    const int64_t ntiles = (len + kTile - 1) / kTile;
    if (tid == 0) {
        s_tile = ntiles - 1 - (int64_t)atomicAdd(&ctl->tiles[3], 1u);
        s_tag = lb_tag(ctl, 3);
        s_fail = 0;
    }
    __syncthreads();
    const int64_t tile = s_tile, lo = tile * kTile;
    const uint32_t tag = s_tag;
    const int n = (int)(len - lo < kTile ? len - lo : kTile);
    if (tid == 0) {
        s_prev = lo > 0 ? key[lo - 1] : 0xFFFFFFFFu;   /* no key is 2^32 - 1 */
        s_next = lo + n < len ? key[lo + n] : 0xFFFFFFFFu;
    }
    {
        uint32_t k[kItems];
        int32_t v[kItems];
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            const int e = j * kT + tid;
            if (e < n) {
                k[j] = key[lo + e];
                v[j] = val[lo + e];
            }
        }
#pragma unroll
        for (int j = 0; j < kItems; j++) {
            const int e = j * kT + tid;
            if (e < n) {
                sk[padded(e)] = k[j];
                sv[padded(e)] = v[j];
            }
        }
    }
    __syncthreads();
    const int e0 = tid * kItems;
    Seg mine = seg_id();
#pragma unroll
    for (int j = kItems - 1; j >= 0; j--) {
        const int e = e0 + j;
        if (e >= n) continue;
        const uint32_t k = sk[padded(e)], kn = e + 1 < n ? sk[padded(e + 1)] : s_next;
        const int32_t v = sv[padded(e)];
        mine = seg_op(mine, Seg{kn != k ? 1 : 0, v, v});
    }
    /* reverse inclusive scan over the warp's lanes (higher lanes come first) */
    Seg inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Seg y = shfl_down_seg(inc, o);
        if (lane + o < 32) inc = seg_op(y, inc);
    }
    Seg after_lane = shfl_down_seg(inc, 1);
    if (lane == 31) after_lane = seg_id();
    if (lane == 0) s_warp[warp] = inc;
    __syncthreads();
    Seg after_warp = seg_id();
#pragma unroll
    for (int w = kWarps - 1; w >= 0; w--)
        if (w > warp) after_warp = seg_op(after_warp, s_warp[w]);
    if (warp == 0) {
        /* warp 0 publishes the tile and looks back 32 tiles a step: lane l
         * reads tile t + l; the lanes up to the first inclusive word must all
         * have published before the step counts */
        const Seg total = seg_op(after_warp, s_warp[0]);
        const bool last = tile == ntiles - 1;
        if (lane == 0) {
            pay[2 * tile] = make_int2(total.lo, total.hi);
            if (last) pay[2 * tile + 1] = make_int2(total.lo, total.hi);
            lb_store(status + tile, ((unsigned long long)tag << 32) | (last ? 2u : 0u) | (uint32_t)total.f);
        }
        Seg carry = seg_id();
        if (!last) {
            const unsigned long long t0 = lb_clock();
            unsigned it = 0;
            for (int64_t t = tile + 1;;) {
                const int64_t tl = t + lane;
                const unsigned long long w = tl < ntiles ? lb_peek(status + tl) : 0ull;
                const bool ready = tl < ntiles && (uint32_t)(w >> 32) == tag;
                const bool incl_bit = ready && ((w >> 1) & 1u);
                /* a tile with a run boundary cuts the chain: the state after
                   it does not reach across it, so its own aggregate is the
                   rest of the carry (most tiles hold one) */
                const bool incl = incl_bit || (ready && (w & 1u));
                const unsigned incl_mask = __ballot_sync(kFull, incl), ready_mask = __ballot_sync(kFull, ready);
                const int m = incl_mask ? __ffs(incl_mask) - 1 : 31;
                const unsigned need = m == 31 ? kFull : (2u << m) - 1u;
                if ((ready_mask & need) == need) {
                    lb_fence();   /* the payloads were written before their words */
                    Seg x = seg_id();
                    if (lane <= m) {
                        const int2 pv = ld_pay(pay + 2 * tl + (incl_bit ? 1 : 0));
                        x = Seg{(int)(w & 1u), pv.x, pv.y};
                    }
                    /* lanes m .. 0 in that order: the farthest tile first */
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const Seg y = shfl_down_seg(x, o);
                        if (lane + o < 32) x = seg_op(y, x);
                    }
                    const Seg step = Seg{__shfl_sync(kFull, x.f, 0), __shfl_sync(kFull, x.lo, 0),
                                         __shfl_sync(kFull, x.hi, 0)};
                    carry = seg_op(step, carry);
                    if (incl_mask) break;
                    t += 32;
                    continue;
                }
                if (__any_sync(kFull, lb_give_up(++it, t0, err))) {   /* the whole warp leaves */
                    if (lane == 0) s_fail = 1;
                    break;
                }
                __nanosleep(32);
            }
            const Seg through = seg_op(carry, total);
            if (lane == 0) {
                pay[2 * tile + 1] = make_int2(through.lo, through.hi);
                lb_store(status + tile, ((unsigned long long)tag << 32) | 2u | (uint32_t)through.f);
            }
        }
        if (lane == 0) s_carry = carry;
    }
    /* both neighbours of the thread's items, read before any item of the
     * tile is overwritten below */
    const uint32_t k_before = e0 == 0 ? s_prev : (e0 <= n ? sk[padded(e0 - 1)] : 0u);
    const uint32_t k_after = e0 + kItems < n ? sk[padded(e0 + kItems)] : s_next;
    __syncthreads();
    if (s_fail) {
        if (tid == 0) atomicOr(err, 2);
        return;
    }
    /* One pass from the tile's end with the state of everything after each
     * item: an item's suffix extrema (of the same key strictly after it)
     * replace its key and value in shared memory, and a run's head also
     * writes the group's extrema and pointer. */
    Seg full = seg_op(s_carry, seg_op(after_warp, after_lane));
    uint32_t kn = k_after;
#pragma unroll
    for (int j = kItems - 1; j >= 0; j--) {
        const int e = e0 + j;
        if (e >= n) continue;
        const uint32_t k = sk[padded(e)];
        const int32_t v = sv[padded(e)];
        const uint32_t kp = j == 0 ? k_before : sk[padded(e - 1)];
        const bool last = kn != k;
        sk[padded(e)] = last ? (uint32_t)INT32_MAX : (uint32_t)full.lo;
        sv[padded(e)] = last ? INT32_MIN : full.hi;
        full = seg_op(full, Seg{last ? 1 : 0, v, v});
        if (kp != k && (uint64_t)k < (uint64_t)G) {
            fmin[k] = tag_up(epoch, full.lo);
            fmax[k] = tag_dn(epoch, full.hi);
            fptr[k] = (int32_t)(lo + e);   /* the run's head: the group's oldest front tuple */
        }
        kn = k;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kItems; j++) {
        const int e = j * kT + tid;
        if (e < n) sufs[lo + e] = make_int2((int32_t)sk[padded(e)], sv[padded(e)]);
    }
}

}  // namespace

int64_t flip_scratch_bytes(int64_t W, int64_t G) { return sort_scratch_bytes(W, G) + 16 * sort_tiles(W); }

cudaError_t flip_alloc(DeviceState &d, cudaStream_t s) {
    cudaError_t e = sort_alloc(d.sort, d.W, d.G, s);
    if (e == cudaSuccess) e = cudaMalloc(&d.seg_pay, sizeof(int2) * 2 * sort_tiles(d.W));
    return e;
}

void flip_free(DeviceState &d) {
    sort_free(d.sort);
    cudaFree(d.seg_pay);
    d.seg_pay = nullptr;
}

cudaError_t launch_flip(DeviceState &d, int64_t fmod, int64_t len, uint32_t epoch, cudaStream_t s,
                        int64_t *launches) {
    if (len <= 0) return cudaSuccess;
    if (!d.sort.ctl) {
        cudaError_t e = flip_alloc(d, s);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = raise_dyn_smem((const void *)seg_scan_kernel, kScanSmem);
    if (e != cudaSuccess) return e;
    e = sort_maintain(d.sort, s);
    if (e != cudaSuccess) return e;
    const SortRing ring{d.ring_k, d.ring_v, d.W, fmod};
    const int cur = stable_sort_by_key(d.sort, len, d.G, &ring, s, d.err, launches);
    if (cur < 0) return cudaErrorInvalidConfiguration;
    seg_scan_kernel<<<(unsigned)sort_tiles(len), kT, kScanSmem, s>>>(
        d.sort.k[cur], d.sort.v[cur], len, d.G, d.sufs, d.fptr, d.fmin, d.fmax, epoch,
        d.sort.ctl, d.sort.status, d.seg_pay, d.err);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

}  // namespace cq
