/*
 * cq_flip.cu -- rebuild the "front" of the MIN/MAX structure.
 *
 * Exact MIN/MAX over a sliding window cannot be retracted like a sum.  The
 * window is kept as two segments of stream indices: the front [H, F), whose
 * tuples only leave, and the back [F, N), to which tuples are only added
 * (the two-stacks sliding-window aggregation folklore).  The back keeps
 * insert-only extrema per group.  For the front, every slot holds the
 * extrema of the same group's front tuples that come after it
 * (sufmin/sufmax); when a tuple leaves, its group's front minimum is raised
 * to that suffix minimum (atomicMax) and the front maximum lowered to the
 * suffix maximum (atomicMin).  Because a suffix minimum can only grow along a
 * group's tuples, the maximum over the departed tuples is exactly the
 * minimum of the survivors, in any order of application.
 *
 * When the front is used up, the back becomes the front: a flip.  The flip
 * needs, per group, a reverse scan over its tuples in stream order, so the
 * segment [F, F + len) is sorted by key with a stable LSD radix sort (tuple
 * order within a key is preserved) and a reverse segmented scan over the
 * sorted run of each key yields every slot's suffix extrema and each group's
 * whole-segment extrema.  A flip costs O(len) and happens at most once per
 * W tuples pushed; a push that replaces the whole window needs none.
 *
 * (The paper recomputes its aggregate from scratch over each group's window
 * after every tuple, Section 5.1; this structure replaces that rescan.)
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "cq_internal.h"
#include "cq_tags.cuh"

namespace cq {

namespace {

constexpr int kT = 256;              /* threads per CTA */
constexpr int kItems = 16;           /* items per thread */
constexpr int kTile = kT * kItems;   /* 4096 */
constexpr int kMaxDigitBits = 11;
constexpr unsigned kFull = 0xFFFFFFFFu;

__global__ void flip_load_kernel(const int32_t *ring_k, const int32_t *ring_v, int64_t W, int64_t G, int64_t fmod,
                                 int64_t len, uint32_t *key, uint32_t *pos, int32_t *val, int *err) {
    if (*(volatile int *)err) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = fmod + i;
        if (s >= W) s -= W;
        int32_t k = ring_k[s];
        if ((uint32_t)k >= (uint32_t)G) {
            atomicOr(err, 1);
            k = 0;
        }
        key[i] = (uint32_t)k;
        pos[i] = (uint32_t)i;
        val[i] = ring_v[s];
    }
}

/* Per-tile digit histogram, written digit-major: hist[d * ntiles + tile]. */
__global__ void __launch_bounds__(kT) radix_hist_kernel(const uint32_t *key, int64_t len, int shift, int bits,
                                                        uint32_t *hist, int64_t ntiles, const int *err) {
    if (*(volatile int *)err) return;
    extern __shared__ uint32_t h[];
    const int bins = 1 << bits;
    for (int d = threadIdx.x; d < bins; d += kT) h[d] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll 4
    for (int j = 0; j < kItems; j++) {
        int64_t i = base + j * kT + threadIdx.x;
        if (i < len) atomicAdd(&h[(key[i] >> shift) & (bins - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < bins; d += kT) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

/* Stable scatter of one tile.  Warp w owns the contiguous 512 items
 * [base + 512w, base + 512w + 512) and walks them in 16 rounds of 32, so the
 * rank of an item among equal digits follows its input index. */
__global__ void __launch_bounds__(kT) radix_scatter_kernel(const uint32_t *key_in, const uint32_t *pos_in,
                                                           const int32_t *val_in, uint32_t *key_out,
                                                           uint32_t *pos_out, int32_t *val_out, int64_t len,
                                                           int shift, int bits, const uint32_t *offsets,
                                                           int64_t ntiles, const int *err) {
    if (*(volatile int *)err) return;
    extern __shared__ uint32_t wh[];   /* [8 warps][bins] */
    const int bins = 1 << bits;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 8 * bins; i += kT) wh[i] = 0;
    __syncthreads();
    const int64_t wbase = (int64_t)blockIdx.x * kTile + warp * (kItems * 32);
    uint32_t info[kItems];   /* digit | rank << 12 | count << 18, or ~0 when empty */
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < kItems; r++) {
        int64_t i = wbase + r * 32 + lane;
        bool ok = i < len;
        uint32_t d = ok ? ((key_in[i] >> shift) & (bins - 1)) : 0xFFFFu;
        unsigned peers = __match_any_sync(kFull, d);
        uint32_t rank = __popc(peers & lt);
        uint32_t cntp = __popc(peers);
        info[r] = ok ? (d | (rank << 12) | (cntp << 18)) : 0xFFFFFFFFu;
        if (ok && rank == 0) wh[warp * bins + d] += cntp;
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < bins; d += kT) {
        uint32_t run = offsets[(int64_t)d * ntiles + blockIdx.x];
        for (int w = 0; w < 8; w++) {
            uint32_t c = wh[w * bins + d];
            wh[w * bins + d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kItems; r++) {
        int64_t i = wbase + r * 32 + lane;
        uint32_t inf = info[r];
        uint32_t d = inf & 0xFFF, rank = (inf >> 12) & 0x3F, cntp = (inf >> 18) & 0x3F;
        uint32_t dst = 0;
        if (inf != 0xFFFFFFFFu) dst = wh[warp * bins + d] + rank;
        __syncwarp();
        if (inf != 0xFFFFFFFFu) {
            key_out[dst] = key_in[i];
            pos_out[dst] = pos_in[i];
            val_out[dst] = val_in[i];
            if (rank == 0) wh[warp * bins + d] += cntp;
        }
        __syncwarp();
    }
}

/* ---- device-wide exclusive scan of uint32 (reduce, scan partials, down) ---- */

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *total) {
    __shared__ uint32_t ws[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) ws[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < nw ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    uint32_t before = warp ? ws[warp - 1] : 0;
    *total = ws[nw - 1];
    __syncthreads();
    return before + v - x;
}

__global__ void __launch_bounds__(kT) scan_reduce_kernel(const uint32_t *in, int64_t n, uint32_t *partial) {
    int64_t base = (int64_t)blockIdx.x * kTile + threadIdx.x * kItems;
    uint32_t s = 0;
    for (int j = 0; j < kItems; j++)
        if (base + j < n) s += in[base + j];
    uint32_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) scan_partials_kernel(uint32_t *partial, int64_t nb) {
    int64_t per = (nb + 1023) / 1024;
    int64_t b0 = threadIdx.x * per;
    uint32_t s = 0;
    for (int64_t j = 0; j < per; j++)
        if (b0 + j < nb) s += partial[b0 + j];
    uint32_t tot;
    uint32_t run = block_exclusive_scan(s, &tot);
    for (int64_t j = 0; j < per; j++)
        if (b0 + j < nb) {
            uint32_t x = partial[b0 + j];
            partial[b0 + j] = run;
            run += x;
        }
}

__global__ void __launch_bounds__(kT) scan_down_kernel(uint32_t *data, int64_t n, const uint32_t *partial) {
    int64_t base = (int64_t)blockIdx.x * kTile + threadIdx.x * kItems;
    uint32_t x[kItems];
    uint32_t s = 0;
    for (int j = 0; j < kItems; j++) {
        x[j] = base + j < n ? data[base + j] : 0;
        s += x[j];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan(s, &tot) + partial[blockIdx.x];
    for (int j = 0; j < kItems; j++) {
        if (base + j < n) data[base + j] = run;
        run += x[j];
    }
}

/* ---- reverse segmented scan over the sorted runs ---- */

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

/* Reverse exclusive scan of per-thread states over the CTA: returns the
 * combination of the carry and all threads with a higher index. */
__device__ Seg block_reverse_exclusive(Seg mine, Seg carry, Seg *total) {
    __shared__ int sf[kT];
    __shared__ int slo[kT], shi[kT];
    const int r = kT - 1 - threadIdx.x;   /* position in scan order */
    sf[r] = mine.f;
    slo[r] = mine.lo;
    shi[r] = mine.hi;
    __syncthreads();
    /* Hillis-Steele inclusive scan in scan order */
    for (int o = 1; o < kT; o <<= 1) {
        Seg cur{sf[r], slo[r], shi[r]};
        Seg prev = seg_id();
        bool has = r >= o;
        if (has) prev = Seg{sf[r - o], slo[r - o], shi[r - o]};
        __syncthreads();
        if (has) {
            Seg c = seg_op(prev, cur);
            sf[r] = c.f;
            slo[r] = c.lo;
            shi[r] = c.hi;
        }
        __syncthreads();
    }
    Seg excl = r ? Seg{sf[r - 1], slo[r - 1], shi[r - 1]} : seg_id();
    Seg all{sf[kT - 1], slo[kT - 1], shi[kT - 1]};
    __syncthreads();
    *total = seg_op(carry, all);
    return seg_op(carry, excl);
}

__device__ __forceinline__ bool last_of_run(const uint32_t *key, int64_t len, int64_t i) {
    return i == len - 1 || key[i + 1] != key[i];
}

__global__ void __launch_bounds__(kT) seg_tile_kernel(const uint32_t *key, const int32_t *val, int64_t len,
                                                      int4 *tile_agg, const int *err) {
    if (*(volatile int *)err) return;
    int64_t lo = (int64_t)blockIdx.x * kTile + threadIdx.x * kItems;
    Seg s = seg_id();
    for (int j = kItems - 1; j >= 0; j--) {
        int64_t i = lo + j;
        if (i >= len) continue;
        int32_t v = val[i];
        s = seg_op(s, Seg{last_of_run(key, len, i) ? 1 : 0, v, v});
    }
    Seg tot;
    block_reverse_exclusive(s, seg_id(), &tot);
    if (threadIdx.x == 0) tile_agg[blockIdx.x] = make_int4(tot.f, tot.lo, tot.hi, 0);
}

/* carry[t] = combination of all tiles after t (scan order is decreasing). */
__global__ void __launch_bounds__(kT) seg_carry_kernel(const int4 *tile_agg, int64_t ntiles, int4 *carry) {
    int64_t per = (ntiles + kT - 1) / kT;
    /* thread j owns tiles [j*per, j*per + per), scanned from its top down */
    int64_t t0 = threadIdx.x * per;
    Seg s = seg_id();
    for (int64_t j = per - 1; j >= 0; j--) {
        int64_t t = t0 + j;
        if (t >= ntiles) continue;
        int4 a = tile_agg[t];
        s = seg_op(s, Seg{a.x, a.y, a.z});
    }
    Seg tot;
    Seg run = block_reverse_exclusive(s, seg_id(), &tot);
    for (int64_t j = per - 1; j >= 0; j--) {
        int64_t t = t0 + j;
        if (t >= ntiles) continue;
        carry[t] = make_int4(run.f, run.lo, run.hi, 0);
        int4 a = tile_agg[t];
        run = seg_op(run, Seg{a.x, a.y, a.z});
    }
}

/* Final pass: suffix extrema for every slot of the segment, and the
 * whole-segment extrema of each group at the head of its run. */
__global__ void __launch_bounds__(kT) seg_out_kernel(const uint32_t *key, const uint32_t *pos, const int32_t *val,
                                                     int64_t len, const int4 *carry, int64_t fmod, int64_t W,
                                                     int64_t G, int32_t *sufmin, int32_t *sufmax,
                                                     unsigned long long *fmin, unsigned long long *fmax,
                                                     uint32_t epoch, const int *err) {
    if (*(volatile int *)err) return;
    int64_t lo = (int64_t)blockIdx.x * kTile + threadIdx.x * kItems;
    Seg s = seg_id();
    for (int j = kItems - 1; j >= 0; j--) {
        int64_t i = lo + j;
        if (i >= len) continue;
        int32_t v = val[i];
        s = seg_op(s, Seg{last_of_run(key, len, i) ? 1 : 0, v, v});
    }
    int4 c = carry[blockIdx.x];
    Seg tot;
    Seg run = block_reverse_exclusive(s, Seg{c.x, c.y, c.z}, &tot);
    for (int j = kItems - 1; j >= 0; j--) {
        int64_t i = lo + j;
        if (i >= len) continue;
        bool last = last_of_run(key, len, i);
        int32_t v = val[i];
        /* extrema of the same key strictly after i */
        int32_t amin = last ? INT32_MAX : run.lo;
        int32_t amax = last ? INT32_MIN : run.hi;
        run = seg_op(run, Seg{last ? 1 : 0, v, v});
        int64_t slot = fmod + (int64_t)pos[i];
        if (slot >= W) slot -= W;
        sufmin[slot] = amin;
        sufmax[slot] = amax;
        uint32_t k = key[i];
        bool head = i == 0 || key[i - 1] != k;
        if (head && k < (uint64_t)G) {
            fmin[k] = tag_up(epoch, run.lo);
            fmax[k] = tag_dn(epoch, run.hi);
        }
    }
}

int digit_bits_total(int64_t G) {
    int b = 0;
    while (b < 31 && ((int64_t)1 << b) < G) b++;
    return b;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

int64_t flip_scratch_bytes(int64_t W, int64_t G) {
    (void)G;
    int64_t ntiles = ceil_div(W, kTile);
    int64_t hist = ((int64_t)1 << kMaxDigitBits) * ntiles;
    int64_t partial = ceil_div(hist, kTile) + 1;
    return 2 * W * 12 + hist * 4 + partial * 4 + 2 * ntiles * 16;
}

cudaError_t flip_alloc(DeviceState &d) {
    int64_t W = d.W;
    int64_t ntiles = ceil_div(W, kTile);
    d.hist_cap = ((int64_t)1 << kMaxDigitBits) * ntiles;
    d.partial_cap = ceil_div(d.hist_cap, kTile) + 1;
    d.seg_cap = ntiles;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; b++) {
        e = cudaMalloc(&d.fk[b], sizeof(uint32_t) * W);
        if (e == cudaSuccess) e = cudaMalloc(&d.fp[b], sizeof(uint32_t) * W);
        if (e == cudaSuccess) e = cudaMalloc(&d.fv[b], sizeof(int32_t) * W);
    }
    if (e == cudaSuccess) e = cudaMalloc(&d.hist, sizeof(uint32_t) * d.hist_cap);
    if (e == cudaSuccess) e = cudaMalloc(&d.partial, sizeof(uint32_t) * d.partial_cap);
    if (e == cudaSuccess) e = cudaMalloc(&d.seg, sizeof(int4) * d.seg_cap);
    if (e == cudaSuccess) e = cudaMalloc(&d.carry, sizeof(int4) * d.seg_cap);
    return e;
}

void flip_free(DeviceState &d) {
    for (int b = 0; b < 2; b++) {
        cudaFree(d.fk[b]);
        cudaFree(d.fp[b]);
        cudaFree(d.fv[b]);
        d.fk[b] = d.fp[b] = nullptr;
        d.fv[b] = nullptr;
    }
    cudaFree(d.hist);
    cudaFree(d.partial);
    cudaFree(d.seg);
    cudaFree(d.carry);
    d.hist = d.partial = nullptr;
    d.seg = d.carry = nullptr;
}

/* Exclusive scan of up to 32768 words in one CTA of 1024 threads (32 a thread). */
__global__ void __launch_bounds__(1024) scan_small_kernel(uint32_t *data, int64_t n) {
    const int per = (int)((n + 1023) / 1024);
    const int64_t b0 = (int64_t)threadIdx.x * per;
    uint32_t x[32];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < 32; j++) {
        x[j] = j < per && b0 + j < n ? data[b0 + j] : 0u;
        s += x[j];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan(s, &tot);
#pragma unroll
    for (int j = 0; j < 32; j++)
        if (j < per && b0 + j < n) {
            data[b0 + j] = run;
            run += x[j];
        }
}

int64_t sort_hist_entries(int64_t len) { return ((int64_t)1 << kMaxDigitBits) * ceil_div(len, kTile); }

int64_t sort_partial_entries(int64_t len) { return ceil_div(sort_hist_entries(len), kTile) + 1; }

cudaError_t exclusive_scan_u32(uint32_t *data, int64_t n, uint32_t *partial, cudaStream_t s, int64_t *launches) {
    if (n <= 0) return cudaSuccess;
    if (n <= 32768) {   /* one launch instead of three */
        scan_small_kernel<<<1, 1024, 0, s>>>(data, n);
        if (launches) *launches += 1;
        return cudaGetLastError();
    }
    const int64_t nb = ceil_div(n, kTile);
    scan_reduce_kernel<<<(unsigned)nb, kT, 0, s>>>(data, n, partial);
    scan_partials_kernel<<<1, 1024, 0, s>>>(partial, nb);
    scan_down_kernel<<<(unsigned)nb, kT, 0, s>>>(data, n, partial);
    if (launches) *launches += 3;
    return cudaGetLastError();
}

cudaError_t sort_prepare() {
    static bool attr_set = false;
    if (attr_set) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(radix_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               8 * (1 << kMaxDigitBits) * (int)sizeof(uint32_t));
    if (e == cudaSuccess) attr_set = true;
    return e;
}

int stable_sort_by_key(const SortBuffers &b, int64_t len, int64_t G, cudaStream_t s, const int *err,
                       int64_t *launches) {
    sort_prepare();
    const int64_t ntiles = ceil_div(len, kTile);
    const int total = digit_bits_total(G);
    const int passes = total == 0 ? 0 : (int)ceil_div(total, kMaxDigitBits);
    int cur = 0, shift = 0;
    for (int p = 0; p < passes; p++) {
        const int bits = (int)ceil_div(total - shift, passes - p);
        const int bins = 1 << bits;
        radix_hist_kernel<<<(unsigned)ntiles, kT, bins * sizeof(uint32_t), s>>>(b.k[cur], len, shift, bits, b.hist,
                                                                                 ntiles, err);
        exclusive_scan_u32(b.hist, (int64_t)bins * ntiles, b.partial, s, launches);
        radix_scatter_kernel<<<(unsigned)ntiles, kT, 8 * bins * sizeof(uint32_t), s>>>(
            b.k[cur], b.p[cur], b.v[cur], b.k[cur ^ 1], b.p[cur ^ 1], b.v[cur ^ 1], len, shift, bits, b.hist, ntiles,
            err);
        if (launches) *launches += 2;
        cur ^= 1;
        shift += bits;
    }
    return cur;
}

cudaError_t launch_flip(DeviceState &d, int64_t fmod, int64_t len, uint32_t epoch, cudaStream_t s,
                        int64_t *launches) {
    if (len <= 0) return cudaSuccess;
    if (!d.fk[0]) {
        cudaError_t e = flip_alloc(d);
        if (e != cudaSuccess) return e;
    }
    const int64_t ntiles = ceil_div(len, kTile);
    const int gload = (int)((len + 255) / 256 < 148 * 16 ? (len + 255) / 256 : 148 * 16);
    flip_load_kernel<<<gload, 256, 0, s>>>(d.ring_k, d.ring_v, d.W, d.G, fmod, len, d.fk[0], d.fp[0], d.fv[0], d.err);
    if (launches) *launches += 1;
    const SortBuffers b{{d.fk[0], d.fk[1]}, {d.fp[0], d.fp[1]}, {d.fv[0], d.fv[1]}, d.hist, d.partial};
    const int cur = stable_sort_by_key(b, len, d.G, s, d.err, launches);
    seg_tile_kernel<<<(unsigned)ntiles, kT, 0, s>>>(d.fk[cur], d.fv[cur], len, d.seg, d.err);
    seg_carry_kernel<<<1, kT, 0, s>>>(d.seg, ntiles, d.carry);
    seg_out_kernel<<<(unsigned)ntiles, kT, 0, s>>>(d.fk[cur], d.fp[cur], d.fv[cur], len, d.carry, fmod, d.W, d.G,
                                                   d.sufmin, d.sufmax, d.fmin, d.fmax, epoch, d.err);
    if (launches) *launches += 3;
    return cudaGetLastError();
}

}  // namespace cq
