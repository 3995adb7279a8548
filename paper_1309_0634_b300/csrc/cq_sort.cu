/*
 * cq_sort.cu -- stable LSD radix sort of (key, position, value) triples by
 * key, used by the MIN/MAX flip and by the per-group windows; and a
 * device-wide exclusive scan of uint32 words.
 *
 * The key space [0, G) is split into digits of at most 11 bits, one pass
 * each (10^6 groups: two passes of 10 bits).  A pass over tiles of 4096
 * items takes three kernels:
 *   count   -- each tile's count of every digit, one row per tile
 *              (counts[tile][d]: every tile writes one coalesced row);
 *   column scan -- for every digit, its count in the tiles before each tile
 *              (a prefix down each column), and its total; a CTA takes 32
 *              digits of 128 tiles, reading and writing whole rows, and finds
 *              the columns' carry from the CTAs above it by decoupled
 *              look-back (Merrill and Garland, "Single-pass parallel prefix
 *              scan with decoupled look-back", 2016), a lane per digit;
 *   scatter -- each tile turns the digit totals into digit starts (a CTA
 *              scan), ranks its items by digit in shared memory (stable: in
 *              input order), stages them there in digit order and writes
 *              them out run by run, so each digit's items leave coalesced.
 * The digit counts of a tile depend only on the pass's input, so no tile of
 * the scatter waits for another.  The first pass may read the triples
 * straight from the window ring (position = offset in the segment), which
 * saves a copy.
 *
 * Look-back words are tagged (cq_sort.cuh), so they are not cleared
 * between sorts; sort_maintain clears them once every 2^27 sorts, before a
 * 28-bit sequence number could bring a stale tag back.
 */
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "cq_internal.h"
#include "cq_sort.cuh"
#include "cq_tags.cuh"

namespace cq {

namespace {

constexpr int kT = 256;              /* threads per CTA */
constexpr int kWarps = kT / 32;
constexpr int kItems = 16;           /* items per thread */
constexpr int kTile = kT * kItems;   /* 4096 items per tile */
static_assert(kTile == kSortTile, "tile size");
/* A pass over at most kSmallLen items with at most 2^kSmallBits digits runs
 * on tiles of kSmallItems items a thread: four times the CTAs for a small
 * sort, whose per-tile work on few digits stays small. */
constexpr int kSmallItems = 4;
constexpr int64_t kSmallLen = 1 << 18;
constexpr int kSmallBits = 8;
bool small_tiles(int64_t len, int bits) { return len <= kSmallLen && bits <= kSmallBits; }
constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kIncl = 0x80000000u;   /* payload bit: an inclusive count (else this tile's own) */
constexpr uint64_t kClearPeriod = (uint64_t)1 << 27;

struct Plan {
    int passes;
    int shift[kSortMaxPasses];
    int bits[kSortMaxPasses];
};

/* Digits of the key space [0, G): as few passes of <= 11 bits as possible,
 * the bits spread evenly over them (at least one bit and one pass). */
Plan make_plan(int64_t G) {
    int total = 1;
    while (total < 31 && ((int64_t)1 << total) < G) total++;
    Plan pl{};
    pl.passes = (total + kSortMaxBits - 1) / kSortMaxBits;
    int shift = 0;
    for (int p = 0; p < pl.passes; p++) {
        const int bits = (total - shift + (pl.passes - p) - 1) / (pl.passes - p);
        pl.shift[p] = shift;
        pl.bits[p] = bits;
        shift += bits;
    }
    return pl;
}

int max_bits(int64_t G) {
    const Plan pl = make_plan(G);
    int b = 0;
    for (int p = 0; p < pl.passes; p++) b = pl.bits[p] > b ? pl.bits[p] : b;
    return b;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

/* Where a pass reads: the window ring (segment [fmod, fmod + len) mod W,
 * positions 0..len-1) or the triple buffers. */
struct Src {
    const uint32_t *k, *p;
    const int32_t *v;
    const int32_t *ring_k, *ring_v;
    int64_t W, fmod;
};
struct Dst {
    uint32_t *k, *p;
    int32_t *v;
};

template <bool kRing, bool kPos = true>
__device__ __forceinline__ void load_item(const Src &s, int64_t g, uint32_t &k, uint32_t &p, int32_t &v) {
    if (kRing) {
        /* 32-bit slots: fmod < W < 2^31 and g < len <= W */
        uint32_t slot = (uint32_t)(s.fmod + g);
        if (slot >= (uint32_t)s.W) slot -= (uint32_t)s.W;
        k = (uint32_t)s.ring_k[slot];
        v = s.ring_v[slot];
        p = (uint32_t)g;
    } else {
        k = s.k[g];
        p = kPos ? s.p[g] : 0u;
        v = s.v[g];
    }
}

/* Lanes of the warp whose digit equals this lane's, from one ballot per
 * digit bit (and one for `ok`): the warp multi-split idiom, cheaper than a
 * general match.  Digits are below 2^11, so bits past a pass's width are 0
 * in every lane and their ballots change nothing. */
__device__ __forceinline__ unsigned digit_peers(uint32_t dg, bool ok) {
    unsigned peers = __ballot_sync(kFull, ok);
    if (!ok) peers = ~peers;
#pragma unroll
    for (int b = 0; b < kSortMaxBits; b++) {
        const bool on = (dg >> b) & 1u;
        const unsigned bal = __ballot_sync(kFull, on);
        peers &= on ? bal : ~bal;
    }
    return peers;
}

/* Count of every digit in each tile, one row per tile: counts[tile * bins
 * + d].  Keys read from the ring are checked against [0, G); `bump`
 * advances the sequence number (first pass of a sort only). */
template <bool kRing, int kIt = kItems>
__global__ void __launch_bounds__(kT, 5) sort_count_kernel(Src s, int64_t len, int64_t G, int shift, int bits,
                                                        uint32_t *counts, int64_t ntiles, SortCtl *ctl, int bump,
                                                        int *err) {
    /* kCopies histograms, interleaved by digit (copy c of digit d at
       d * kCopies + c, other banks): warp w counts into copy w mod kCopies,
       so a digit that takes much of a tile (a heavy key's) serialises a
       quarter of the warps on each of its words, not all of them */
    constexpr int kCopies = 4;
    __shared__ uint32_t h[kSortMaxBins * kCopies];
    if (*(volatile int *)err) return;
    const int bins = 1 << bits;
    const uint32_t mask = (uint32_t)bins - 1u;
    const int tid = threadIdx.x;
    const uint32_t copy = (uint32_t)(tid >> 5) & (kCopies - 1);
    for (int i = tid; i < bins * kCopies; i += kT) h[i] = 0u;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * (kT * kIt);
    uint32_t k[kIt];
    if (kRing) {
        /* ring slots in 32 bits: fmod < W < 2^31 and base + tid < len <= W */
        const uint32_t W32 = (uint32_t)s.W;
        uint32_t slot = (uint32_t)(s.fmod + base + tid);
        if (slot >= W32) slot -= W32;
#pragma unroll
        for (int j = 0; j < kIt; j++) {
            k[j] = base + j * kT + tid < len ? (uint32_t)s.ring_k[slot] : 0u;
            slot += kT;
            if (slot >= W32) slot -= W32;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kIt; j++) {
            const int64_t g = base + j * kT + tid;
            k[j] = g < len ? s.k[g] : 0u;
        }
    }
    bool bad = false;
#pragma unroll
    for (int j = 0; j < kIt; j++) {
        const bool ok = base + j * kT + tid < len;
        uint32_t key = k[j];
        if (kRing && ok && (uint64_t)key >= (uint64_t)G) {
            bad = true;
            key = 0u;
        }
        if (ok) atomicAdd(&h[((key >> shift) & mask) * kCopies + copy], 1u);
    }
    if (bad) atomicOr(err, 1);
    __syncthreads();
    for (int dg = tid; dg < bins; dg += kT) {
        uint32_t c = 0u;
#pragma unroll
        for (int q = 0; q < kCopies; q++) c += h[dg * kCopies + q];
        counts[(int64_t)blockIdx.x * bins + dg] = c;
    }
    if (bump && blockIdx.x == 0 && tid == 0) ctl->seq += 1u;
}

/* Column scan of the count rows: a[t][d] becomes digit d's count in tiles
 * 0 .. t-1, and totals[d] its count in all ntiles tiles.  A CTA takes the
 * block of kColDigits digits by kColTiles tiles claimed next from the stage's
 * counter (all blocks of a row of tile blocks before the next row), a lane
 * per digit and kColTiles / kWarps rows a warp.  Warp 0 publishes the block's
 * column sums, then adds those of the blocks above it (same digits, earlier
 * tiles) until it meets an inclusive word: one tagged 64-bit word per digit
 * and tile block. */
constexpr int kColDigits = 32;
constexpr int kColTiles = 128;
constexpr int kColRows = kColTiles / kWarps;   /* rows a warp takes */

__global__ void __launch_bounds__(kT) sort_colscan_kernel(uint32_t *a, int64_t ntiles, int bins, uint32_t *totals,
                                                          SortCtl *ctl, int stage, unsigned long long *status,
                                                          int *err) {
    __shared__ uint32_t ws[kWarps][kColDigits];
    __shared__ uint32_t s_carry[kColDigits];
    __shared__ int64_t s_blk;
    __shared__ uint32_t s_tag;
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (*(volatile int *)err) return;
    if (tid == 0) {
        s_blk = atomicAdd(&ctl->tiles[stage], 1u);
        s_tag = lb_tag(ctl, stage);
        s_fail = 0;
    }
    __syncthreads();
    const int ndb = (bins + kColDigits - 1) / kColDigits;
    const int64_t ntb = (ntiles + kColTiles - 1) / kColTiles;
    const int64_t tb = s_blk / ndb;
    const int db = (int)(s_blk % ndb);
    const uint32_t tag = s_tag;
    const int d = db * kColDigits + lane;
    const bool dok = d < bins;
    const int64_t t0 = tb * kColTiles + (int64_t)warp * kColRows;
    uint32_t x[kColRows];
#pragma unroll
    for (int r = 0; r < kColRows; r++) x[r] = dok && t0 + r < ntiles ? a[(t0 + r) * bins + d] : 0u;
    uint32_t sum = 0u;
#pragma unroll
    for (int r = 0; r < kColRows; r++) sum += x[r];
    ws[warp][lane] = sum;
    __syncthreads();
    if (warp == 0) {
        uint32_t total = 0u;
#pragma unroll
        for (int w = 0; w < kWarps; w++) total += ws[w][lane];
        unsigned long long *st = status + ((int64_t)tb * ndb + db) * kColDigits;
        lb_put(st + lane, ((unsigned long long)tag << 32) | total | (tb == 0 ? kIncl : 0u));
        uint32_t carry = 0u;
        if (tb > 0) {
            const unsigned long long c0 = lb_clock();
            unsigned it = 0;
            bool done = false;
            for (int64_t p = tb - 1;;) {
                /* each lane walks up its own column; the warp polls until
                   every lane has met an inclusive word */
                bool moved = false;
                if (!done) {
                    const unsigned long long w = lb_peek(status + ((int64_t)p * ndb + db) * kColDigits + lane);
                    if ((uint32_t)(w >> 32) == tag) {
                        carry += (uint32_t)w & ~kIncl;
                        if ((uint32_t)w & kIncl) done = true;
                        else p--;
                        moved = true;
                    }
                }
                if (__all_sync(kFull, done)) break;
                if (!__any_sync(kFull, moved)) {
                    if (__any_sync(kFull, lb_give_up(++it, c0, err))) {
                        if (lane == 0) s_fail = 1;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            lb_put(st + lane, ((unsigned long long)tag << 32) | (carry + total) | kIncl);
        }
        s_carry[lane] = carry;
        if (tb == ntb - 1 && dok) totals[d] = carry + total;
    }
    __syncthreads();
    if (s_fail) {
        if (tid == 0) atomicOr(err, 2);
        return;
    }
    uint32_t run = s_carry[lane];
    for (int w = 0; w < warp; w++) run += ws[w][lane];
#pragma unroll
    for (int r = 0; r < kColRows; r++)
        if (dok && t0 + r < ntiles) {
            a[(t0 + r) * bins + d] = run;
            run += x[r];
        }
}

/* In-place exclusive scan of a[0, n) by the CTA (n <= kT * 8); a[n] = total. */
__device__ void cta_scan(uint32_t *a, int n) {
    __shared__ uint32_t ws[kWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + kT - 1) / kT;
    const int b0 = tid * per;
    uint32_t x[8];
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        x[j] = j < per && b0 + j < n ? a[b0 + j] : 0u;
        sum += x[j];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kWarps; w++) {
        before += w < warp ? ws[w] : 0u;
        total += ws[w];
    }
    uint32_t run = before + inc - sum;
#pragma unroll
    for (int j = 0; j < 8; j++)
        if (j < per && b0 + j < n) {
            a[b0 + j] = run;
            run += x[j];
        }
    if (tid == 0) a[n] = total;
    __syncthreads();
}

/* Dynamic shared memory of a scatter with `bins` digits and tiles of `tile` items. */
__host__ __device__ constexpr int scatter_smem_bytes(int bins, int tile = kTile, bool pos = true) {
    return (2 * bins + 4) * 4 + kWarps * bins * 2 + (pos ? 3 : 2) * tile * 4;
}

/* One pass: the tile's items, stably, to their digit's place.  `offsets`
 * holds each digit's count in the tiles before each tile (a row per tile),
 * `totals` each digit's count in the pass: a digit's items start in the
 * output after those of all smaller digits. */
template <bool kRing, int kIt = kItems, bool kPos = true>
__global__ void __launch_bounds__(kT, kPos ? 2 : 3) sort_scatter_kernel(Src s, Dst d, int64_t len, int shift, int bits,
                                                             const uint32_t *offsets, const uint32_t *totals,
                                                             int *err) {
    constexpr int kTileIt = kT * kIt;
    extern __shared__ __align__(16) uint32_t sm[];
    const int bins = 1 << bits;
    const uint32_t mask = (uint32_t)bins - 1u;
    uint32_t *lstart = sm;                        /* bins + 1: the tile's digit starts */
    uint32_t *gbase = lstart + bins + 2;          /* bins: digit starts in the output */
    uint16_t *wh = (uint16_t *)(gbase + bins + 2);/* [warp][digit] counts, then offsets */
    uint32_t *sk = (uint32_t *)(wh + kWarps * bins);
    uint32_t *sp = sk + kTileIt;   /* positions: only when kPos */
    int32_t *sv = (int32_t *)(kPos ? sp + kTileIt : sp);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (*(volatile int *)err) return;
    for (int i = tid; i < kWarps * bins / 2; i += kT) ((uint32_t *)wh)[i] = 0u;
    const int64_t tile = blockIdx.x;
    for (int dg = tid; dg < bins; dg += kT) gbase[dg] = totals[dg];
    __syncthreads();
    cta_scan(gbase, bins);
    for (int dg = tid; dg < bins; dg += kT) gbase[dg] += offsets[tile * bins + dg];
    __syncthreads();
    const int64_t base = tile * kTileIt;
    const int n_tile = (int)(len - base < kTileIt ? len - base : kTileIt);
    /* warp w holds items [32 kIt w, 32 kIt (w + 1)) of the tile, 32 per round */
    /* lr: rank in the warp's digit run (below 32 kIt), two to a register */
    uint32_t kk[kIt], pp[kIt], lr[(kIt + 1) / 2];
    int32_t vv[kIt];
#pragma unroll
    for (int r = 0; r < kIt; r++) {
        const int i = warp * (kIt * 32) + r * 32 + lane;
        kk[r] = 0u;
        pp[r] = 0u;
        vv[r] = 0;
        if (i < n_tile) load_item<kRing, kPos>(s, base + i, kk[r], pp[r], vv[r]);
    }
    /* rank within the warp's digit run, in input order */
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < kIt; r++) {
        const int i = warp * (kIt * 32) + r * 32 + lane;
        const bool ok = i < n_tile;
        const uint32_t dg = (kk[r] >> shift) & mask;
        const unsigned peers = digit_peers(dg, ok);
        const int leader = __ffs(peers) - 1;
        uint32_t before = 0u;
        if (ok && lane == leader) {
            before = wh[warp * bins + dg];
            wh[warp * bins + dg] = (uint16_t)(before + __popc(peers));
        }
        before = __shfl_sync(kFull, before, leader);
        const uint32_t rank = before + __popc(peers & lt);
        if (r & 1)
            lr[r >> 1] |= rank << 16;
        else
            lr[r >> 1] = rank;
        __syncwarp();
    }
    __syncthreads();
    /* per digit: the tile's count and each warp's offset in it */
    for (int dg = tid; dg < bins; dg += kT) {
        uint32_t c = 0u;
#pragma unroll
        for (int w = 0; w < kWarps; w++) {
            const uint32_t x = wh[w * bins + dg];
            wh[w * bins + dg] = (uint16_t)c;
            c += x;
        }
        lstart[dg] = c;
    }
    __syncthreads();
    cta_scan(lstart, bins);
    /* the tile into shared memory in digit order, then out run by run */
#pragma unroll
    for (int r = 0; r < kIt; r++) {
        const int i = warp * (kIt * 32) + r * 32 + lane;
        if (i < n_tile) {
            const uint32_t dg = (kk[r] >> shift) & mask;
            const uint32_t at = lstart[dg] + wh[warp * bins + dg] + ((lr[r >> 1] >> (16 * (r & 1))) & 0xFFFFu);
            sk[at] = kk[r];
            if (kPos) sp[at] = pp[r];
            sv[at] = vv[r];
        }
    }
    __syncthreads();
    for (int e = tid; e < n_tile; e += kT) {
        const uint32_t k = sk[e], dg = (k >> shift) & mask;
        /* 32-bit positions: len < 2^31 */
        const uint32_t o = gbase[dg] + ((uint32_t)e - lstart[dg]);
        if (o < (uint32_t)len) {
            d.k[o] = k;
            if (kPos) d.p[o] = sp[e];
            d.v[o] = sv[e];
        }
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

}  // namespace

int64_t sort_tiles(int64_t len) { return ceil_div(len, kTile); }

/* Digit counts of the largest pass of a sort of up to cap items. */
int64_t count_words(int64_t cap, int64_t G) {
    const int64_t big = ceil_div(cap, kTile) << max_bits(G);
    const int64_t small = ceil_div(cap < kSmallLen ? cap : kSmallLen, kT * kSmallItems) << kSmallBits;
    return big > small ? big : small;
}

/* Look-back words of a column scan over the tiles of `tile` items of a pass
 * of `bits`-bit digits: one per digit (in blocks of kColDigits) and block of
 * kColTiles tiles. */
int64_t colscan_words(int64_t len, int bits, int tile) {
    return ceil_div(ceil_div(len, tile), kColTiles) * ceil_div((int64_t)1 << bits, kColDigits) * kColDigits;
}

int64_t sort_status_entries(int64_t len, int64_t G) {
    /* look-back words: the column scans of the passes and the flip's scan tiles */
    const int64_t a = ceil_div(len, kTile), b = colscan_words(len, max_bits(G), kTile);
    const int64_t c = colscan_words(len < kSmallLen ? len : kSmallLen, kSmallBits, kT * kSmallItems);
    const int64_t m = a > b ? a : b;
    return (m > c ? m : c) + 1;
}

int64_t sort_scratch_bytes(int64_t cap, int64_t G) {
    return 2 * cap * 12 + 4 * count_words(cap, G) + 4 * kSortMaxBins + 8 * sort_status_entries(cap, G) +
           (int64_t)sizeof(SortCtl);
}

cudaError_t sort_alloc(SortBuffers &b, int64_t cap, int64_t G, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; i++) {
        e = cudaMalloc(&b.k[i], sizeof(uint32_t) * cap);
        if (e == cudaSuccess) e = cudaMalloc(&b.p[i], sizeof(uint32_t) * cap);
        if (e == cudaSuccess) e = cudaMalloc(&b.v[i], sizeof(int32_t) * cap);
    }
    b.status_entries = sort_status_entries(cap, G);
    if (e == cudaSuccess) e = cudaMalloc(&b.counts, sizeof(uint32_t) * count_words(cap, G));
    if (e == cudaSuccess) e = cudaMalloc(&b.totals, sizeof(uint32_t) * kSortMaxBins);
    if (e == cudaSuccess) e = cudaMalloc(&b.ctl, sizeof(SortCtl));
    if (e == cudaSuccess) e = cudaMalloc(&b.status, sizeof(unsigned long long) * b.status_entries);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.ctl, 0, sizeof(SortCtl), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.status, 0, sizeof(unsigned long long) * b.status_entries, s);
    b.sorts = 0;
    return e;
}

void sort_free(SortBuffers &b) {
    for (int i = 0; i < 2; i++) {
        cudaFree(b.k[i]);
        cudaFree(b.p[i]);
        cudaFree(b.v[i]);
    }
    cudaFree(b.counts);
    cudaFree(b.totals);
    cudaFree(b.ctl);
    cudaFree(b.status);
    b = SortBuffers{};
}

cudaError_t sort_maintain(SortBuffers &b, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (b.sorts > 0 && b.sorts % kClearPeriod == 0)
        e = cudaMemsetAsync(b.status, 0, sizeof(unsigned long long) * b.status_entries, s);
    b.sorts++;
    return e;
}

cudaError_t sort_prepare() {
    const int smem = scatter_smem_bytes(kSortMaxBins), smem_np = scatter_smem_bytes(kSortMaxBins, kTile, false);
    cudaError_t e = raise_dyn_smem((const void *)sort_scatter_kernel<true>, smem);
    if (e == cudaSuccess) e = raise_dyn_smem((const void *)sort_scatter_kernel<false>, smem);
    if (e == cudaSuccess) e = raise_dyn_smem((const void *)sort_scatter_kernel<true, kItems, false>, smem_np);
    if (e == cudaSuccess) e = raise_dyn_smem((const void *)sort_scatter_kernel<false, kItems, false>, smem_np);
    return e;
}

/* One scatter launch of the variant the pass needs. */
template <bool kPos>
void launch_scatter(bool ring, bool small, unsigned nt, int smem, cudaStream_t s, const Src &in, const Dst &dst,
                    int64_t len, int sh, int bits, const uint32_t *offsets, const uint32_t *totals, int *err) {
    if (ring && small)
        sort_scatter_kernel<true, kSmallItems, kPos><<<nt, kT, smem, s>>>(in, dst, len, sh, bits, offsets, totals, err);
    else if (ring)
        sort_scatter_kernel<true, kItems, kPos><<<nt, kT, smem, s>>>(in, dst, len, sh, bits, offsets, totals, err);
    else if (small)
        sort_scatter_kernel<false, kSmallItems, kPos><<<nt, kT, smem, s>>>(in, dst, len, sh, bits, offsets, totals,
                                                                           err);
    else
        sort_scatter_kernel<false, kItems, kPos><<<nt, kT, smem, s>>>(in, dst, len, sh, bits, offsets, totals, err);
}

int stable_sort_by_key(SortBuffers &b, int64_t len, int64_t G, const SortRing *ring, cudaStream_t s, int *err,
                       int64_t *launches) {
    if (len >= (1LL << 31)) return -1;   /* the scatter's positions are 32-bit */
    if (sort_prepare() != cudaSuccess) return -1;
    const Plan pl = make_plan(G);
    cudaMemsetAsync(b.ctl, 0, offsetof(SortCtl, seq), s);
    Src src{b.k[0], b.p[0], b.v[0], nullptr, nullptr, 0, 0};
    if (ring) {
        src.ring_k = ring->k;
        src.ring_v = ring->v;
        src.W = ring->W;
        src.fmod = ring->fmod;
    }
    /* ring input: pass p writes buffer p & 1; buffer input: pass p reads p & 1, writes the other.
       A ring-sourced sort carries no positions (its caller reads keys and
       values only): a third less traffic in every scatter. */
    int cur = ring ? -1 : 0;
    uint32_t *const *pos = ring ? nullptr : b.p;
    for (int p = 0; p < pl.passes; p++) {
        const int out = cur < 0 ? 0 : cur ^ 1;
        const Dst dst{b.k[out], pos ? pos[out] : nullptr, b.v[out]};
        const Src in = cur < 0 ? src : Src{b.k[cur], pos ? pos[cur] : nullptr, b.v[cur], nullptr, nullptr, 0, 0};
        const bool small = small_tiles(len, pl.bits[p]);
        const int tile = small ? kT * kSmallItems : kTile;
        const int64_t ntiles = ceil_div(len, tile);
        const int64_t n_colblk = ceil_div(ntiles, kColTiles) * ceil_div((int64_t)1 << pl.bits[p], kColDigits);
        const int smem = scatter_smem_bytes(1 << pl.bits[p], tile, pos != nullptr);
        const int sh = pl.shift[p], bits = pl.bits[p];
        const unsigned nt = (unsigned)ntiles;
        if (cur < 0 && small)
            sort_count_kernel<true, kSmallItems><<<nt, kT, 0, s>>>(in, len, G, sh, bits, b.counts, ntiles, b.ctl, p == 0,
                                                                   err);
        else if (cur < 0)
            sort_count_kernel<true><<<nt, kT, 0, s>>>(in, len, G, sh, bits, b.counts, ntiles, b.ctl, p == 0, err);
        else if (small)
            sort_count_kernel<false, kSmallItems><<<nt, kT, 0, s>>>(in, len, G, sh, bits, b.counts, ntiles, b.ctl,
                                                                    p == 0, err);
        else
            sort_count_kernel<false><<<nt, kT, 0, s>>>(in, len, G, sh, bits, b.counts, ntiles, b.ctl, p == 0, err);
        sort_colscan_kernel<<<(unsigned)n_colblk, kT, 0, s>>>(b.counts, ntiles, 1 << bits, b.totals, b.ctl, p,
                                                              b.status, err);
        if (pos)
            launch_scatter<true>(cur < 0, small, nt, smem, s, in, dst, len, sh, bits, b.counts, b.totals, err);
        else
            launch_scatter<false>(cur < 0, small, nt, smem, s, in, dst, len, sh, bits, b.counts, b.totals, err);
        cur = out;
    }
    if (launches) *launches += 3 * pl.passes;
    return cur;
}

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

}  // namespace cq
