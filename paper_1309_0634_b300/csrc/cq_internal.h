/*
 * cq_internal.h -- query state and kernel launchers shared by the CUDA
 * translation units of libcq.  Not part of the public ABI (include/cq.h).
 *
 * Device state of one query (all in HBM, allocated at cq_create):
 *   ring_k[W], ring_v[W]     the window: tuple with stream index t lives in
 *                            slot t mod W (the paper's per-group window ring
 *                            with a moving oldest pointer, Section 3.2,
 *                            turned into one global ring)
 *   sum[G] (int64), cnt[G]   running SUM / COUNT = the published results
 *   rmin[G], rmax[G], ravg[G] published MIN / MAX / AVG of touched groups
 *   bmin[G], bmax[G]         insert-only extrema of the "back" segment
 *   fmin[G], fmax[G]         extrema of the surviving "front" segment
 *   sufs[W] (int2)           the front sorted by group, stream order within
 *                            a group (set at a flip): per position, the
 *                            (min, max) of the same group's later front
 *                            tuples
 *   fptr[G]                  per group: position in sufs of its oldest
 *                            front tuple still in the window
 *   touched[Gpad]            1 for groups changed by the current push
 *                            (direct-atomics path only)
 *   stage, off, hotpart      exchange buffers of the partitioned push
 *   hotlist[2][2][kMaxHot]   heavy hitters of the current / next push: the
 *                            keys sure of a slot, then the others
 * The four extrema arrays hold 64-bit epoch-tagged values (see cq_tags.cuh)
 * so a whole segment is reset in O(1) by advancing the epoch.
 */
#ifndef CQ_INTERNAL_H
#define CQ_INTERNAL_H

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cq.h"

namespace cq {

/* ---- stable LSD radix sort (cq_sort.cu) ----
 * Sorts (key, position, value) triples by key (keys < G), stably.  The input
 * is buffers [0], or the window ring when a SortRing is given (the segment
 * [fmod, fmod + len) mod W; such a sort moves (key, value) pairs only and
 * leaves the position buffers untouched).  The other buffers are
 * ping-pong space.  stable_sort_by_key returns the index (0 or 1) of the
 * buffers holding the sorted triples (-1 for len >= 2^31); call sort_maintain once before every
 * sort (or replay of a captured sort), outside any graph capture. */
constexpr int kSortMaxPasses = 3;
constexpr int kSortMaxBits = 11;
constexpr int kSortMaxBins = 1 << kSortMaxBits;
constexpr int kSortTile = 4096;   /* items per tile of the sort and of the scans that use its look-back words */
struct SortCtl {
    uint32_t tiles[8];   /* tile counters of the look-back scans: passes 0..2, and a scan after the sort (3) */
    uint32_t seq;        /* advanced once per sort on the device; never cleared */
    uint32_t pad[7];
};
struct SortBuffers {
    uint32_t *k[2] = {nullptr, nullptr};
    uint32_t *p[2] = {nullptr, nullptr};
    int32_t *v[2] = {nullptr, nullptr};
    uint32_t *counts = nullptr;             /* per-tile digit counts (a row per tile), then each digit's
                                               count in the tiles before */
    uint32_t *totals = nullptr;             /* each digit's count in the whole pass */
    SortCtl *ctl = nullptr;
    unsigned long long *status = nullptr;   /* tagged look-back words */
    int64_t status_entries = 0;
    uint64_t sorts = 0;                     /* sorts issued, counted on the host */
};
struct SortRing {
    const int32_t *k, *v;
    int64_t W, fmod;
};
int64_t sort_tiles(int64_t len);
int64_t sort_status_entries(int64_t len, int64_t G);
int64_t sort_scratch_bytes(int64_t cap, int64_t G);
cudaError_t sort_alloc(SortBuffers &b, int64_t cap, int64_t G, cudaStream_t s);
void sort_free(SortBuffers &b);
cudaError_t sort_maintain(SortBuffers &b, cudaStream_t s);
int stable_sort_by_key(SortBuffers &b, int64_t len, int64_t G, const SortRing *ring, cudaStream_t s, int *err,
                       int64_t *launches);
/* Kernel attributes of the sort on the current device; call before
 * capturing a sort into a graph.  stable_sort_by_key returns -1 when they
 * cannot be set. */
cudaError_t sort_prepare();

/* Raise the dynamic shared-memory limit of kernel `fn` on the current device
 * to at least `bytes` (cq_attr.cu: per device, thread-safe, never lowered). */
cudaError_t raise_dyn_smem(const void *fn, int bytes);

struct DeviceState {
    int64_t G = 0, W = 0, Gpad = 0;
    int32_t *ring_k = nullptr, *ring_v = nullptr;
    unsigned long long *sum = nullptr;
    int32_t *cnt = nullptr, *rmin = nullptr, *rmax = nullptr;
    double *ravg = nullptr;
    unsigned long long *bmin = nullptr, *bmax = nullptr, *fmin = nullptr, *fmax = nullptr;
    int2 *sufs = nullptr;
    int32_t *fptr = nullptr;
    int32_t *fdep = nullptr;       /* direct path: front departures per group in a push */
    uint8_t *touched = nullptr;
    int *err = nullptr;            /* device error word, sticky */
    int *err_host = nullptr;       /* device alias of a mapped pinned host word */
    /* flip scratch */
    SortBuffers sort;              /* radix sort of the flipped segment */
    int2 *seg_pay = nullptr;       /* look-back payloads of the reverse segmented scan */
    /* partitioned push */
    void *stage = nullptr;         /* per-chunk delta runs */
    int64_t stage_bytes = 0;
    uint32_t *off = nullptr;       /* per-chunk partition offsets */
    int64_t off_bytes = 0;
    void *hotpart = nullptr;       /* per-CTA heavy-hitter partial records */
    void *hotacc = nullptr;        /* kMaxHot heavy-hitter accumulators of the group kernel */
    int32_t *emkey = nullptr;      /* kEmSlots keys found heavy within a push (-1 = free) */
    void *emacc = nullptr;         /* their kHotRep x kEmSlots accumulators, at identity between launches */
    unsigned long long *emfolds = nullptr;   /* runs folded by them so far */
    int64_t hotpart_bytes = 0;
    int32_t *hotlist = nullptr;    /* [2 pushes][2 tiers][kMaxHot] heavy hitters (current / next push) */
    int *hotlist_n = nullptr;      /* [2 pushes][2 tiers] counts */
    int32_t *hotlist_cnt = nullptr;/* insert counts of the heavy hitters, laid out as hotlist */
    unsigned long long *bar = nullptr;   /* grid-barrier counter */
};

constexpr int kMaxHot = 128;       /* max heavy hitters per push */
constexpr int kEmSlots = 16;       /* max keys a push finds heavy within itself */

struct Options {
    int hot_keys = 128;        /* heavy hitters privatised per push, 0 = off */
    int hot_threshold = 0;     /* inserts per push that make a key hot, 0 = automatic */
    int warp_agg = 1;          /* direct path: combine equal keys within a warp */
    int ctas_per_sm = 8;       /* cap on co-resident CTAs per SM */
    int partition_bits = 0;    /* log2 groups per partition, 0 = automatic */
    int path = 0;              /* 0 auto, 1 partitioned, 2 direct atomics */
};

/* Parameters of one fused ingest/expire launch (one push). */
struct IngestArgs {
    const int32_t *keys;   /* effective batch: the last n_eff tuples of the push */
    const int32_t *vals;
    int64_t n;             /* n_eff <= W */
    int64_t slot0;         /* ring slot of the first effective tuple */
    int64_t hmod;          /* (old window head) mod W */
    int64_t old_len;       /* tuples in the old window, min(N, W) */
    int64_t fa, fb;        /* old-window offsets [fa, fb) whose expiry updates the front extrema */
    uint32_t epoch;        /* current min/max epoch */
    int minmax;            /* MIN or MAX requested */
};

/* launchers (cq_kernels.cu) */
cudaError_t launch_ingest(const DeviceState &d, const IngestArgs &a, const Options &o, int num_sms,
                          cudaStream_t s);
cudaError_t launch_finalize(const DeviceState &d, uint32_t epoch, int minmax, int avg, int num_sms,
                            cudaStream_t s);
cudaError_t launch_init_state(const DeviceState &d, int minmax, cudaStream_t s);
cudaError_t launch_reset_tags(const DeviceState &d, cudaStream_t s);
/* flip (cq_flip.cu): rebuild the front from stream indices [F, F + len) */
cudaError_t launch_flip(DeviceState &d, int64_t fmod, int64_t len, uint32_t epoch, cudaStream_t s,
                        int64_t *launches);
int64_t flip_scratch_bytes(int64_t W, int64_t G);
cudaError_t flip_alloc(DeviceState &d, cudaStream_t s);
void flip_free(DeviceState &d);

/* Exclusive scan of data[0, n) in place; partial holds ceil(n / 4096) + 1 words. */
cudaError_t exclusive_scan_u32(uint32_t *data, int64_t n, uint32_t *partial, cudaStream_t s, int64_t *launches);

}  // namespace cq

#endif
