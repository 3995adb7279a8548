/*
 * cq_stream.cuh -- descriptors of the persistent multi-batch push
 * (cq_stream.cu): one cooperative launch folds a whole sequence of batches
 * of one query into its window, batch after batch, in stream order.
 *
 * The launch holds two CTAs per SM with two roles:
 *   producers (one per SM, two on some SMs when a skewed stream makes
 *   cutting the batch the slower role) cut every batch into chunks, counting-sort each
 *   chunk's deltas by key range into runs (the paper's two-pass reordering
 *   of a batch, Section 3.1, done per chunk on the device), write the runs
 *   and the chunk's run table row to a scratch slot and the new tuples to
 *   the window ring;
 *   consumers (one per SM) each own one key range of the query's groups for
 *   the whole launch, with its per-group state in shared memory; per batch
 *   a consumer gathers its runs from every chunk, folds them and rewrites
 *   the results of its touched groups.
 * Producers and consumers meet through per-slot arrival counters instead of
 * a grid barrier: kSSlots batches can be in flight, so producers cut batch
 * i + 1 while consumers fold batch i.
 */
#ifndef CQ_STREAM_CUH
#define CQ_STREAM_CUH

#include <stdint.h>

#include "cq_group.cuh"
#include "cq_internal.h"

namespace cq {

constexpr int kSThreads = 512;             /* threads of a producer or a consumer CTA */
constexpr int kSSlots = 4;                 /* scratch slots: batches in flight between the roles */
constexpr int kSRefresh = 16;              /* batches between heavy-hitter list refreshes */
constexpr int kSMaxBatches = 2048;         /* batches of one launch */
constexpr int kSListSlots = 3;             /* list slots: two alternating refreshes, the hand-off list */
constexpr int kSListN = kSMaxBatches / kSRefresh + 2;   /* refresh lists of a launch (+ the hand-off list) */
constexpr int kSSmem = 110 * 1024;         /* dynamic shared memory of every CTA: two CTAs per SM */
constexpr int kSMinChunk = 256;            /* least tuples per chunk */
constexpr int kSMaxChunk = 8192;           /* most tuples per chunk (16-bit ranks, exact half sums) */

/* SB_REPLACE: every old tuple leaves (the batch fills the window and the
 *   window held tuples): no evicted slot is read, and the new state of a
 *   group is that of the batch's tuples alone.
 * SB_RING: old tuples leave the window: each chunk reads the ring slots it
 *   overwrites and retracts their tuples.
 * SB_FRONT: some leaving tuples leave the front segment of the MIN/MAX
 *   structure: their retracts carry the front-departure bit.
 * SB_ALIGNED: the batch and its ring slots allow 16-byte bulk copies. */
enum SFlags { SB_REPLACE = 1, SB_RING = 2, SB_FRONT = 4, SB_ALIGNED = 8 };

/* One batch of a launch, built by the host (window bookkeeping of cq_api.cu). */
struct SBatch {
    const int32_t *keys, *vals;   /* the effective batch: the last n of the pushed tuples */
    int32_t n;                    /* effective tuples, <= W */
    int32_t S, C;                 /* tuples per chunk (multiple of 4), chunks */
    int32_t slot0;                /* ring slot of the first effective tuple */
    int32_t hmod;                 /* (old window head) mod W */
    int32_t old_len;              /* tuples in the old window */
    int32_t fa, fb;               /* old-window offsets [fa, fb) whose departure shrinks the front */
    uint32_t epoch;               /* MIN/MAX epoch of the batch */
    int32_t flags;                /* SFlags */
    int32_t ring_dep;             /* batch of this launch whose ring writes must be complete before this
                                     batch touches the ring (-1: none of this launch) */
    uint32_t hot_threshold;       /* inserts that make a key a heavy hitter of a later batch */
    uint32_t hot_gthr;            /* inserts that make it sure of a list slot */
    int32_t pad_[3];              /* 80 bytes: copied to shared memory in 16-byte pieces */
};
static_assert(sizeof(SBatch) % 16 == 0, "batch descriptors are copied in 16-byte pieces");

/* Arrival counters and role words of a launch (64-bit words, zeroed before
 * every launch). */
enum SCtl {
    SC_A = 0,                      /* [kSSlots] producer arrivals per slot */
    SC_B = kSSlots,                /* [kSSlots] consumer arrivals per slot */
    SC_ROLE_A = 2 * kSSlots,       /* producers so far */
    SC_ROLE_B,                     /* consumers so far */
    SC_ABORT,                      /* set by a CTA whose wait gave up: every CTA leaves */
    SC_PP,                         /* second CTAs of an SM made producers so far */
    SC_SM,                         /* [kSSmSlots] CTAs placed on each SM so far (by %smid) */
    SC_CLAIM = SC_SM + 512,        /* [kSMaxBatches] chunks of each batch claimed so far */
    SC_FLAG = SC_CLAIM + kSMaxBatches,   /* [kSSlots][1024] 1 when producer p cut chunks of the slot's batch */
    SC_END = SC_FLAG + kSSlots * 1024
};
constexpr int kSSmSlots = SC_CLAIM - SC_SM;   /* %smid values the placement counts cover */

struct SArgs {
    const SBatch *b;              /* nb batch descriptors (device) */
    int nb;
    int64_t G, W;
    int minmax, avg;
    int nA, nB;                   /* producers, consumers: grid = nA + nB, two CTAs per SM: a producer
                                     and a consumer, or on (nA - nB) / 2 SMs two producers */
    int R;                        /* key ranges, one per consumer (R <= nB) */
    uint32_t M;                   /* range of key k: __umulhi(k, M) */
    int tcap;                     /* groups of the largest range */
    int Smax;                     /* tuples of the longest chunk */
    int Cpad;                     /* entries of a run-table row: most chunks of a batch, even */
    int64_t stride;               /* deltas of one chunk's region of a stage slot (even) */
    int dcap;                     /* deltas gathered per round by a consumer */
    int ring_any;                 /* some batch has SB_RING */
    uint32_t epoch0;              /* epoch before the first batch: decodes the stored extrema */
    int64_t stage_slot;           /* deltas of one stage slot */
    int64_t pairs_slot;           /* run-table entries of one slot */
    /* query state */
    int32_t *ring_k, *ring_v;
    const int2 *sufs;             /* the front sorted by group: (min, max) of the same group's later tuples */
    int32_t *fptr;                /* per group: position in sufs of its oldest front tuple still in */
    unsigned long long *sum;
    int32_t *cnt;
    unsigned long long *bmin, *bmax, *fmin, *fmax;
    int32_t *rmin, *rmax;
    double *ravg;
    /* scratch */
    void *stage;                  /* [kSSlots][stage_slot] deltas */
    uint2 *pairs;                 /* [kSSlots][R][Cpad] (begin, padded length) of each chunk's run */
    HotAcc *hotpart;              /* [kSSlots][nA][kMaxHot] producers' heavy-hitter partials */
    /* Heavy-hitter lists.  Batch i < kSSlots privatises the query's list;
       batch i >= kSSlots the list found by batch m * kSRefresh, m =
       (i - kSSlots) / kSRefresh (list slot m % 2, counts list_n[m]).  The
       last batch also lists its heavy hitters in slot 2 (counts
       list_n[kSListN - 1]): the query's list after the launch. */
    int32_t *lists;               /* [kSListSlots][2 tiers][kMaxHot] keys */
    int32_t *list_cnt;            /* their insert counts, laid out as lists */
    int *list_n;                  /* [kSListN][2] entries appended per list and tier */
    const int32_t *q_hot, *q_hot_cnt;   /* the query's list (2 tiers) */
    const int *q_hot_n;
    int hot_cap;
    unsigned long long *ctl;      /* SCtl words */
    int *err, *err_host;          /* sticky error word (1 bad key, 2 timeout) and its host mirror */
    unsigned long long wait_ns;   /* bound of every wait */
    int stall_batch;              /* test hook: producer 0 never reports this batch (-1: off) */
    /* optional per-batch outputs (NULL: not wanted) */
    int64_t *snap_sum;            /* [nb][G] results after each batch */
    int32_t *snap_cnt, *snap_min, *snap_max;
    double *snap_avg;
    unsigned long long *stamp_begin;   /* [nb]: when the first producer began a batch (%globaltimer ns) */
    unsigned long long *stamp_end;     /* [nb]: when the last consumer finished it */
    unsigned long long *trace;         /* NULL, or [nA + nB][nb][12] phase stamps (producers first) */
};

/* First key of key range r (r = 0 .. R): the least k whose range
 * __umulhi(k, M) = floor(k * M / 2^32) is r or more; G for r = R when
 * M <= R * 2^32 / G.  The ranges partition [0, G) for any M >= 1. */
__host__ __device__ inline int64_t stream_range_lo(uint32_t r, uint32_t M, int64_t G) {
    const unsigned long long x = (((unsigned long long)r << 32) + M - 1) / M;
    return (int64_t)x < G ? (int64_t)x : G;
}

/* Shared-memory bytes a launch needs (the larger of the two roles), or -1 if
 * it does not fit kSSmem. */
int64_t stream_smem_bytes(int Smax, int R, int tcap, int Cpad, int dcap, bool ring, int ds, bool minmax);
/* Tuples per chunk that fit kSSmem for a launch of R ranges. */
int stream_max_chunk(int R, bool ring, int ds);
/* Groups per range a consumer can hold with `dcap` gathered deltas of `ds` bytes. */
int stream_max_range(int Cpad, int dcap, int ds, bool minmax);
/* Launch over a.nA + a.nB CTAs with ds-byte deltas (8). */
cudaError_t launch_stream(const SArgs &a, int ds, cudaStream_t s);
/* Whether the launch's two roles fit exactly two CTAs per SM of the current
 * device (false: cq_push_many pushes batch by batch). */
bool stream_launchable();

}  // namespace cq

#endif
