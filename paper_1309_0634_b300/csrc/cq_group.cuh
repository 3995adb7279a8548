/*
 * cq_group.cuh -- per-query descriptors of the partitioned push kernel
 * (cq_group.cu).  One cooperative launch serves any number of queries: it
 * walks a global list of chunks (phase A) and of key ranges (phase B) that
 * concatenates every query's work.
 */
#ifndef CQ_GROUP_CUH
#define CQ_GROUP_CUH

#include <stdint.h>

namespace cq {

constexpr int kGThreads = 512;      /* threads per CTA, two CTAs per SM */
constexpr int kGChunk = 2048;       /* max tuples per chunk */
constexpr int kGChunkReplace = 4096;/* max tuples per chunk of a window-replacing single-query launch */
constexpr int kGTable = 1024;       /* max groups per phase-B range */
constexpr int kGMaxParts = 1024;    /* max key-range partitions of a query */

/* QF_REPLACE: the push replaces the whole window (n >= W with tuples in it):
 * every old tuple leaves, so the new aggregates are those of the new tuples
 * alone; the evicted slots are not read and no retraction is formed, and
 * groups that held tuples but receive none are emptied. */
enum QFlags { QF_MINMAX = 1, QF_FRONT = 2, QF_AVG = 4, QF_ALIGNED = 8, QF_REPLACE = 16 };

/* A heavy hitter's updates of one push, summed by device atomics in phase A
 * into one of kHotRep replicas (chunk c into replica c mod kHotRep, which
 * keeps the contention on any one address low) and read, then reset to this
 * identity, by the key's owner in phase B. */
constexpr int kHotRep = 32;
struct __align__(32) HotAcc {
    long long sum;              /* inserted minus retracted values */
    int32_t ins, ret;           /* inserts, retracts */
    int32_t imin, imax;         /* extrema of the inserted values (INT32_MAX / INT32_MIN) */
    int32_t fdep, pad_;         /* front tuples that left (0) */
};

/* One query's share of a launch. */
struct QDesc {
    /* the push */
    const int32_t *keys, *vals;   /* the effective batch (last n of the pushed tuples) */
    int64_t n;
    int64_t slot0, hmod, old_len, fa, fb;
    int64_t G, W;
    int64_t S;                    /* tuples per chunk (multiple of 4) */
    int64_t stride;               /* deltas per chunk region of `stage` (even) */
    uint32_t epoch;
    int flags;                    /* QFlags */
    int rbits, P, C, ppp, R;      /* partitions of 2^rbits groups; C chunks; R ranges of ppp partitions */
    int chunk_base, range_base;   /* first global chunk / range of the query */
    int hot_cap;
    uint32_t hot_threshold;
    uint32_t hot_gthr;   /* inserts that guarantee a slot: more than n / hot_cap */
    uint32_t heavy_min, heavy_bound;   /* keys heavy within the push: per-run count, partition bound */
    /* device state */
    int32_t *ring_k, *ring_v;
    const int2 *sufs;             /* the front sorted by group (stream order within a group): per
                                     position, the (min, max) of the same group's later front tuples */
    int32_t *fptr;                /* per group: position in sufs of its oldest front tuple still in */
    unsigned long long *sum;
    int32_t *cnt;
    unsigned long long *bmin, *bmax, *fmin, *fmax;
    int32_t *rmin, *rmax;
    double *ravg;
    void *stage;                  /* C regions of `stride` deltas */
    uint32_t *off;                /* C rows of P + 1 offsets */
    HotAcc *hotacc;               /* kHotRep x kMaxHot accumulators, at identity between launches */
    int32_t *emkey;               /* keys found heavy within the push (cq_heavy.cuh) */
    HotAcc *emacc;                /* their kHotRep x kEmSlots accumulators */
    unsigned long long *emfolds;  /* runs folded so far */
    const int32_t *hot_cur;
    const int *hot_cur_n;
    const int32_t *hot_cur_cnt;
    int32_t *hot_next;
    int *hot_next_n;
    int32_t *hot_next_cnt;
    int *err, *err_host, *bad;    /* bad: keys outside [0, G) seen in phase A */
};

struct GroupArgs {
    QDesc q0;                     /* the query of a single-query launch */
    const QDesc *qs;              /* device array of nq descriptors (nq > 1) */
    const int *chunk_base;        /* nq + 1 prefix counts (nq > 1) */
    const int *range_base;        /* nq + 1 prefix counts (nq > 1) */
    int nq;
    int C_tot, R_tot;
    int grid;
    int maxP, maxC, tcap, dcap;   /* shared-memory sizing over the launch's queries */
    int maxS;                     /* largest chunk (tuples) */
    int dbuf;                     /* two chunk input sets (single-query launches) */
    int replace_all;              /* every query replaces its window: inputs and one delta per tuple */
    unsigned long long *bar;
    unsigned long long bar_target;
    unsigned long long *trace;    /* NULL, or grid x 8 phase stamps */
};

int64_t group_smem_bytes(int maxP, int maxC, int maxS, int tcap, int dcap, bool front, int nq, bool dbuf,
                         bool replace_all);
const void *group_kernel_ptr(bool front);

}  // namespace cq

#endif
