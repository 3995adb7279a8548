/*
 * cq_push.cuh -- parameters of the partitioned push kernel (cq_push.cu).
 */
#ifndef CQ_PUSH_CUH
#define CQ_PUSH_CUH

#include <stdint.h>

namespace cq {

constexpr int kPushThreads = 1024;                   /* threads per CTA (one CTA per SM) */
constexpr int kTPT = 4;                              /* tuples per thread per chunk */
constexpr int kChunkCap = kPushThreads * kTPT;       /* max tuples per chunk */
constexpr int kMaxParts = 1024;                      /* max key-range partitions */
constexpr int kMaxRBits = 11;                        /* max 2048 groups per partition */
constexpr int kMaxTable = 2048;                      /* max groups in a CTA's phase-B table */

/* Shape of one push: chunks (phase A work units) and partitions (phase B). */
struct PushPlan {
    int grid = 0;      /* CTAs, all co-resident (cooperative launch) */
    int rounds = 0;    /* chunks per CTA */
    int C = 0;         /* chunks = grid * rounds */
    int64_t S = 0;     /* tuples per chunk (the last one may be shorter) */
    int rbits = 0;     /* groups per partition = 2^rbits */
    int P = 0;         /* partitions = ceil(G / 2^rbits) */
    int tcap = 0;      /* groups a CTA aggregates per pass (phase B table) */
    int ppp = 0;       /* partitions per pass = tcap >> rbits */
    int dcap = 0;      /* deltas gathered per batch (<= 8192: exact 32-bit half sums) */
    int64_t stride = 0;/* deltas per chunk region of the staging buffer */
    int tma = 0;       /* 1: TMA-staged kernel */
    int64_t smem = 0;  /* dynamic shared memory per CTA */
};

struct PushArgs {
    const int32_t *keys;   /* effective batch */
    const int32_t *vals;
    int64_t n;             /* effective tuples */
    int64_t slot0, hmod, old_len, fa, fb;
    int64_t G, W;
    uint32_t epoch;
    int avg;
    int grid, rounds, C;
    int64_t S;
    int rbits, P;
    int tcap, ppp, dcap;
    int64_t stride;
    int32_t *ring_k, *ring_v;
    const int2 *sufs;             /* the front sorted by group: (min, max) of the same group's later tuples */
    int32_t *fptr;                /* per group: position in sufs of its oldest front tuple still in */
    unsigned long long *sum;
    int32_t *cnt;
    unsigned long long *bmin, *bmax, *fmin, *fmax;
    int32_t *rmin, *rmax;
    double *ravg;
    void *stage;           /* C chunks x 2S deltas */
    uint32_t *off;         /* C rows of P + 1 offsets */
    void *hotpart;         /* [hot key][CTA] partial records */
    const int32_t *hot_cur;
    const int *hot_cur_n;
    const int32_t *hot_cur_cnt;   /* insert counts of hot_cur at detection */
    int32_t *hot_next;
    int *hot_next_n;
    int32_t *hot_next_cnt;
    int32_t *emkey;        /* keys found heavy within the push (cq_heavy.cuh) */
    void *emacc;           /* their kHotRep x kEmSlots accumulators */
    unsigned long long *emfolds;   /* runs folded so far */
    int hot_cap;
    uint32_t hot_threshold;
    uint32_t hot_gthr;   /* inserts that guarantee a slot: more than n / hot_cap */
    uint32_t heavy_min, heavy_bound;   /* keys heavy within the push: per-run count, partition bound */
    unsigned long long *bar;      /* [0] grid-barrier arrivals, [1] phase-B range draws (both only grow) */
    unsigned long long bar_target;
    unsigned long long draw_base; /* range draws before this launch */
    int *err, *err_host;
    unsigned long long *trace;   /* NULL, or grid x 8 phase stamps */
};

int64_t push_smem_bytes(const PushPlan &pl, bool front);
int push_delta_cap(bool front);
const void *push_kernel_ptr(bool minmax, bool front);
int64_t hot_rec_bytes();

}  // namespace cq

#endif
