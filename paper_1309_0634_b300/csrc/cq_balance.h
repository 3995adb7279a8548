/*
 * cq_balance.h -- the owner-computes mode's device-side lay-out and
 * rebalancing (cq_balance.cu), used by cq_owner.cu.  Not part of the public
 * ABI (include/cq.h).
 */
#ifndef CQ_BALANCE_H
#define CQ_BALANCE_H

#include "cq_internal.h"

namespace cq {

/* The thread-to-groups mapping as doubly linked lists: thread t's groups run
 * head[t], nxt[head[t]], ... (-1 ends a list), prv the reverse links, tail[t]
 * its last group, len[t] its length; own[g] the owner of group g. */
constexpr int kBalMaxThreads = 16384;   /* owner threads the policy CTA holds in shared memory */
struct BalStats {
    long long moves, last_moves, last_max, last_min;
};
/* One laid-out batch; two of them, used in turn, let the next batch be laid
 * out while the owner kernel still reads the last. */
struct LaySet {
    SortBuffers by_owner;        /* (owner, stream position, group), sorted by owner */
    uint32_t *ind = nullptr;     /* T + 1: each thread's first laid-out tuple, then n */
    int32_t *rv = nullptr;       /* cap: the values in laid-out order */
};
struct OwnerDev {
    int64_t G = 0;
    int T = 0;
    int32_t *own = nullptr, *nxt = nullptr, *prv = nullptr, *head = nullptr, *tail = nullptr, *len = nullptr;
    int32_t *count = nullptr;    /* G: each group's tuples in the batch */
    uint32_t *gstart = nullptr;  /* G: first position of a group's run in the by-group order */
    uint32_t *rank = nullptr;    /* cap: per stream position, the earlier tuples of its group */
    LaySet set[2];
    SortBuffers by_group;
    BalStats *st = nullptr;
    int *err = nullptr;
    int64_t cap = 0;
};
/* Allocates for G groups and T threads, uploads the mapping (h_own: G owners,
 * h_order: the groups thread by thread, h_off: T + 1 starts into it). */
cudaError_t owner_dev_alloc(OwnerDev &d, int64_t G, int T, const int32_t *h_off, const int32_t *h_order,
                            cudaStream_t s);
/* Room for batches of n tuples; the caller has drained the streams using it. */
cudaError_t owner_dev_reserve(OwnerDev &d, int64_t n, cudaStream_t s);
void owner_dev_free(OwnerDev &d);
/* Lays out n tuples (device keys in [0, G), values) by the current mapping
 * into set[si]: returns the index of its by_owner buffers holding (owner,
 * stream position, group) in thread order, stream order within a thread;
 * fills its ind and rv, count and, when `ranks`, the by-group sort's input.
 * -1 on a launch error. */
int owner_dev_lay_out(OwnerDev &d, int si, const int32_t *d_keys, const int32_t *d_vals, int64_t n, bool ranks,
                      cudaEvent_t after_map, cudaStream_t s, int64_t *launches);
/* After owner_dev_lay_out's map step (a stream waiting for after_map): each
 * tuple's rank among its group's tuples in the batch, by stream position. */
cudaError_t owner_dev_ranks(OwnerDev &d, int64_t n, cudaStream_t s, int64_t *launches);
/* One CTA runs the policy on the batch laid out in set[si] (buffer index idx). */
cudaError_t owner_dev_balance(OwnerDev &d, int si, int idx, int policy, int64_t threshold, double pot,
                              cudaStream_t s);
/* Copies the mapping back: off (T + 1) and the groups thread by thread. */
cudaError_t owner_dev_mapping(const OwnerDev &d, int32_t *off, int32_t *groups);

}  // namespace cq

#endif
