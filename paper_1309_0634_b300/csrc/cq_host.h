/*
 * cq_host.h -- host-side hooks of the query library used by the serving loop
 * (cq_serve.cu).  Not part of the C ABI.
 */
#ifndef CQ_HOST_H
#define CQ_HOST_H

#include <cuda_runtime.h>
#include <stdint.h>

#include "cq.h"

namespace cq {

/* Device bytes the partitioned kernel's scratch can need for any batch of at
 * most max_batch tuples of a query of `groups` groups pushed in a group
 * launch; -1 when the group kernel cannot take such a query. */
int64_t group_scratch_bound(int64_t groups, int64_t window, int64_t max_batch);

/* Grow q's scratch to group_scratch_bound now, so that later group pushes of
 * batches up to max_batch allocate nothing. */
cudaError_t reserve_group_scratch(cq_query *q, int64_t max_batch);

/* Launch g's pushes directly, never from a captured CUDA graph. */
void group_disable_graphs(cq_group *g);

/* The stream q's work is ordered on. */
cudaStream_t query_stream(const cq_query *q);

}  // namespace cq

#endif
