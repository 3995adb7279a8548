"""Placement of independent standing queries on the GPUs of a multi-GPU job.

Queries do not share state, so a set of them shards by query with no
exchange at all: each query lives on one rank's GPU, its batches go there,
and only timing (the slowest rank) is reduced across ranks.  This is the
paper's partitioned (intra-operator) parallelism over groups (Section 1,
Section 3.1) lifted one level: whole queries are the units of work.

``assign_queries`` is longest-processing-time-first list scheduling: queries
in order of decreasing weight, each to the rank with the least weight so far
(ties: the least memory so far, then the lowest rank).  Every rank computes
the same assignment from the same inputs, so no rank needs to tell another.
The heaviest rank then carries at most the mean load plus one query's weight.
"""
from __future__ import annotations


def assign_queries(weights, world: int, memory=None):
    """Ranks' query lists (indices into ``weights``), each list ascending.

    ``weights``: work per query (any non-negative numbers, e.g. bytes moved
    per round); ``memory``: device bytes per query for tie-breaks (None: all
    equal); ``world``: number of ranks (>= 1)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    n = len(weights)
    mem = list(memory) if memory is not None else [0] * n
    if len(mem) != n:
        raise ValueError("memory must have one entry per query")
    order = sorted(range(n), key=lambda q: (-float(weights[q]), -float(mem[q]), q))
    load = [0.0] * world
    used = [0.0] * world
    out = [[] for _ in range(world)]
    for q in order:
        r = min(range(world), key=lambda k: (load[k], used[k], k))
        out[r].append(q)
        load[r] += float(weights[q])
        used[r] += float(mem[q])
    return [sorted(x) for x in out]


def round_bytes(groups: int, window: int, batch: int) -> float:
    """Work of one round of a query of the batched workload: the algorithmic
    bytes of one push once its window is full (8 B read and 8 B written per
    new tuple, 8 B read per expired tuple, 68 B per touched group, at most
    the groups or the tuples that can touch them)."""
    b = min(batch, window)
    touched = min(groups, 2 * b)
    return 24.0 * b + 68.0 * touched
