"""Queries driven from several host threads at once.

Different queries may be pushed concurrently (one thread per query, no
locking per query).  The first push of a shape raises its kernel's
dynamic shared-memory limit on the device; two threads doing that at once
for kernels of different needs must both end with a limit that covers
their launch.  Each thread's query is compared with the oracle after every
push.
"""
import threading

import numpy as np
import pytest

import oracle
import paper_1309_0634_b300 as cq
import streamgen
from gpu_util import assert_same

pytestmark = pytest.mark.gpu


def _drive(G, W, sizes, seed, aggs, options, errors, barrier):
    import torch
    try:
        stream = torch.cuda.Stream()
        st = streamgen.Stream(G, keys="zipf", s=1.1, vals="uniform", lo=-10**6, hi=10**6, seed=seed)
        q = cq.Query(G, W, aggs, stream=stream, **options)
        o = oracle.Oracle(G, W)
        try:
            t = 0
            batches = []
            for b in sizes:
                batches.append(st.fill(t, b))
                t += b
            barrier.wait(timeout=120)   # the first pushes of both threads start together
            for i, (k, v) in enumerate(batches):
                with torch.cuda.stream(stream):
                    kt = torch.from_numpy(k).cuda()
                    vt = torch.from_numpy(v).cuda()
                stream.synchronize()
                assert q.push(kt, vt) == cq.CQ_OK, (G, i)
                assert q.sync() == cq.CQ_OK
                o.push(k, v)
                assert_same(q.results(), o.results(), aggs, where="G=%d push %d" % (G, i))
        finally:
            q.close()
    except Exception as exc:   # reported by the main thread
        errors.append((G, repr(exc)))


@pytest.mark.parametrize("shapes", [
    # (groups, window, batch sizes, aggregates, options)
    ((300, 6_000, [2_000, 4_000, 6_000, 1_000, 5_000], cq.CQ_ALL, {}),
     (120_000, 300_000, [100_000, 150_000, 90_000, 160_000], cq.CQ_ALL, {})),
    ((40_000, 80_000, [30_000, 50_000, 70_000], cq.CQ_SUM | cq.CQ_COUNT, {"path": 1}),
     (5_000, 50_000, [20_000, 40_000, 10_000, 35_000], cq.CQ_MIN | cq.CQ_MAX, {"path": 3})),
])
def test_two_threads_push_queries_of_different_shared_memory_needs(shapes):
    errors = []
    barrier = threading.Barrier(len(shapes))
    threads = [threading.Thread(target=_drive, args=(G, W, sizes, 40 + j, aggs, opts, errors, barrier))
               for j, (G, W, sizes, aggs, opts) in enumerate(shapes)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=600)
        assert not th.is_alive()
    assert not errors, errors
