"""Helpers of the GPU parity tests: run a stream through the CUDA path and the
oracle side by side and compare every result bit for bit."""
import numpy as np

import oracle
import paper_1309_0634_b300 as cq

FIELDS = ("sum", "count", "min", "max", "avg")
AGG_FIELDS = {cq.CQ_SUM: ("sum",), cq.CQ_COUNT: ("count",), cq.CQ_MIN: ("min",), cq.CQ_MAX: ("max",),
              cq.CQ_AVG: ("avg",)}


def fields_of(aggs):
    out = []
    for bit, names in AGG_FIELDS.items():
        if aggs & bit:
            out.extend(names)
    return out


def assert_same(gpu, ref, aggs=cq.CQ_ALL, where=""):
    """Bitwise equality of the requested aggregates (AVG compared as bits)."""
    for f in fields_of(aggs):
        a, b = gpu[f], ref[f]
        if f == "avg":
            a, b = a.view(np.uint64), b.view(np.uint64)
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0]
            g = int(bad[0])
            raise AssertionError("%s %s differs at %d groups, first g=%d: gpu %r oracle %r (count gpu %d oracle %d)"
                                 % (where, f, bad.size, g, gpu[f][g], ref[f][g], gpu["count"][g], ref["count"][g]))


def run_pair(groups, window, batches, aggs=cq.CQ_ALL, check_every=1, options=None, host=False):
    """Push the (keys, vals) batches to a GPU query and to the oracle; compare
    after every `check_every` pushes and after the last one."""
    import torch
    q = cq.Query(groups, window, aggs, **(options or {}))
    o = oracle.Oracle(groups, window)
    checked = -1
    i = -1
    try:
        for i, (k, v) in enumerate(batches):
            if host:
                st = q.push(np.asarray(k), np.asarray(v))
            else:
                kt = torch.from_numpy(np.ascontiguousarray(k, np.int32)).cuda()
                vt = torch.from_numpy(np.ascontiguousarray(v, np.int32)).cuda()
                st = q.push(kt, vt)
            assert st == cq.CQ_OK, (i, st)
            assert o.push(k, v) == 0
            if (i + 1) % check_every == 0:
                assert_same(q.results(), o.results(), aggs, where="push %d" % i)
                checked = i
        if checked != i:
            assert_same(q.results(), o.results(), aggs, where="push %d" % i)
        return q.stats()
    finally:
        q.close()
