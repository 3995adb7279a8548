"""cq_push_noalloc against cq_push: the same batches, two calls in a row, give
bit-identical results, and the no-allocation push leaves device memory as it was.

Collected last (file name) so that it also runs after every other GPU test in
one process; it creates all it needs itself, so it passes alone as well."""
import numpy as np
import pytest

import oracle
import paper_1309_0634_b300 as cq
import streamgen
from gpu_util import assert_same

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()


CASES = [
    # groups, window, first batch, second batch, aggregates, key distribution, Zipf s
    (1000, 10_000, 6_000, 7_000, cq.CQ_ALL, "zipf", 1.5),          # the second call flips the front stack
    (777, 3_333, 5_000, 100, cq.CQ_ALL, "zipf", 1.0),              # batch longer than the window; unaligned ring
    (100_000, 1_000_000, 500_000, 500_000, cq.CQ_ALL, "uniform", 0.0),
    (50_000, 200_000, 150_000, 120_000, cq.CQ_SUM | cq.CQ_COUNT | cq.CQ_AVG, "zipf", 2.0),
    (1, 64, 1, 63, cq.CQ_MIN | cq.CQ_MAX, "uniform", 0.0),
    (20_000, 300_000, 100_000, 300_000, cq.CQ_ALL, "zipf", 1.5),   # the second call replaces the whole window
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_noalloc_matches_push_two_calls_in_a_row(case):
    G, W, n1, n2, aggs, keys, s = CASES[case]
    st = streamgen.Stream(G, keys=keys, s=s, vals="uniform", lo=-10**6, hi=10**6, seed=100 + case)
    k1, v1 = st.fill(0, n1)
    k2, v2 = st.fill(n1, n2)
    o = oracle.Oracle(G, W)
    assert o.push(k1, v1) == 0 and o.push(k2, v2) == 0
    d = [(_dev(k1), _dev(v1)), (_dev(k2), _dev(v2))]
    qa, qb = cq.Query(G, W, aggs), cq.Query(G, W, aggs)
    try:
        for k, v in d:                       # two calls in a row, no sync between
            assert qa.push(k, v) == cq.CQ_OK
        for k, v in d:
            assert qb.push_noalloc(k, v) == cq.CQ_OK
        ra, rb = qa.results(), qb.results()
        assert_same(rb, ra, aggs, where="no-alloc vs push")
        assert_same(rb, o.results(), aggs, where="no-alloc vs oracle")
        sa, sb = qa.stats(), qb.stats()
        for f in ("tuples_seen", "window_len", "pushes", "flips", "resets"):
            assert sa[f] == sb[f], f
    finally:
        qa.close()
        qb.close()


def test_noalloc_allocates_nothing():
    """A push larger than any before grows cq_push's scratch, never the fixed area's."""
    import torch
    G, W = 100_000, 1_000_000
    st = streamgen.Stream(G, keys="zipf", s=1.5, vals="uniform", lo=-1000, hi=1000, seed=7)
    small = [_dev(a) for a in st.fill(0, 1_000)]
    big = [_dev(a) for a in st.fill(1_000, 600_000)]
    q = cq.Query(G, W)
    try:
        assert q.push_noalloc(*small) == cq.CQ_OK   # first call: looks up the area, loads the kernels
        assert q.sync() == cq.CQ_OK
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert q.push_noalloc(*big) == cq.CQ_OK
        assert q.sync() == cq.CQ_OK
        assert torch.cuda.mem_get_info()[0] == free0
    finally:
        q.close()


def test_noalloc_rejects_oversize_batch_and_leaves_query_unchanged():
    G, W = 100_000, 2_000_000
    st = streamgen.Stream(G, keys="uniform", vals="uniform", lo=-1000, hi=1000, seed=8)
    k0, v0 = st.fill(0, 10_000)
    kb, vb = st.fill(10_000, 1_000_000)         # ~32 bytes a tuple: more than the area holds
    o = oracle.Oracle(G, W)
    assert o.push(k0, v0) == 0
    q = cq.Query(G, W)
    try:
        assert q.push_noalloc(_dev(k0), _dev(v0)) == cq.CQ_OK
        before = q.stats()
        assert q.push_noalloc(_dev(kb), _dev(vb)) == cq.CQ_ESCRATCH
        assert "scratch" in cq.cq_strerror(cq.CQ_ESCRATCH)
        after = q.stats()
        for f in ("tuples_seen", "window_len", "pushes", "flips", "resets", "kernel_launches"):
            assert after[f] == before[f], f
        assert_same(q.results(), o.results(), cq.CQ_ALL, where="after rejection")
        # the query still takes a batch that fits
        k1, v1 = st.fill(1_010_000, 300_000)
        assert o.push(k1, v1) == 0
        assert q.push_noalloc(_dev(k1), _dev(v1)) == cq.CQ_OK
        assert_same(q.results(), o.results(), cq.CQ_ALL, where="after a fitting push")
    finally:
        q.close()


def test_noalloc_rejects_key_space_beyond_the_kernel():
    q = cq.Query(2**21 + 5, 1000)
    try:
        k = _dev(np.arange(100, dtype=np.int32))
        assert q.push_noalloc(k, k) == cq.CQ_ESCRATCH
        assert q.stats()["tuples_seen"] == 0
        assert q.push_noalloc(k[:0], k[:0]) == cq.CQ_OK
    finally:
        q.close()
