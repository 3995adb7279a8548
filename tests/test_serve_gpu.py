"""The serving loop: admission by device footprint, continuous batching of
requests from many queries, and results identical to each query pushed alone."""
import numpy as np
import pytest

import oracle
import paper_1309_0634_b300 as cq
import streamgen
from streamgen import workloads
from gpu_util import assert_same

pytestmark = pytest.mark.gpu

GIB = 1 << 30


def _dev(a):
    """A device copy, complete before return (the server launches on its own stream)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
    torch.cuda.current_stream().synchronize()
    return t


def _small_specs(nq, seed=5, max_window=400_000, max_groups=200_000):
    """Queries of the serving configuration, windows and key spaces capped so
    that the oracle keeps up in a test."""
    out = []
    for sp in workloads.multi_query(nq, seed=seed, batches=0, prefix="t"):
        out.append((min(sp.groups, max_groups), min(sp.window, max_window), sp.stream_kw))
    return out


def test_serving_matches_each_query_alone():
    nq, pool_len, max_batch = 24, 1 << 17, 60_000
    specs = _small_specs(nq)
    qs_, idx, arr, sizes = workloads.serving_requests(nq, 0.25, tuples_per_s=4e8, seed=11, max_batch=max_batch)
    assert len(qs_) > 200
    pools = []
    for q, (G, W, kw) in enumerate(specs):
        k, v = streamgen.Stream(G, **kw).fill(0, pool_len)
        pools.append((k, v, _dev(k), _dev(v)))
    srv = cq.Server(64 * GIB)
    served = [srv.admit(G, W, cq.CQ_ALL, max_batch) for G, W, _ in specs]
    keys, vals, queries = [], [], []
    per_query = [[] for _ in range(nq)]
    for q, i, n in zip(qs_, idx, sizes):
        o = workloads.serving_pool_offset(int(q), int(i), int(n), pool_len)
        keys.append(pools[q][2][o:o + n])
        vals.append(pools[q][3][o:o + n])
        queries.append(served[q])
        per_query[q].append((o, int(n)))
    try:
        assert srv.replay(queries, arr, keys, vals) == cq.CQ_OK
        st = srv.stats()
        assert st["completed"] == st["submitted"] == len(qs_)
        assert st["tuples"] == int(sizes.sum())
        assert st["batches_launched"] == len(qs_)
        assert st["launches"] <= len(qs_)
        assert 0 < st["latency_p50_us"] <= st["latency_p99_us"] <= st["latency_max_us"]
        # every query against the oracle; the first eight also against the same batches pushed alone
        for q in range(nq):
            G, W, _ = specs[q]
            o_ = oracle.Oracle(G, W)
            alone = cq.Query(G, W) if q < 8 else None
            for off, n in per_query[q]:
                k, v = pools[q][0][off:off + n], pools[q][1][off:off + n]
                assert o_.push(k, v) == 0
                if alone is not None:
                    assert alone.push(pools[q][2][off:off + n], pools[q][3][off:off + n]) == cq.CQ_OK
            r = served[q].results()
            assert_same(r, o_.results(), cq.CQ_ALL, where="served query %d vs oracle" % q)
            if alone is not None:
                assert_same(r, alone.results(), cq.CQ_ALL, where="served query %d vs alone" % q)
                alone.close()
    finally:
        srv.close()


def test_serving_admission_by_footprint():
    G, W, B = 50_000, 1_000_000, 100_000
    one = cq.cq_footprint_bytes(G, W, cq.CQ_ALL)
    assert one > 0
    probe = cq.Server(64 * GIB)
    probe.admit(G, W, cq.CQ_ALL, B)
    need = probe.stats()["reserved_bytes"]          # state plus the scratch of a B-tuple batch
    probe.close()
    assert need > one
    srv = cq.Server(int(2.5 * need))
    try:
        a = srv.admit(G, W, cq.CQ_ALL, B)
        b = srv.admit(G, W, cq.CQ_ALL, B)
        reserved = srv.stats()["reserved_bytes"]
        assert reserved == 2 * need
        with pytest.raises(cq.CQError) as e:
            srv.admit(G, W, cq.CQ_ALL, B)
        assert e.value.status == cq.CQ_EBUDGET
        assert srv.stats()["reserved_bytes"] == reserved and srv.stats()["queries"] == 2
        # a smaller query still fits in what is left
        c = srv.admit(100, 1000, cq.CQ_SUM, 1000)
        assert srv.stats()["queries"] == 3
        with pytest.raises(cq.CQError):
            srv.admit(2**20 + 1, 1000, cq.CQ_ALL, 100)     # beyond the group kernel
        # batches above the declared maximum are refused
        k = _dev(np.zeros(B + 1, np.int32))
        with pytest.raises(cq.CQError):
            srv.submit(a, k, k)
        del b, c
    finally:
        srv.close()


def test_serving_tickets_order_and_bad_key():
    G, W = 1000, 20_000
    srv = cq.Server(8 * GIB)
    good = srv.admit(G, W, cq.CQ_ALL, 10_000)
    bad = srv.admit(10, 100, cq.CQ_ALL, 100)
    o = oracle.Oracle(G, W)
    st = streamgen.Stream(G, keys="zipf", s=1.2, vals="uniform", lo=-500, hi=500, seed=3)
    try:
        tickets, held = [], []
        for i in range(30):
            k, v = st.fill(i * 7_000, 7_000)
            assert o.push(k, v) == 0
            kd, vd = _dev(k), _dev(v)
            held.append((kd, vd))
            tickets.append(srv.submit(good, kd, vd))
            if i == 5:
                kb = _dev(np.array([3, 99], np.int32))
                held.append((kb, kb))
                # the bad key is found when its launch runs: later batches of the query are refused
                assert srv.wait(srv.submit(bad, kb, kb)) == cq.CQ_OK
            if i > 5 and i % 4 == 0:
                kb = _dev(np.array([1], np.int32))
                held.append((kb, kb))
                t_bad = srv.submit(bad, kb, kb)
        for t in tickets:
            assert srv.wait(t) == cq.CQ_OK
        assert srv.wait(t_bad) in (cq.CQ_EKEY, cq.CQ_EPOISONED)
        assert srv.drain() == cq.CQ_OK
        assert_same(good.results(), o.results(), cq.CQ_ALL, where="good query")
        assert srv.reset_stats() == cq.CQ_OK
        assert srv.stats()["submitted"] == 0
    finally:
        srv.close()


def test_serving_every_batch_in_the_mix_matches_oracle_and_alone():
    """Round by round, one batch of every query is submitted and the round's
    tickets are awaited; the pending batches of a round go through the
    dispatcher's continuous batching together.  After every round each of 16
    queries (windows and key spaces capped for the oracle) is compared with
    the oracle, and 4 queries at their full serving-configuration sizes (the
    largest windows of the configuration, up to 10^7 tuples and 10^6 groups)
    on rounds 1, 3 and 5; eight of the queries, two of them full-size, are
    also compared with the same batches pushed alone, after every round."""
    import torch
    full = sorted(workloads.config5(), key=lambda sp: -sp.window)[:4]
    capped = _small_specs(16, seed=17, max_window=300_000, max_groups=150_000)
    specs = [(G, W, kw, False) for G, W, kw in capped] + [(sp.groups, sp.window, sp.stream_kw, True) for sp in full]
    assert max(W for _, W, _, f in specs if f) >= 5_000_000
    nq = len(specs)
    srv = cq.Server(96 * GIB)
    served = [srv.admit(G, W, cq.CQ_ALL, 10**6) for G, W, _, _ in specs]
    streams = [streamgen.Stream(G, **kw) for G, _, kw, _ in specs]
    oracles = [oracle.Oracle(G, W) for G, W, _, _ in specs]
    alone_ids = list(range(6)) + [16, 17]
    alone = {q: cq.Query(specs[q][0], specs[q][1]) for q in alone_ids}
    t = [0] * nq
    try:
        for rnd in range(6):
            tickets, held = [], []
            for q in range(nq):
                n = workloads.serving_batch_size(q, rnd, seed=17)
                if not specs[q][3]:
                    n = min(n, 200_000)
                k, v = streams[q].fill(t[q], n)
                t[q] += n
                assert oracles[q].push(k, v) == 0
                kd, vd = _dev(k), _dev(v)
                held.append((kd, vd))
                tickets.append(srv.submit(served[q], kd, vd))
                if q in alone:
                    assert alone[q].push(kd, vd) == cq.CQ_OK
            for tk in tickets:
                assert srv.wait(tk) == cq.CQ_OK
            torch.cuda.synchronize()
            for q in range(nq):
                r = served[q].results()
                if not specs[q][3] or rnd % 2 == 1:
                    assert_same(r, oracles[q].results(), cq.CQ_ALL, where="round %d query %d vs oracle" % (rnd, q))
                if q in alone:
                    assert_same(r, alone[q].results(), cq.CQ_ALL, where="round %d query %d vs alone" % (rnd, q))
        st = srv.stats()
        assert st["completed"] == st["submitted"] == 6 * nq
    finally:
        for a in alone.values():
            a.close()
        srv.close()
