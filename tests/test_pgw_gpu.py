"""One window per group (the paper's own workload): every tuple's output --
its group's window SUM right after it entered -- matches the oracle bit for
bit, for uniform, round-robin and heavily skewed keys."""
import numpy as np
import pytest

import oracle
import paper_1309_0634_b300 as cq
import streamgen
from streamgen import workloads

pytestmark = pytest.mark.gpu


def _dev(a, dtype=np.int32):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype)).cuda()


def _run(G, w, passes, batches, keys="zipf", s=1.2, seed=0, vals=None):
    import torch
    q = cq.GroupWindows(G, w, passes)
    o = oracle.WindowsOracle(G, w, passes)
    st = streamgen.Stream(G, keys=keys, s=s, vals="uniform", lo=-2**31, hi=2**31 - 1, seed=seed) if vals is None \
        else streamgen.Stream(G, keys=keys, s=s, vals=vals, seed=seed)
    t = 0
    try:
        for i, n in enumerate(batches):
            k, v = st.fill(t, n)
            t += n
            ost, expect = o.push(k, v)
            assert ost == 0
            out = torch.empty(n, dtype=torch.int64, device="cuda")
            assert q.push(_dev(k), _dev(v), out) == cq.CQ_OK
            assert q.sync() == cq.CQ_OK
            got = out.cpu().numpy()
            bad = np.nonzero(got != expect)[0]
            assert bad.size == 0, "batch %d: %d wrong, first at %d: %d != %d" % (
                i, bad.size, bad[0], got[bad[0]], expect[bad[0]])
        assert q.stats()["tuples_seen"] == t
    finally:
        q.close()


@pytest.mark.parametrize("G,w,passes", [(1, 1, 1), (1, 7, 2), (7, 5, 1), (1000, 100, 1), (40_000, 100, 10),
                                        (3, 1000, 1), (50_000, 2, 1), (5_000_000, 2, 1)])
def test_pgw_matches_oracle_ragged(G, w, passes):
    rng = np.random.default_rng(G + w)
    batches = [0, 1, 3, int(rng.integers(1, 5000)), 20_000, 1, 70_000, 0, 12_345]
    _run(G, w, passes, batches, seed=G * 7 + w)


@pytest.mark.parametrize("keys,s", [("uniform", 0.0), ("round_robin", 0.0), ("zipf", 2.0)])
def test_pgw_key_distributions(keys, s):
    _run(5_000, 64, 1, [30_000] * 6, keys=keys, s=s, seed=11)


@pytest.mark.parametrize("name", ["DS1", "DS2", "DS3"])
def test_pgw_paper_datasets(name):
    """The paper's dataset shapes (40,000 groups, windows of 100, batches of
    50K), 20 batches each."""
    sp = workloads.paper_dataset(name, tuples=20 * workloads.PAPER_BATCH)
    import torch
    q = cq.GroupWindows(sp.groups, sp.window, 1)
    o = oracle.WindowsOracle(sp.groups, sp.window, 1)
    st = sp.stream()
    try:
        for b in range(sp.batches):
            k, v = st.fill(b * sp.batch, sp.batch)
            expect = o.push(k, v)[1]
            out = torch.empty(sp.batch, dtype=torch.int64, device="cuda")
            assert q.push(_dev(k), _dev(v), out) == cq.CQ_OK
            assert np.array_equal(out.cpu().numpy(), expect), "batch %d" % b
    finally:
        q.close()


def test_pgw_bad_key_poisons_and_leaves_windows():
    import torch
    q = cq.GroupWindows(10, 4, 1)
    try:
        k = _dev(np.array([1, 2, 3], np.int32))
        out = torch.empty(3, dtype=torch.int64, device="cuda")
        assert q.push(k, k, out) == cq.CQ_OK
        assert q.sync() == cq.CQ_OK
        assert out.cpu().tolist() == [1, 2, 3]
        bad = _dev(np.array([1, 10], np.int32))
        q.push(bad, bad, torch.empty(2, dtype=torch.int64, device="cuda"))
        assert q.sync() in (cq.CQ_EKEY, cq.CQ_EPOISONED)
        assert q.push(k, k, out) == cq.CQ_EPOISONED
        with pytest.raises(cq.CQError):
            cq.GroupWindows(0, 4)
        with pytest.raises(cq.CQError):
            cq.GroupWindows(10, 0)
    finally:
        q.close()


def test_pgw_graph_replay_on_own_stream():
    """Pushes of one length on a non-default stream replay a captured graph;
    outputs stay exact, including pushes issued back to back."""
    import torch
    s = torch.cuda.Stream()
    G, w = 3_000, 50
    q = cq.GroupWindows(G, w, 2, stream=s)
    o = oracle.WindowsOracle(G, w, 2)
    st = streamgen.Stream(G, keys="zipf", s=1.1, vals="uniform", lo=-10**6, hi=10**6, seed=21)
    try:
        outs, expects, keep = [], [], []
        for b in range(12):
            n = 8_000 if b < 10 else 5_000
            k, v = st.fill(b * 8_000, n)
            expects.append(o.push(k, v)[1])
            with torch.cuda.stream(s):
                kd, vd = _dev(k), _dev(v)
                out = torch.empty(n, dtype=torch.int64, device="cuda")
            torch.cuda.synchronize()
            keep.append((kd, vd))
            assert q.push(kd, vd, out) == cq.CQ_OK
            outs.append(out)
        assert q.sync() == cq.CQ_OK
        for b, (got, exp) in enumerate(zip(outs, expects)):
            assert np.array_equal(got.cpu().numpy(), exp), "batch %d" % b
    finally:
        q.close()
