"""The paper's owner-computes execution (cqo_*): every policy gives every
tuple's window SUM bit for bit as the oracle does, and the thread-to-groups
mapping it leaves after each push is the oracle policy's (Section 4, one
batch later)."""
import numpy as np
import pytest

import oracle
from oracle import policies as P
import paper_1309_0634_b300 as cq
import streamgen
from streamgen import workloads

pytestmark = pytest.mark.gpu


def _out(n):
    import torch
    return torch.empty(n, dtype=torch.int64, device="cuda")


@pytest.mark.parametrize("policy", cq.CQO_POLICIES)
def test_owner_sums_and_mapping_follow_the_oracle(policy):
    G, w, passes, grid, thr = 1000, 40, 2, 1, 60
    T = 256 * grid
    q = cq.OwnerWindows(G, w, passes, grid=grid, policy=policy, threshold=thr)
    o = oracle.WindowsOracle(G, w, passes)
    m_ref = P.initial_mapping(G, T)
    st = streamgen.Stream(G, keys="zipf", s=1.1, permute=False, vals="uniform", lo=-2**31, hi=2**31 - 1, seed=5)
    t = 0
    try:
        for b, n in enumerate([3000, 1, 4096, 0, 2500, 3333, 5000]):
            k, v = st.fill(t, n)
            t += n
            status, expect = o.push(k, v)
            assert status == 0
            out = _out(n)
            assert q.push(k, v, out) == cq.CQ_OK
            assert q.sync() == cq.CQ_OK
            assert np.array_equal(out.cpu().numpy(), expect), "batch %d" % b
            if n:
                m_ref, moves = P.rebalance(policy, m_ref, k.tolist(), threshold=thr)
                assert q.mapping() == m_ref, "batch %d" % b
                assert q.stats()["last_moves"] == moves
        s = q.stats()
        assert s["tuples_seen"] == t and s["pushes"] == 6
    finally:
        q.close()


@pytest.mark.parametrize("name", ["DS1", "DS2", "DS3"])
@pytest.mark.parametrize("policy", ["none", "probCheck", "shiftLocal"])
def test_owner_paper_datasets(name, policy):
    """The paper's dataset shapes (40,000 groups, w = 100, batches of 50K)
    at grid size 4, eight batches each."""
    sp = workloads.paper_dataset(name, tuples=8 * workloads.PAPER_BATCH)
    q = cq.OwnerWindows(sp.groups, sp.window, 1, grid=4, policy=policy)
    o = oracle.WindowsOracle(sp.groups, sp.window, 1)
    st = sp.stream()
    try:
        for b in range(sp.batches):
            k, v = st.fill(b * sp.batch, sp.batch)
            expect = o.push(k, v)[1]
            out = _out(sp.batch)
            assert q.push(k, v, out) == cq.CQ_OK
            assert q.sync() == cq.CQ_OK
            assert np.array_equal(out.cpu().numpy(), expect), "batch %d" % b
    finally:
        q.close()


def test_owner_bad_key_and_arguments():
    q = cq.OwnerWindows(300, 4, 1, grid=1, policy="getFirst")
    try:
        k = np.array([1, 2, 300], np.int32)
        assert q.push(k, k, _out(3)) == cq.CQ_EKEY
        assert q.push(k[:2], k[:2], _out(2)) == cq.CQ_EPOISONED
        assert q.stats()["tuples_seen"] == 0
    finally:
        q.close()
    with pytest.raises(cq.CQError):
        cq.OwnerWindows(100, 4, 1, grid=1)                   # 256 threads for 100 groups
    with pytest.raises(cq.CQError):
        cq.OwnerWindows(1000, 4, 1, grid=1, pot=1.5)
