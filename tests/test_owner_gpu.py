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


# ---- lay-out and policy on the device (CQO_ON_DEVICE) ----

def _run_against_oracle(G, w, grid, policy, thr, batches, device=True, passes=1):
    """Push `batches` (key arrays) through the device-mode query and the
    oracle side by side: every output, the mapping after every push, the
    moves and the tpt extremes equal the oracle's."""
    T = 256 * grid
    q = cq.OwnerWindows(G, w, passes, grid=grid, policy=policy, threshold=thr, device=device)
    o = oracle.WindowsOracle(G, w, passes)
    m_ref = P.initial_mapping(G, T)
    rng = np.random.default_rng(G + grid)
    total = 0
    try:
        for b, k in enumerate(batches):
            k = np.asarray(k, np.int32)
            v = rng.integers(-2**31, 2**31 - 1, k.size, dtype=np.int64).astype(np.int32)
            status, expect = o.push(k, v)
            assert status == 0
            out = _out(k.size)
            assert q.push(k, v, out) == cq.CQ_OK
            assert q.sync() == cq.CQ_OK
            assert np.array_equal(out.cpu().numpy(), expect), "batch %d" % b
            if k.size:
                tpt = P.reorder(m_ref, k.tolist())[0]
                m_ref, moves = P.rebalance(policy, m_ref, k.tolist(), threshold=thr)
                assert q.mapping() == m_ref, "batch %d" % b
                s = q.stats()
                assert s["last_moves"] == moves, "batch %d" % b
                assert (s["last_max_tpt"], s["last_min_tpt"]) == (max(tpt), min(tpt))
                total += moves
        assert q.stats()["moves"] == total
    finally:
        q.close()
    return total


@pytest.mark.parametrize("policy", cq.CQO_DEVICE_POLICIES)
def test_device_policies_follow_the_oracle(policy):
    """The host-mode case above, lay-out and policy on the device."""
    st = streamgen.Stream(1000, keys="zipf", s=1.1, permute=False, vals="uniform", lo=0, hi=1, seed=5)
    batches, t = [], 0
    for n in [3000, 1, 4096, 0, 2500, 3333, 5000]:
        batches.append(st.fill(t, n)[0])
        t += n
    _run_against_oracle(1000, 40, 1, policy, 60, batches)


@pytest.mark.parametrize("policy", cq.CQO_DEVICE_POLICIES)
def test_device_policies_partial_tree_nodes(policy):
    """T = 1280: the arg-max / arg-min tree has 40 first-level nodes, the last
    of its second level half full; permuted Zipf keys move the heavy groups
    around, getFirst up to the G-move cap."""
    st = streamgen.Stream(3000, keys="zipf", s=1.1, permute=True, vals="uniform", lo=0, hi=1, seed=7)
    batches, t = [], 0
    for n in [6000, 5000, 7000]:
        batches.append(st.fill(t, n)[0])
        t += n
    moves = _run_against_oracle(3000, 16, 5, policy, 100, batches)
    assert policy == "none" or moves > 0


def test_device_get_first_full_tree():
    """T = 16384 (the paper's grid 64): 100 groups of 200 tuples on the first
    threads, over a uniform background; getFirst splits every doubly loaded
    thread and stops."""
    G = 20000
    rng = np.random.default_rng(11)
    hot = np.repeat(np.arange(100, dtype=np.int32), 200)
    batches = []
    for _ in range(3):
        k = np.concatenate([hot, rng.integers(0, G, 6000).astype(np.int32)])
        batches.append(k[rng.permutation(k.size)])
    assert _run_against_oracle(G, 8, 64, "getFirst", 300, batches) > 10


@pytest.mark.parametrize("policy", ["checkAll", "probCheck", "bestBalance"])
def test_device_scan_policies_full_tree(policy):
    """T = 16384 again: permuted Zipf batches around one where 100 groups of
    200 tuples load the first threads."""
    st = streamgen.Stream(20000, keys="zipf", s=1.3, permute=True, vals="uniform", lo=0, hi=1, seed=3)
    rng = np.random.default_rng(12)
    hot = np.concatenate([np.repeat(np.arange(100, dtype=np.int32), 200), rng.integers(0, 20000, 6000)])
    batches = [st.fill(0, 30000)[0], hot[rng.permutation(hot.size)].astype(np.int32), st.fill(30000, 30000)[0]]
    assert _run_against_oracle(20000, 8, 64, policy, 300, batches) > 10


@pytest.mark.parametrize("policy", ["none", "getFirst", "probCheck", "bestBalance"])
def test_device_paper_datasets_equal_host_mode(policy):
    """DS2 at grid 4, six batches of 50K: outputs equal the oracle's, and the
    device-mode mapping equals the host mode's after every batch."""
    sp = workloads.paper_dataset("DS2", tuples=6 * workloads.PAPER_BATCH)
    qd = cq.OwnerWindows(sp.groups, sp.window, 1, grid=4, policy=policy, device=True)
    qh = cq.OwnerWindows(sp.groups, sp.window, 1, grid=4, policy=policy)
    o = oracle.WindowsOracle(sp.groups, sp.window, 1)
    st = sp.stream()
    try:
        for b in range(sp.batches):
            k, v = st.fill(b * sp.batch, sp.batch)
            expect = o.push(k, v)[1]
            for q in (qd, qh):
                out = _out(sp.batch)
                assert q.push(k, v, out) == cq.CQ_OK
                assert q.sync() == cq.CQ_OK
                assert np.array_equal(out.cpu().numpy(), expect), "batch %d" % b
            assert qd.mapping() == qh.mapping(), "batch %d" % b
            assert qd.stats()["last_moves"] == qh.stats()["last_moves"]
    finally:
        qd.close()
        qh.close()


def test_device_mode_arguments():
    for policy in ("shift", "shiftLocal"):
        with pytest.raises(cq.CQError):
            cq.OwnerWindows(1000, 4, 1, grid=1, policy=policy, device=True)
    with pytest.raises(cq.CQError):
        cq.OwnerWindows(20000, 4, 1, grid=65, policy="getFirst", device=True)   # T = 16640 threads
    q = cq.OwnerWindows(300, 4, 1, grid=1, policy="probCheck", device=True)
    try:
        k = np.array([1, 2, 300], np.int32)
        assert q.push(k, k, _out(3)) == cq.CQ_EKEY
        assert q.push(k[:2], k[:2], _out(2)) == cq.CQ_EPOISONED
    finally:
        q.close()


@pytest.mark.parametrize("device", [False, True])
def test_owner_batches_that_grow_the_buffers(device):
    """Batches past the first staging and lay-out capacity (2^16 tuples) make
    the query drain its streams and reallocate between pushes."""
    G = 5000
    st = streamgen.Stream(G, keys="zipf", s=1.2, permute=True, vals="uniform", lo=-1000, hi=1000, seed=21)
    batches, t = [], 0
    for n in [1000, 100_000, 70_000, 300_000, 5]:
        batches.append(st.fill(t, n)[0])
        t += n
    _run_against_oracle(G, 12, 2, "probCheck", 500, batches, device=device)
