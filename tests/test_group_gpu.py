"""Many queries pushed together (one launch per round) match the oracle bit for bit."""
import numpy as np
import pytest

import oracle
import paper_1309_0634_b300 as cq
import streamgen
from streamgen import workloads
from gpu_util import assert_same

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()


class Member:
    def __init__(self, G, W, aggs=cq.CQ_ALL, seed=0, s=1.0, **opts):
        self.q = cq.Query(G, W, aggs, **opts)
        self.o = oracle.Oracle(G, W)
        self.st = streamgen.Stream(G, keys="zipf", s=s, vals="uniform", lo=-10**6, hi=10**6, seed=seed)
        self.t = 0
        self.aggs = aggs

    def next_batch(self, b):
        k, v = self.st.fill(self.t, b)
        self.t += b
        assert self.o.push(k, v) == 0
        return k, v

    def check(self, where=""):
        assert_same(self.q.results(), self.o.results(), self.aggs, where=where)

    def close(self):
        self.q.close()


def test_group_mixed_queries_several_rounds():
    rng = np.random.default_rng(3)
    members = [
        Member(1000, 10_000, seed=1, s=0.0),
        Member(1, 7, seed=2),
        Member(777, 3_333, seed=3, s=1.5),               # window not a multiple of 4: unaligned ring
        Member(50_000, 200_000, seed=4, s=2.0),
        Member(3, 1, seed=5),
        Member(20_000, 65_536, cq.CQ_SUM | cq.CQ_COUNT, seed=6, s=1.2),
        Member(5_000, 40_000, cq.CQ_MIN | cq.CQ_MAX, seed=7, s=0.7),
        Member(1_000, 999, cq.CQ_AVG, seed=8, s=1.0),
    ]
    g = cq.Group()
    try:
        for rnd in range(10):
            batches = []
            for m in members:
                b = int(rng.integers(0, 2 * m.q.window + 3)) if rnd % 3 else m.q.window // 5 + 1
                batches.append(m.next_batch(b))
            st = [0] * len(members)
            assert g.push([m.q for m in members], [_dev(k) for k, _ in batches], [_dev(v) for _, v in batches], st) == 0
            assert st == [0] * len(members)
            for i, m in enumerate(members):
                m.check("round %d query %d" % (rnd, i))
        for m in members:
            assert m.q.stats()["last_path"] in (2, 3)
    finally:
        for m in members:
            m.close()
        g.close()


def test_group_interleaves_with_single_pushes_and_skips_poisoned():
    a = Member(2000, 20_000, seed=11, s=1.0)
    b = Member(300, 5_000, seed=12, s=2.0)
    bad = cq.Query(10, 100)
    g = cq.Group()
    try:
        for rnd in range(6):
            ka, va = a.next_batch(7_000)
            kb, vb = b.next_batch(1_234)
            if rnd % 2:
                assert a.q.push(_dev(ka), _dev(va)) == 0
                assert g.push([b.q], [_dev(kb)], [_dev(vb)]) == 0
            else:
                st = [0, 0, 0]
                kbad = _dev(np.array([1, 2, 55], np.int32)) if rnd == 0 else _dev(np.array([1], np.int32))
                assert g.push([a.q, b.q, bad], [_dev(ka), _dev(kb), kbad],
                              [_dev(va), _dev(vb), _dev(np.zeros(kbad.numel(), np.int32))], st) == 0
                assert st[0] == 0 and st[1] == 0
                if rnd > 0:
                    assert st[2] in (cq.CQ_EKEY, cq.CQ_EPOISONED)
            a.check("a round %d" % rnd)
            b.check("b round %d" % rnd)
        assert bad.sync() in (cq.CQ_EKEY, cq.CQ_EPOISONED)
    finally:
        a.close()
        b.close()
        bad.close()
        g.close()


def test_group_member_beyond_group_kernel_range():
    big = Member(2**21 + 5, 10_000, seed=21, s=1.0)   # more partitions than the group kernel takes
    small = Member(100, 1000, seed=22)
    g = cq.Group()
    try:
        for rnd in range(3):
            k1, v1 = big.next_batch(6_000)
            k2, v2 = small.next_batch(700)
            assert g.push([big.q, small.q], [_dev(k1), _dev(k2)], [_dev(v1), _dev(v2)]) == 0
            big.check()
            small.check()
        assert small.q.stats()["last_path"] == 3
        assert big.q.stats()["last_path"] in (1, 2)
    finally:
        big.close()
        small.close()
        g.close()


def test_group_rejects_bad_arguments():
    q = cq.Query(10, 10)
    g = cq.Group()
    k = _dev(np.zeros(4, np.int32))
    try:
        assert g.push([q, q], [k, k], [k, k]) == cq.CQ_EINVAL
        st, h = cq.cqg_create(0)
        assert st == 0
        assert cq.cqg_push(h, [q], [k], [k], [-1], None) == cq.CQ_OK   # refused per query
        s = [0]
        cq.cqg_push(h, [q], [k], [k], [-1], s)
        assert s[0] == cq.CQ_EINVAL
        cq.cqg_destroy(h)
    finally:
        q.close()
        g.close()


def test_batched_config_64_queries_full_size():
    """The batched configuration: 64 standing queries, one launch per round;
    every query checked against the oracle after every round."""
    specs = workloads.config4()
    members = []
    g = cq.Group()
    try:
        for sp in specs:
            m = Member(sp.groups, sp.window, seed=sp.stream_kw["seed"], s=sp.stream_kw["s"])
            m.batch = sp.batch
            members.append(m)
        for rnd in range(3):
            batches = [m.next_batch(m.batch) for m in members]
            assert g.push([m.q for m in members], [_dev(k) for k, _ in batches], [_dev(v) for _, v in batches]) == 0
            for i, m in enumerate(members):
                m.check("round %d query %d" % (rnd, i))
    finally:
        for m in members:
            m.close()
        g.close()


def test_group_graph_replay_on_own_stream():
    """Repeated launch shapes replay a captured CUDA graph; results stay exact."""
    import torch
    s = torch.cuda.Stream()
    members = [Member(1000, 8_000, seed=31, s=1.5), Member(300, 3_000, seed=32, s=0.0),
               Member(40_000, 100_000, seed=33, s=1.0)]
    g = cq.Group(s)
    try:
        for rnd in range(12):
            batches = [m.next_batch(b) for m, b in zip(members, (1_000, 600, 25_000))]
            with torch.cuda.stream(s):
                kd = [_dev(k) for k, _ in batches]
                vd = [_dev(v) for _, v in batches]
            assert g.push([m.q for m in members], kd, vd) == 0
            assert g.sync() == 0
            for i, m in enumerate(members):
                m.check("round %d query %d" % (rnd, i))
        st = g.stats()
        assert st["launches"] == 12
        assert st["graph_launches"] > 0
    finally:
        for m in members:
            m.close()
        g.close()


def test_group_back_to_back_without_sync():
    """Two descriptor slots: consecutive pushes overlap host preparation with the previous launch."""
    members = [Member(2_000, 20_000, seed=41, s=1.2), Member(100, 1_000, seed=42, s=2.0)]
    g = cq.Group()
    try:
        keep = []
        for rnd in range(20):
            batches = [m.next_batch(b) for m, b in zip(members, (5_000, 333))]
            kd = [_dev(k) for k, _ in batches]
            vd = [_dev(v) for _, v in batches]
            keep.append((kd, vd))
            assert g.push([m.q for m in members], kd, vd) == 0
        assert g.sync() == 0
        for i, m in enumerate(members):
            m.check("query %d" % i)
    finally:
        for m in members:
            m.close()
        g.close()


def test_group_members_replacing_their_windows():
    """Members whose batches replace their whole windows beside members that
    slide, in the same launches."""
    members = [Member(2_000, 5_000, seed=51, s=1.5), Member(3_000, 40_000, seed=52, s=0.5),
               Member(500, 500, seed=53, s=2.0), Member(10_000, 8_192, cq.CQ_SUM | cq.CQ_COUNT | cq.CQ_AVG, seed=54)]
    g = cq.Group()
    try:
        for rnd in range(6):
            sizes = (5_000 if rnd % 2 else 7_000, 4_000, 500 + rnd, 8_192)
            batches = [m.next_batch(b) for m, b in zip(members, sizes)]
            assert g.push([m.q for m in members], [_dev(k) for k, _ in batches], [_dev(v) for _, v in batches]) == 0
            for i, m in enumerate(members):
                m.check("round %d query %d" % (rnd, i))
    finally:
        for m in members:
            m.close()
        g.close()


def test_group_members_flip_side_by_side():
    """Six MIN/MAX members whose windows are twice their batches flip every
    other round, several in the same round (their flips run on the group's
    side streams before the launch); two of them share a stream of their
    own.  Every member matches the oracle after every round."""
    import torch
    own = torch.cuda.Stream()
    members = [Member(G, 2 * B, seed=40 + i, s=1.3, stream=own if i < 2 else None)
               for i, (G, B) in enumerate([(300, 4000), (5000, 20_000), (64, 1000), (20_000, 50_000),
                                            (1000, 3000), (7, 500)])]
    g = cq.Group()
    try:
        for rnd in range(7):
            batches = [m.next_batch(m.q.window // 2) for m in members]
            st = [0] * len(members)
            assert g.push([m.q for m in members], [_dev(k) for k, _ in batches], [_dev(v) for _, v in batches], st) == 0
            assert st == [0] * len(members)
            for i, m in enumerate(members):
                m.check("round %d member %d" % (rnd, i))
        assert all(m.q.stats()["flips"] >= 2 for m in members)
    finally:
        for m in members:
            m.close()
        g.close()


def test_autotuned_members_stay_in_the_group_launch():
    """Members pinned to the group kernel's path (CQ_OPT_PATH = 1) and tuned by
    cq_autotune keep that path, get their own partition width / heavy-hitter
    settings, and still match the oracle after every round of group pushes."""
    members = [Member(1000, 10_000, seed=21, s=0.0), Member(30_000, 150_000, seed=22, s=1.5),
               Member(200_000, 1_000_000, seed=23, s=1.0), Member(100, 2_000, seed=24, s=2.0)]
    g = cq.Group()
    try:
        for m in members:
            m.q.set_option("path", 1)
            k, v = m.st.fill(10**9, m.q.window // 10 + 1)          # a sample batch from far ahead in the stream
            st, us = cq.cq_autotune(m.q.handle, _dev(k), _dev(v), len(k), 2)
            assert st == cq.CQ_OK and us > 0
            assert m.q.get_option("path") == 1                     # the pinned path is kept
        for rnd in range(8):
            batches = [m.next_batch(m.q.window // 10 + 1) for m in members]
            st = [0] * len(members)
            assert g.push([m.q for m in members], [_dev(k) for k, _ in batches], [_dev(v) for _, v in batches],
                          st) == 0
            assert st == [0] * len(members)
            for i, m in enumerate(members):
                m.check("round %d member %d" % (rnd, i))
                assert m.q.stats()["last_path"] == 3               # pushed by the group kernel
    finally:
        g.close()
        for m in members:
            m.close()
