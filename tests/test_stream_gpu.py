"""Parity of cq_push_many (the persistent multi-batch launch) with the CPU
oracle, bit for bit, after EVERY batch: the launch writes each batch's full
result table to caller arrays, which are compared with the oracle's results
after the same batch.

Cases span whole-window replacement (the benchmark's configurations 1 and
2 at full size), retraction with front expiry and flips between launches,
ragged and empty batches, batches longer than the window, windows that are
not a multiple of four slots, unaligned batch pointers, aggregate subsets,
skew heavy enough for the heavy-hitter lists, calls mixed with cq_push, the
batch-by-batch fallback, bad keys, and a device wait that runs out.
"""
import numpy as np
import pytest

import oracle
import paper_1309_0634_b300 as cq
import streamgen
from streamgen import workloads
from gpu_util import assert_same

pytestmark = pytest.mark.gpu

INT32_MAX = 2**31 - 1
INT32_MIN = -(2**31)
FIELDS = ("sum", "count", "min", "max", "avg")


def _dev(x, offset=0):
    """A device copy of int32 array x whose data starts `offset` elements into
    its allocation (offset 1: not 16-byte aligned)."""
    import torch
    buf = torch.empty(len(x) + offset + 4, dtype=torch.int32, device="cuda")
    t = buf[offset:offset + len(x)]
    if len(x):
        t.copy_(torch.from_numpy(np.ascontiguousarray(x, np.int32)))
    return t


def _out(G, k):
    import torch
    d = dict(sum=torch.empty(k * G, dtype=torch.int64, device="cuda"),
             count=torch.empty(k * G, dtype=torch.int32, device="cuda"),
             min=torch.empty(k * G, dtype=torch.int32, device="cuda"),
             max=torch.empty(k * G, dtype=torch.int32, device="cuda"),
             avg=torch.empty(k * G, dtype=torch.float64, device="cuda"),
             stamps=torch.empty(2 * k, dtype=torch.int64, device="cuda"))
    return d


def _row(out, b, G):
    return {f: out[f][b * G:(b + 1) * G].cpu().numpy() for f in FIELDS}


def run_many(G, W, batches, calls, aggs=cq.CQ_ALL, options=None, offset=0, expect_path=4, q=None, o=None):
    """Push `batches` through cq_push_many in calls of the sizes in `calls`;
    compare the results after every batch with the oracle's."""
    import torch
    own = q is None
    if own:
        q = cq.Query(G, W, aggs, **(options or {}))
        o = oracle.Oracle(G, W)
    j = 0
    try:
        for size in calls:
            group = batches[j:j + size]
            kt = [_dev(k, offset) for k, _ in group]
            vt = [_dev(v, offset) for _, v in group]
            out = _out(G, size)
            st = q.push_many(kt, vt, out)
            assert st == cq.CQ_OK, (j, st)
            torch.cuda.synchronize()
            assert q.sync() == cq.CQ_OK
            for b, (k, v) in enumerate(group):
                assert o.push(k, v) == 0
                assert_same(_row(out, b, G), o.results(), aggs, where="batch %d (call of %d)" % (j + b, size))
            if expect_path is not None:
                assert q.stats()["last_path"] == expect_path
            stamps = out["stamps"].cpu().numpy().view(np.uint64)
            if expect_path == 4:
                begin, end = stamps[:size], stamps[size:]
                worked = np.array([len(k) > 0 for k, _ in group])
                assert np.all(begin[worked] > 0) and np.all(end[worked] >= begin[worked])
            j += size
        assert_same(q.results(), o.results(), aggs, where="after the last call")
        return q.stats()
    finally:
        if own:
            q.close()


def _stream_batches(stream, sizes):
    t, out = 0, []
    for b in sizes:
        out.append(stream.fill(t, b))
        t += b
    return out


@pytest.mark.parametrize("s", [0.0, 0.45, 1.5, 2.0])
def test_window_replacement_skewed(s):
    """B = W: every batch replaces the window; Zipf keys feed the heavy-hitter
    lists (s = 0.45 lists a few keys: the producers' short-list path)."""
    G, W = 20_000, 200_000
    st = streamgen.Stream(G, keys="zipf", s=s, vals="uniform", lo=-10**6, hi=10**6, seed=11)
    batches = _stream_batches(st, [W] * 12)
    q = cq.Query(G, W)
    o = oracle.Oracle(G, W)
    try:
        stats = run_many(G, W, batches, calls=[1, 7, 4], q=q, o=o)
        if s == 0.45:
            assert 1 <= len(q.hot_list()[0]) <= 4   # a list the producers compare key by key
    finally:
        q.close()
    assert stats["tuples_seen"] == 12 * W


def test_retraction_with_flips_between_launches():
    """B = W/2 with MIN/MAX: old tuples leave every batch, the front shrinks,
    and every second batch needs a flip, so each call is cut into launches."""
    G, W = 5_000, 40_000
    st = streamgen.Stream(G, keys="zipf", s=1.2, vals="normal", mean=0, sd=1e6, lo=-10**9, hi=10**9, seed=12)
    batches = _stream_batches(st, [W // 2] * 16)
    stats = run_many(G, W, batches, calls=[3, 9, 4])
    assert stats["flips"] >= 5


@pytest.mark.parametrize("G,W", [(3, 5), (37, 999), (3000, 9999), (12_000, 30_001)])
def test_ragged_empty_and_long_batches(G, W):
    """Random sizes 0 .. 2W (empty batches, batches longer than the window);
    windows that are not a multiple of four slots; extreme values."""
    rng = np.random.default_rng(G + 7 * W)
    sizes = [int(x) for x in rng.integers(0, 2 * W + 2, size=18)] + [0, W, 1, 3 * W, W - 1]
    batches = []
    for b in sizes:
        k = rng.integers(0, G, size=b).astype(np.int32)
        v = rng.integers(-1000, 1000, size=b).astype(np.int32)
        if b:
            v[rng.random(b) < 0.05] = INT32_MAX
            v[rng.random(b) < 0.05] = INT32_MIN
        batches.append((k, v))
    run_many(G, W, batches, calls=[5, 1, 10, 7])


def test_unaligned_batch_pointers():
    """Batches whose device pointers are 4 bytes past a 16-byte boundary take
    the per-element copies instead of bulk copies."""
    G, W = 4_000, 24_000
    st = streamgen.Stream(G, keys="uniform", vals="uniform", lo=0, hi=10**6, seed=13)
    batches = _stream_batches(st, [6_000, 7_001, 24_000, 3, 10_000, 30_000, 5_555])
    run_many(G, W, batches, calls=[7], offset=1)


@pytest.mark.parametrize("aggs", [cq.CQ_SUM | cq.CQ_COUNT, cq.CQ_MIN, cq.CQ_MAX | cq.CQ_AVG])
def test_aggregate_subsets(aggs):
    G, W = 2_000, 16_000
    st = streamgen.Stream(G, keys="zipf", s=1.0, vals="uniform", lo=-5000, hi=5000, seed=14)
    batches = _stream_batches(st, [5_000, 16_000, 4_000, 4_000, 12_000, 20_000])
    run_many(G, W, batches, calls=[2, 4], aggs=aggs)


def test_calls_mixed_with_single_pushes():
    """cq_push, then cq_push_many, then cq_push again: the launch takes over the
    stored extrema and heavy hitters and hands them back."""
    import torch
    G, W = 10_000, 60_000
    st = streamgen.Stream(G, keys="zipf", s=1.8, vals="uniform", lo=-10**6, hi=10**6, seed=15)
    sizes = [20_000, 30_000, 15_000, 60_000, 25_000, 25_000, 10_000, 40_000, 33_000]
    batches = _stream_batches(st, sizes)
    q = cq.Query(G, W)
    o = oracle.Oracle(G, W)
    try:
        for k, v in batches[:2]:
            assert q.push(torch.from_numpy(k).cuda(), torch.from_numpy(v).cuda()) == cq.CQ_OK
            o.push(k, v)
        assert_same(q.results(), o.results(), where="single pushes")
        run_many(G, W, batches[2:6], calls=[4], q=q, o=o)
        for k, v in batches[6:8]:
            assert q.push(torch.from_numpy(k).cuda(), torch.from_numpy(v).cuda()) == cq.CQ_OK
            o.push(k, v)
            assert_same(q.results(), o.results(), where="single push after the launch")
        run_many(G, W, batches[8:], calls=[1], q=q, o=o)
    finally:
        q.close()


def test_config1_full_in_one_call():
    """Configuration 1 (G = 1000, W = B = 10^4, 100 batches) in one call."""
    spec = workloads.config1()
    st = spec.stream()
    batches = _stream_batches(st, [spec.batch] * spec.batches)
    run_many(spec.groups, spec.window, batches, calls=[spec.batches])


@pytest.mark.parametrize("s", [0.0, 0.5, 1.5, 2.0])
def test_config2_full_size(s):
    """Configuration 2 at full size (G = 10^5, W = B = 10^6), as the benchmark
    launches it, every batch checked."""
    spec = workloads.config2(s)
    st = spec.stream()
    batches = _stream_batches(st, [spec.batch] * 8)
    run_many(spec.groups, spec.window, batches, calls=[3, 5])


@pytest.mark.parametrize("G,W", [(3000, 9999), (20_000, 100_000)])
def test_replacing_batches_after_a_retracting_one(G, W):
    """A retracting batch, then window-replacing batches, in one launch: the
    first replacing batch may only overwrite the ring once every producer
    has read the slots the retracting batch takes its old tuples from (with
    producers stealing chunks some run a batch ahead of others)."""
    rng = np.random.default_rng(G)
    sizes = [W, W // 3, W, W + 7, 2 * W, W // 2, W, W, W // 5, W]
    batches = [(rng.integers(0, G, size=b).astype(np.int32), rng.integers(-10**6, 10**6, size=b).astype(np.int32))
               for b in sizes]
    run_many(G, W, batches, calls=[len(sizes)])


@pytest.mark.parametrize("case", ["replace_s1.5", "retract_flips", "ragged", "config2_s1.5", "wide_keys"])
def test_two_producers_on_some_sms(case):
    """CQ_OPT_STREAM_PRODUCERS: on some SMs both CTAs cut batches, so there
    are more producers than consumers and each consumer owns a wider key
    range.  Every batch matches the oracle; a key space too wide for the
    fewer consumers falls back to one producer an SM (same results)."""
    if case == "replace_s1.5":
        G, W = 20_000, 200_000
        st = streamgen.Stream(G, keys="zipf", s=1.5, vals="uniform", lo=-10**6, hi=10**6, seed=21)
        batches, calls, pp = _stream_batches(st, [W] * 10), [4, 6], 40
    elif case == "retract_flips":
        G, W = 5_000, 40_000
        st = streamgen.Stream(G, keys="zipf", s=1.2, vals="normal", mean=0, sd=1e6, lo=-10**9, hi=10**9, seed=22)
        batches, calls, pp = _stream_batches(st, [W // 2] * 12), [5, 7], 74
    elif case == "ragged":
        G, W = 3000, 9999
        rng = np.random.default_rng(23)
        sizes = [int(x) for x in rng.integers(0, 2 * W + 2, size=12)] + [0, W, 1]
        batches = [(rng.integers(0, G, size=b).astype(np.int32), rng.integers(-1000, 1000, size=b).astype(np.int32))
                   for b in sizes]
        calls, pp = [6, 9], 4000
    elif case == "config2_s1.5":
        spec = workloads.config2(1.5)
        G, W = spec.groups, spec.window
        batches, calls, pp = _stream_batches(spec.stream(), [spec.batch] * 6), [2, 4], 48
    else:
        G, W = 140_000, 280_000
        st = streamgen.Stream(G, keys="uniform", vals="uniform", lo=0, hi=10**6, seed=24)
        batches, calls, pp = _stream_batches(st, [140_000] * 6), [6], 120
    run_many(G, W, batches, calls=calls, options={"stream_producers": pp})


def test_large_key_space_falls_back_batch_by_batch():
    """More groups than the consumers can keep: pushed with cq_push's kernels,
    same results, per-batch outputs still filled."""
    G, W = 600_000, 100_000
    st = streamgen.Stream(G, keys="uniform", vals="uniform", lo=0, hi=10**6, seed=16)
    batches = _stream_batches(st, [50_000, 100_000, 30_000])
    run_many(G, W, batches, calls=[3], expect_path=None)


def test_forced_path_falls_back():
    G, W = 1_000, 5_000
    st = streamgen.Stream(G, keys="uniform", vals="uniform", lo=0, hi=10**6, seed=17)
    batches = _stream_batches(st, [2_000, 5_000, 4_000])
    stats = run_many(G, W, batches, calls=[3], options={"path": 2}, expect_path=2)
    assert stats["last_path"] == 2


def test_bad_key_poisons_the_query():
    import torch
    G, W = 1_000, 8_000
    q = cq.Query(G, W)
    try:
        k = [np.arange(4_000, dtype=np.int32) % G for _ in range(3)]
        k[1][1234] = G + 5
        v = [np.ones(4_000, np.int32) for _ in range(3)]
        assert q.push_many([_dev(x) for x in k], [_dev(x) for x in v]) == cq.CQ_OK
        torch.cuda.synchronize()
        assert q.sync() == cq.CQ_EKEY
        assert q.sync() == cq.CQ_EPOISONED
    finally:
        q.close()


def test_wait_that_runs_out_poisons_only_its_query():
    """A producer that never reports a batch (test hook): the consumers' bounded
    waits run out after 2 ms, the launch ends, the query reports CQ_ETIMEOUT and
    then CQ_EPOISONED; another query is unaffected."""
    import torch
    G, W = 2_000, 8_000
    st = streamgen.Stream(G, keys="uniform", vals="uniform", lo=0, hi=10**6, seed=18)
    batches = _stream_batches(st, [4_000] * 5)
    bad = cq.Query(G, W, wait_limit_us=2_000, stall_batch=1)
    try:
        assert bad.get_option("wait_limit_us") == 2_000
        kt = [_dev(k) for k, _ in batches]
        vt = [_dev(v) for _, v in batches]
        assert bad.push_many(kt, vt) == cq.CQ_OK
        torch.cuda.synchronize()
        assert bad.sync() == cq.CQ_ETIMEOUT
        assert bad.sync() == cq.CQ_EPOISONED
        assert bad.push_many(kt, vt) == cq.CQ_EPOISONED
    finally:
        bad.close()
    run_many(G, W, batches, calls=[5])
