"""Parity of the CUDA path with the CPU oracle, bit for bit, after every push.

Small cases span several ring wraps, ragged batches, empty batches, batches
longer than the window and every front/back flip case of the MIN/MAX
structure; the full-size cases run the benchmark configurations with the
launch configuration the benchmark uses.
"""
import numpy as np
import pytest

import oracle
import paper_1309_0634_b300 as cq
import streamgen
from streamgen import workloads
from gpu_util import assert_same, run_pair

pytestmark = pytest.mark.gpu

INT32_MAX = 2**31 - 1
INT32_MIN = -(2**31)


def batches_from(stream, sizes):
    t = 0
    for b in sizes:
        yield stream.fill(t, b)
        t += b


def test_hand_worked_example_on_gpu():
    G, W = 3, 4
    pushes = [
        ([0, 1, 0], [1, 5, -2]),
        ([2, 1], [7, -3]),
        ([], []),
        ([0, 0, 2, 1, 2, 0], [10, 20, -5, 0, 3, 4]),
        ([1, 1], [INT32_MAX, INT32_MAX]),
        ([0], [INT32_MIN]),
        ([1], [1]),
    ]
    batches = [(np.array(k, np.int32), np.array(v, np.int32)) for k, v in pushes]
    run_pair(G, W, batches)


@pytest.mark.parametrize("G,W", [(1, 1), (1, 7), (3, 5), (8, 64), (37, 1000), (1000, 4097), (5000, 30_000)])
def test_random_ragged_batches(G, W):
    rng = np.random.default_rng(G * 131 + W)
    sizes = [int(x) for x in rng.integers(0, 2 * W + 2, size=14)] + [0, W, 1, W - 1 if W > 1 else 1, 3 * W]
    batches = []
    for b in sizes:
        k = rng.integers(0, G, size=b, dtype=np.int64).astype(np.int32)
        v = rng.integers(-1000, 1000, size=b).astype(np.int32)
        if b:
            v[rng.random(b) < 0.05] = INT32_MAX
            v[rng.random(b) < 0.05] = INT32_MIN
        batches.append((k, v))
    stats = run_pair(G, W, batches)
    assert stats["tuples_seen"] == sum(sizes)


@pytest.mark.parametrize("s", [0.0, 1.0, 2.0])
@pytest.mark.parametrize("W,B", [(50_000, 7_919), (65_536, 16_384), (100_000, 100_000), (20_000, 33_333)])
def test_zipf_small_batches_flip(s, W, B):
    """B < W exercises flips (front exhausted while old tuples remain)."""
    st = streamgen.Stream(2000, keys="zipf", s=s, vals="uniform", lo=-10**6, hi=10**6, seed=17)
    stats = run_pair(2000, W, batches_from(st, [B] * 25))
    if B < W:
        assert stats["flips"] > 0


@pytest.mark.parametrize("G", [2, 2049, 5_000_000])
def test_flip_digit_plans(G):
    """Flips whose radix sort takes one 1-bit pass (G = 2), two 6-bit passes
    (G = 2049) and three passes of 8, 8 and 7 bits (G = 5 * 10^6), with
    segments that end in ragged tiles."""
    W = 150_001
    st = streamgen.Stream(G, keys="zipf", s=0.8, vals="uniform", lo=-10**6, hi=10**6, seed=G % 97)
    stats = run_pair(G, W, batches_from(st, [40_000, 60_000, 50_001, 70_000, 45_000, 99_999, 30_000]),
                     check_every=2)
    assert stats["flips"] >= 2


@pytest.mark.parametrize("G,s", [(4096, 2.0), (70_000, 1.3)])
def test_flip_heavy_key_over_many_tiles(G, s):
    """Two-pass flips whose heaviest key spans tens of 4096-item tiles of the
    sort and of the segmented scan: its suffix extrema cross tiles by look-back."""
    W = 300_007
    st = streamgen.Stream(G, keys="zipf", s=s, vals="normal", mean=0, sd=1e6, lo=-10**9, hi=10**9, seed=G)
    stats = run_pair(G, W, batches_from(st, [100_000, 200_007, 150_000, 150_000, 123_457, 176_550, 299_999]),
                     check_every=1)
    assert stats["flips"] >= 3


@pytest.mark.parametrize("aggs", [cq.CQ_SUM, cq.CQ_COUNT, cq.CQ_MIN, cq.CQ_MAX, cq.CQ_AVG,
                                  cq.CQ_MIN | cq.CQ_MAX, cq.CQ_SUM | cq.CQ_AVG])
def test_aggregate_subsets(aggs):
    st = streamgen.Stream(300, keys="zipf", s=1.0, vals="uniform", lo=-500, hi=500, seed=5)
    run_pair(300, 5000, batches_from(st, [1234, 4000, 777, 6000, 10, 2500] * 3), aggs=aggs)


@pytest.mark.parametrize("opts", [
    dict(path=2), dict(path=2, warp_agg=0), dict(path=1), dict(path=3), dict(path=3, hot_keys=0),
    dict(path=1, hot_keys=0), dict(path=3, hot_keys=128, hot_threshold=1),
    dict(path=1, hot_keys=128, hot_threshold=1), dict(path=1, hot_keys=8, hot_threshold=50),
    dict(path=1, partition_bits=1), dict(path=1, partition_bits=11), dict(path=1, ctas_per_sm=1),
])
def test_options_do_not_change_results(opts):
    """Skew handling and launch shape change only where work runs, never a result."""
    st = streamgen.Stream(2000, keys="zipf", s=1.5, vals="uniform", lo=-10**6, hi=10**6, seed=31)
    sizes = [20_000] * 6 + [60_000] * 3 + [70_000, 5, 0, 33_333, 59_999, 1]
    stats = run_pair(2000, 60_000, batches_from(st, sizes), options=opts)
    want = {2: (2,), 3: (1,)}.get(opts.get("path"), (1, 3))
    assert stats["last_path"] in want


def test_hot_key_cap_change_between_pushes():
    import torch
    st = streamgen.Stream(3000, keys="zipf", s=2.0, vals="uniform", seed=41)
    q = cq.Query(3000, 50_000, hot_keys=8, hot_threshold=10)
    o = oracle.Oracle(3000, 50_000)
    t = 0
    for cap in [8, 128, 0, 64, 128]:
        q.set_option("hot_keys", cap)
        for _ in range(2):
            k, v = st.fill(t, 17_000)
            t += 17_000
            assert q.push(torch.from_numpy(k).cuda(), torch.from_numpy(v).cuda()) == cq.CQ_OK
            assert o.push(k, v) == 0
            assert_same(q.results(), o.results())
    q.close()


@pytest.mark.parametrize("warp_agg", [0, 1])
def test_warp_aggregation_does_not_change_results(warp_agg):
    st = streamgen.Stream(100, keys="zipf", s=2.0, vals="uniform", lo=-10**6, hi=10**6, seed=8)
    run_pair(100, 40_000, batches_from(st, [9_000] * 12), options=dict(warp_agg=warp_agg, path=2))


def test_host_push_matches_device_push():
    st = streamgen.Stream(500, keys="zipf", s=1.5, vals="uniform", seed=12)
    run_pair(500, 12_345, batches_from(st, [5000, 20_000, 0, 12_345, 100]), host=True)


def test_pipelined_host_pushes_and_async_result_reads():
    """Host batches from pinned memory pushed back to back, each followed by an
    asynchronous read of all results into its own pinned arrays, with one
    sync at the end: the copy stream runs ahead of the pushes, yet every
    step's results equal the oracle's after that step.  Batch sizes grow (the
    staging slots are reallocated) and one batch is longer than the window."""
    import torch
    G, W = 700, 9_000
    st = streamgen.Stream(G, keys="zipf", s=1.3, permute=True, vals="uniform", lo=-10**6, hi=10**6, seed=31)
    sizes = [100, 3000, 3000, 8000, 20_000, 50, 9_000, 4000]
    q = cq.Query(G, W, cq.CQ_ALL)
    o = oracle.Oracle(G, W)
    expect, outs, keep = [], [], []
    try:
        t = 0
        for n in sizes:
            k, v = st.fill(t, n)
            t += n
            kh = torch.from_numpy(k).pin_memory()
            vh = torch.from_numpy(v).pin_memory()
            keep.append((kh, vh))   # unchanged until the final sync
            res = [torch.empty(G, dtype=dt, pin_memory=True)
                   for dt in (torch.int64, torch.int32, torch.int32, torch.int32, torch.float64)]
            assert cq.cq_push_host(q.handle, kh, vh, n) == cq.CQ_OK
            assert cq.cq_results_copy_async(q.handle, *res) == cq.CQ_OK
            outs.append(res)
            assert o.push(k, v) == 0
            expect.append(o.results())
        assert q.sync() == cq.CQ_OK
        for i, (res, ref) in enumerate(zip(outs, expect)):
            got = {f: r.numpy() for f, r in zip(("sum", "count", "min", "max", "avg"), res)}
            assert_same(got, ref, where="step %d" % i)
    finally:
        q.close()


def test_round_robin_closed_form_counts():
    G, W = 40, 4000
    st = streamgen.Stream(G, keys="round_robin", vals="index", lo=-7, hi=10**9, seed=0)
    q = cq.Query(G, W)
    import torch
    t = 0
    for b in [1000, 3000, 4000, 2500, 9000]:
        k, v = st.fill(t, b)
        assert q.push(torch.from_numpy(k).cuda(), torch.from_numpy(v).cuda()) == cq.CQ_OK
        t += b
        r = q.results()
        if t >= W:
            assert (r["count"] == W // G).all()
        L = max(0, t - W)
        for g in (0, 1, G - 1):
            first = L + ((g - L) % G)
            last = (t - 1) - ((t - 1 - g) % G)
            assert r["min"][g] == -7 + first and r["max"][g] == -7 + last
    q.close()


def test_bad_key_poisons_without_fault():
    import torch
    q = cq.Query(10, 100)
    k = torch.tensor([1, 2, 10, 3], dtype=torch.int32, device="cuda")
    v = torch.tensor([1, 2, 3, 4], dtype=torch.int32, device="cuda")
    st = q.push(k, v)
    assert st in (cq.CQ_OK, cq.CQ_EKEY)
    st2 = q.sync()
    codes = {st, st2}
    assert cq.CQ_EKEY in codes
    assert q.push(k, v) == cq.CQ_EPOISONED
    with pytest.raises(cq.CQError):
        q.results()
    q.close()
    # a negative key is caught the same way, and other queries stay usable
    q = cq.Query(10, 100)
    q.push(torch.tensor([-1], dtype=torch.int32, device="cuda"), torch.tensor([0], dtype=torch.int32, device="cuda"))
    assert q.sync() == cq.CQ_EKEY
    q.close()
    run_pair(10, 100, [(np.arange(10, dtype=np.int32), np.arange(10, dtype=np.int32))])


def test_argument_errors():
    import torch
    q = cq.Query(10, 100)
    k = torch.zeros(4, dtype=torch.int32, device="cuda")
    assert cq.cq_push(q.handle, None, None, 4) == cq.CQ_EINVAL
    assert cq.cq_push(q.handle, k, k, -1) == cq.CQ_EINVAL
    assert cq.cq_push(q.handle, None, None, 0) == cq.CQ_OK
    for bad in [(0, 10), (10, 0), (2**31, 5), (5, 2**31)]:
        st, h = cq.cq_create(bad[0], bad[1], cq.CQ_ALL, 0)
        assert st == cq.CQ_EINVAL
    st, h = cq.cq_create(10, 10, 0, 0)
    assert st == cq.CQ_EINVAL
    st, h = cq.cq_create(10, 10, 64, 0)
    assert st == cq.CQ_EINVAL
    assert cq.cq_set_option(q.handle, cq.CQ_OPT_PARTITION_BITS, 12) == cq.CQ_EINVAL
    q.close()


# ---- full-size configurations, launch configuration of the benchmark ---------

def test_config1_uniform_full():
    spec = workloads.config1()
    st = spec.stream()
    run_pair(spec.groups, spec.window, batches_from(st, [spec.batch] * spec.batches))


@pytest.mark.parametrize("s", workloads.ZIPF_SWEEP)
def test_config2_skew_sweep_full_size(s):
    spec = workloads.config2(s)
    st = spec.stream()
    run_pair(spec.groups, spec.window, batches_from(st, [spec.batch] * 6))


def test_config3_drifting_skew_full_size():
    spec = workloads.config3()
    st = spec.stream()
    # 24 batches: 12 flips and one re-draw of the heavy hitters at batch 20
    stats = run_pair(spec.groups, spec.window, batches_from(st, [spec.batch] * 24), check_every=1)
    assert stats["flips"] >= 10


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()


def test_autotune_keeps_state_and_results():
    G, W = 20_000, 200_000
    q = cq.Query(G, W)
    o = oracle.Oracle(G, W)
    st = streamgen.Stream(G, keys="zipf", s=1.5, vals="uniform", lo=-1000, hi=1000, seed=77)
    t = 0
    try:
        for i in range(8):
            k, v = st.fill(t, 50_000)
            t += 50_000
            assert o.push(k, v) == 0
            assert q.push(_dev(k), _dev(v)) == 0
            if i == 3:
                before = q.stats()["tuples_seen"]
                us = q.autotune(_dev(k), _dev(v), trials=2)
                assert us > 0
                assert q.get_option("ctas_per_sm") in (1, 8)   # one of the tuner's two CTA settings
                assert q.stats()["tuples_seen"] == before
                assert_same(q.results(), o.results(), cq.CQ_ALL, where="after autotune")
        assert_same(q.results(), o.results(), cq.CQ_ALL, where="end")
    finally:
        q.close()


def _batches(G, sizes, s=1.5, seed=0, lo=-10**6, hi=10**6):
    st = streamgen.Stream(G, keys="zipf", s=s, vals="uniform", lo=lo, hi=hi, seed=seed)
    t, out = 0, []
    for n in sizes:
        out.append(st.fill(t, n))
        t += n
    return out


@pytest.mark.parametrize("aggs", [cq.CQ_ALL, cq.CQ_SUM | cq.CQ_COUNT, cq.CQ_AVG, cq.CQ_MIN | cq.CQ_MAX, cq.CQ_COUNT])
def test_whole_window_replacement_after_partial_window(aggs):
    """A push of n >= W into a window that is not yet full, then pushes that
    replace full windows, with groups that disappear between pushes."""
    G, W = 3_000, 20_000
    stats = run_pair(G, W, _batches(G, [7_000, 20_000, 25_000, 20_000, 3_000, 20_000, 40_000], seed=aggs), aggs)
    assert stats["resets"] >= 0


@pytest.mark.parametrize("opts", [{}, {"path": 1}, {"path": 3}, {"path": 2}, {"hot_keys": 0}, {"hot_keys": 128, "hot_threshold": 1}])
def test_whole_window_replacement_paths_and_skew(opts):
    """Replacing pushes (B = W) under heavy skew on every push path; groups
    of the previous window that get no tuple must come out empty."""
    G, W = 50_000, 100_000
    run_pair(G, W, _batches(G, [W] * 5, s=2.0, seed=7), cq.CQ_ALL, options=opts)
    run_pair(G, W, _batches(G, [W + 13, W, 2 * W + 1, W - 1, W], s=0.3, seed=8), cq.CQ_ALL, options=opts)


def test_whole_window_replacement_unaligned_and_tiny():
    run_pair(7, 3, _batches(7, [2, 3, 5, 1, 3, 3, 4], seed=9))          # W = 3: replacements of a tiny window
    run_pair(1_000, 10_001, _batches(1_000, [10_001, 10_001, 30_000, 5, 10_001], seed=10))   # W not a multiple of 4


@pytest.mark.parametrize("s,thr", [(1.0, 800), (1.5, 500), (2.0, 300), (0.0, 64)])
def test_heavy_hitter_detection_is_exact(s, thr):
    """The heavy hitters a push detects are exactly the groups whose insert
    count reached the threshold (capped at the heavy-hitter limit), checked
    against an exact host histogram of the pushed keys."""
    G, W, B = 100_000, 1_000_000, 1_000_000
    st = streamgen.Stream(G, keys="zipf", s=s, permute=True, vals="uniform", lo=0, hi=10**6, seed=31)
    q = cq.Query(G, W, cq.CQ_ALL, hot_threshold=thr, hot_keys=64)
    try:
        for i in range(3):
            k, v = st.fill(i * B, B)
            assert q.push(_dev(k), _dev(v)) == cq.CQ_OK
            expect = int((np.bincount(k, minlength=G) >= thr).sum())
            assert q.stats()["hot_keys"] == min(64, expect), i
    finally:
        q.close()


@pytest.mark.parametrize("path", [1, 3])
def test_heavy_hitters_sure_of_a_slot(path):
    """With a cap of 4 and a threshold of 1 every key of a push qualifies,
    thousands of them; the two keys holding 30 % of a push each (more than
    n/4) must still be listed, ahead of the others, with their exact counts."""
    import torch
    G, W, n = 5000, 100_000, 40_000
    rng = np.random.default_rng(3)
    q = cq.Query(G, W, cq.CQ_ALL, hot_keys=4, hot_threshold=1, path=path)
    o = oracle.Oracle(G, W)
    try:
        for i in range(4):
            u = rng.random(n)
            k = rng.integers(0, G, n).astype(np.int32)
            k[u < 0.3] = 11
            k[(u >= 0.3) & (u < 0.6)] = 4242
            v = rng.integers(-1000, 1000, n).astype(np.int32)
            assert q.push(torch.from_numpy(k).cuda(), torch.from_numpy(v).cuda()) == cq.CQ_OK
            assert o.push(k, v) == 0
            keys, counts = q.hot_list()
            c = np.bincount(k, minlength=G)
            assert len(keys) == 4 and len(set(keys)) == 4, keys
            assert set(keys[:2]) == {11, 4242}, keys
            assert counts == [int(c[x]) for x in keys]
            assert_same(q.results(), o.results(), where="push %d" % i)
    finally:
        q.close()


@pytest.mark.parametrize("path", [0, 3])
def test_keys_heavy_within_a_push(path):
    """Keys that turn heavy inside a push (not on the previous push's list)
    are folded out of their overloaded runs and merged back exactly: eight
    keys take 9 % of a batch each with no warning, later eight others, and
    the first eight then leave the window (heavy retractions of keys no
    longer listed).  Every push matches the oracle, and the list the next
    push privatises carries the first eight with their exact insert counts,
    so the folded inserts were counted."""
    import torch
    G, W, n = 100_000, 1_500_000, 600_000
    rng = np.random.default_rng(11)
    heavy_a = rng.choice(G, 8, replace=False)
    heavy_b = rng.choice(np.setdiff1d(np.arange(G), heavy_a), 8, replace=False)
    q = cq.Query(G, W, cq.CQ_ALL, path=path)
    o = oracle.Oracle(G, W)

    def batch(heavy):
        k = rng.integers(0, G, n).astype(np.int32)
        if heavy is not None:
            u = rng.random(n)
            for j, key in enumerate(heavy):
                k[(u >= 0.09 * j) & (u < 0.09 * (j + 1))] = key
        v = rng.integers(-10**6, 10**6, n).astype(np.int32)
        return k, v

    try:
        folds = [0]
        for i, heavy in enumerate([None, heavy_a, None, heavy_b, None, None]):
            k, v = batch(heavy)
            assert q.push(torch.from_numpy(k).cuda(), torch.from_numpy(v).cuda()) == cq.CQ_OK
            assert o.push(k, v) == 0
            assert_same(q.results(), o.results(), where="push %d" % i)
            folds.append(q.stats()["heavy_folds"])
            if i == 1:
                keys, counts = q.hot_list()
                c = np.bincount(k, minlength=G)
                listed = dict(zip(keys, counts))
                for key in heavy_a:
                    assert listed.get(int(key)) == int(c[key]), (int(key), listed.get(int(key)), int(c[key]))
        d = np.diff(folds)
        # the new heavy keys were folded in pushes 1 and 3, and heavy_a's tuples
        # left the window (pushes 3-5) after heavy_b had taken the list
        assert d[0] == 0 and d[1] > 0 and d[2] == 0 and d[3] > 0 and d[4] + d[5] > 0, d
    finally:
        q.close()


@pytest.mark.parametrize("s", [1.0, 1.5, 2.0])
def test_steady_skew_folds_nothing(s):
    """In a steady skewed stream (10^5 groups, W = B = 10^6) the keys found
    heavy within the first push are on the list from the second push on, so
    later pushes fold nothing."""
    import torch
    spec = workloads.config2(s)
    st = spec.stream()
    q = cq.Query(spec.groups, spec.window, cq.CQ_ALL)
    try:
        folds = []
        for i in range(5):
            k, v = st.fill(i * spec.batch, spec.batch)
            assert q.push(torch.from_numpy(k).cuda(), torch.from_numpy(v).cuda()) == cq.CQ_OK
            folds.append(q.stats()["heavy_folds"])
        assert folds[0] > 0, folds            # the first push meets the skew unwarned
        assert folds[-1] == folds[1], folds    # and from the second push on the list covers it
    finally:
        q.close()
