"""Pins of the per-group-window oracle (the paper's own aggregate, Sections
3.2 and 5.1: a window of the last w values per group, its SUM recomputed
after every tuple), each independent of the oracle's code."""
import numpy as np
import pytest

import oracle

I32_MAX, I32_MIN = 2**31 - 1, -2**31


def brute_force(G, w, keys, vals):
    """Window sum after each tuple from the full stream history: the last
    min(count, w) values of the tuple's group, found by scanning backwards."""
    out = []
    for i in range(len(keys)):
        k = keys[i]
        s, taken = 0, 0
        for j in range(i, -1, -1):
            if keys[j] == k:
                s += int(vals[j])
                taken += 1
                if taken == w:
                    break
        out.append(s)
    return out


@pytest.mark.parametrize("G,w,passes", [(1, 1, 1), (1, 3, 2), (2, 2, 1), (5, 7, 10), (3, 100, 1), (8, 4, 3)])
def test_brute_force_full_history(G, w, passes):
    rng = np.random.default_rng(G * 1000 + w)
    o = oracle.WindowsOracle(G, w, passes)
    keys_all, vals_all = [], []
    for b in range(12):
        n = int(rng.integers(0, 3 * w + 4))
        keys = rng.integers(0, G, n).astype(np.int32)
        extreme = rng.choice(np.array([I32_MAX, I32_MIN, 0, -1, 1], np.int64), n)
        uniform = rng.integers(I32_MIN, I32_MAX, n, endpoint=True)
        vals = np.where(rng.random(n) < 0.5, extreme, uniform).astype(np.int32)
        st, out = o.push(keys, vals)
        assert st == 0
        keys_all += keys.tolist()
        vals_all += vals.tolist()
        expect = brute_force(G, w, keys_all, vals_all)[len(keys_all) - n:]
        assert out.tolist() == expect
    assert o.seen == len(keys_all)


def test_round_robin_closed_form():
    """Round-robin keys (the paper's DS1 construction, Section 5.1), value =
    stream index t: tuple t is the m-th of group g = t mod G (m = t // G + 1)
    and its window holds the group's last c = min(m, w) tuples, whose indices
    are g + jG for j = m - c .. m - 1."""
    G, w = 7, 5
    o = oracle.WindowsOracle(G, w)
    t = np.arange(0, 400, dtype=np.int64)
    st, out = o.push((t % G).astype(np.int32), t.astype(np.int32))
    assert st == 0
    m = t // G + 1
    c = np.minimum(m, w)
    g = t % G
    expect = c * g + G * c * (2 * m - c - 1) // 2
    assert np.array_equal(out, expect)


def test_window_of_one_is_the_value():
    o = oracle.WindowsOracle(4, 1)
    rng = np.random.default_rng(1)
    keys = rng.integers(0, 4, 500).astype(np.int32)
    vals = rng.integers(I32_MIN, I32_MAX, 500).astype(np.int32)
    st, out = o.push(keys, vals)
    assert st == 0 and np.array_equal(out, vals.astype(np.int64))


def test_window_longer_than_the_stream_is_a_running_sum():
    rng = np.random.default_rng(2)
    keys = rng.integers(0, 3, 300).astype(np.int32)
    vals = rng.integers(-1000, 1000, 300).astype(np.int32)
    st, out = oracle.WindowsOracle(3, 1000).push(keys, vals)
    assert st == 0
    for g in range(3):
        sel = keys == g
        assert np.array_equal(out[sel], np.cumsum(vals[sel].astype(np.int64)))


def test_passes_do_not_change_the_sums():
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 50, 5000).astype(np.int32)
    vals = rng.integers(I32_MIN, I32_MAX, 5000).astype(np.int32)
    a = oracle.WindowsOracle(50, 17, 1).push(keys, vals)[1]
    b = oracle.WindowsOracle(50, 17, 10).push(keys, vals)[1]
    assert np.array_equal(a, b)


def test_group_sum_matches_last_output_and_bad_key_poisons():
    rng = np.random.default_rng(4)
    o = oracle.WindowsOracle(20, 6)
    keys = rng.integers(0, 20, 1000).astype(np.int32)
    vals = rng.integers(-50, 50, 1000).astype(np.int32)
    st, out = o.push(keys, vals)
    assert st == 0
    for g in range(20):
        idx = np.nonzero(keys == g)[0]
        s, c = o.group_sum(g)
        assert c == min(6, idx.size)
        assert s == (out[idx[-1]] if idx.size else 0)
    assert o.push(np.zeros(0, np.int32), np.zeros(0, np.int32))[0] == 0
    st, _ = o.push(np.array([1, 20], np.int32), np.array([5, 5], np.int32))
    assert st == oracle.EKEY
    assert o.seen == 1000
    assert o.push(np.array([1], np.int32), np.array([1], np.int32))[0] == oracle.EPOISONED
