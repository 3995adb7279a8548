"""Pins of the CPU oracle against results fixed by something other than itself.

The oracle (oracle/oracle.c) is the plain definition of the query of
Section 3 (a group-by over (id, attr) tuples whose aggregates depend on a
fixed-size window of recent tuples), processed in batch iterations
(Section 3.1), under the global count-based window reading.  Each test below
fixes the expected values independently of the oracle's code:

* a hand-derived worked example (tests/golden/hand_example.txt);
* a brute force over the full stream history in pure Python (no ring buffer,
  no modular indexing) on an exhaustive small grid;
* closed forms for round-robin keys (the paper's DS1 construction,
  Section 5.1) with values equal to the stream index;
* numpy reductions for a single group;
* invariants (total count, total sum from an independent prefix sum,
  MIN <= AVG <= MAX, empty-group sentinels);
* CPython's IEEE double arithmetic for AVG, including sums above 2**53 where
  the int64 -> double conversion rounds.
"""
import math
import os
import random
import struct

import numpy as np
import pytest

import oracle
import streamgen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
INT32_MAX = 2**31 - 1
INT32_MIN = -(2**31)


def f64_bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def expected_from_values(values):
    """(sum, count, min, max, avg) of a list of ints, using CPython only."""
    if not values:
        return 0, 0, INT32_MAX, INT32_MIN, float("nan")
    s = sum(values)
    return s, len(values), min(values), max(values), float(s) / float(len(values))


def check_group(res, g, exp):
    s, c, lo, hi, avg = exp
    assert int(res["sum"][g]) == s, (g, "sum")
    assert int(res["count"][g]) == c, (g, "count")
    assert int(res["min"][g]) == lo, (g, "min")
    assert int(res["max"][g]) == hi, (g, "max")
    got = float(res["avg"][g])
    if c == 0:
        assert f64_bits(got) == oracle.NAN_BITS, (g, "avg sentinel")
    else:
        assert f64_bits(got) == f64_bits(avg), (g, "avg", got, avg)


# --------------------------------------------------------------------------
# Hand-worked example
# --------------------------------------------------------------------------

def test_hand_worked_example():
    lines = open(os.path.join(GOLDEN, "hand_example.txt")).read().splitlines()
    q = None
    G = W = None
    nexp = 0
    for raw in lines:
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        tok = line.split()
        if tok[0] == "groups":
            G = int(tok[1])
        elif tok[0] == "window":
            W = int(tok[1])
            q = oracle.Oracle(G, W)
        elif tok[0] in ("push", "push_status"):
            want = 0
            pairs = tok[1:]
            if tok[0] == "push_status":
                want, pairs = int(tok[1]), tok[2:]
            keys = [int(p.split(":")[0]) for p in pairs]
            vals = [int(p.split(":")[1]) for p in pairs]
            assert q.push(np.array(keys, np.int32), np.array(vals, np.int32)) == want
        elif tok[0] == "read_status":
            with pytest.raises(oracle.OracleError) as ei:
                q.results()
            assert ei.value.status == int(tok[1])
        elif tok[0] == "expect":
            g, s, c, lo, hi = (int(x) for x in tok[1:6])
            avg = float(tok[6])
            check_group(q.results(), g, (s, c, lo, hi, avg))
            nexp += 1
    assert nexp == 21


# --------------------------------------------------------------------------
# Brute force over the full history
# --------------------------------------------------------------------------

def brute_force(history, G, W):
    window = history[max(0, len(history) - W):]
    per = [[] for _ in range(G)]
    for k, v in window:
        per[k].append(v)
    return [expected_from_values(p) for p in per]


EXTREMES = [INT32_MIN, INT32_MIN + 1, -1, 0, 1, INT32_MAX - 1, INT32_MAX]


@pytest.mark.parametrize("G", [1, 2, 3, 8])
@pytest.mark.parametrize("W", [1, 2, 3, 5, 8, 13, 31, 64])
def test_brute_force_small_grid(G, W):
    rng = random.Random(1000 * G + W)
    q = oracle.Oracle(G, W)
    history = []
    for step in range(12):
        b = rng.randint(0, 2 * W)
        keys = [rng.randrange(G) for _ in range(b)]
        vals = [rng.choice(EXTREMES) if rng.random() < 0.3 else rng.randint(-1000, 1000) for _ in range(b)]
        assert q.push(np.array(keys, np.int32), np.array(vals, np.int32)) == 0
        history.extend(zip(keys, vals))
        assert q.seen == len(history)
        res = q.results()
        for g, exp in enumerate(brute_force(history, G, W)):
            check_group(res, g, exp)


# --------------------------------------------------------------------------
# Closed forms: round-robin keys, values = lo + stream index
# --------------------------------------------------------------------------

def round_robin_closed_form(G, lo, L, R, g):
    """Group g over stream indices [L, R) with key t mod G and value lo + t."""
    if R <= L:
        return expected_from_values([])
    first = L + ((g - L) % G)
    last = (R - 1) - ((R - 1 - g) % G)
    if first > R - 1:
        return expected_from_values([])
    c = (last - first) // G + 1
    s = c * lo + (first + last) * c // 2
    return s, c, lo + first, lo + last, float(s) / float(c)


@pytest.mark.parametrize("G,W,batches", [
    (7, 50, [10, 0, 60, 3, 49, 50, 51, 1]),
    (10, 100, [100] * 5),                 # B = W: window = exactly the last batch
    (64, 1000, [333, 777, 1, 2000, 999]),
    (1, 9, [4, 4, 4, 20]),
])
def test_round_robin_closed_form(G, W, batches):
    lo = -5000
    st = streamgen.Stream(G, keys="round_robin", vals="index", lo=lo, hi=lo + 10**9, seed=0)
    q = oracle.Oracle(G, W)
    N = 0
    for b in batches:
        k, v = st.fill(N, b)
        assert q.push(k, v) == 0
        N += b
        res = q.results()
        L, R = max(0, N - W), N
        for g in range(G):
            check_group(res, g, round_robin_closed_form(G, lo, L, R, g))
        if W % G == 0 and N >= W:
            assert (res["count"] == W // G).all()


# --------------------------------------------------------------------------
# Single group: numpy reductions over the last W values
# --------------------------------------------------------------------------

def test_single_group_matches_numpy():
    rng = np.random.default_rng(5)
    W = 777
    q = oracle.Oracle(1, W)
    hist = np.empty(0, np.int64)
    for b in [100, 900, 0, 1, 5000, 776, 778]:
        v = rng.integers(INT32_MIN, INT32_MAX, size=b, endpoint=True, dtype=np.int64)
        assert q.push(np.zeros(b, np.int32), v.astype(np.int32)) == 0
        hist = np.concatenate([hist, v])
        win = hist[-W:]
        r = q.results()
        assert int(r["sum"][0]) == int(win.sum())
        assert int(r["count"][0]) == win.size
        assert int(r["min"][0]) == int(win.min())
        assert int(r["max"][0]) == int(win.max())
        assert f64_bits(float(r["avg"][0])) == f64_bits(float(int(win.sum())) / float(win.size))


# --------------------------------------------------------------------------
# Invariants on skewed random streams
# --------------------------------------------------------------------------

@pytest.mark.parametrize("s", [0.0, 1.0, 2.0])
def test_invariants_zipf(s):
    G, W = 500, 3000
    st = streamgen.Stream(G, keys="zipf", s=s, vals="uniform", lo=-10**6, hi=10**6, seed=11)
    q = oracle.Oracle(G, W)
    allv = np.empty(0, np.int64)
    N = 0
    for b in [1000, 2500, 4000, 10, 3000, 2999, 1]:
        k, v = st.fill(N, b)
        assert q.push(k, v) == 0
        N += b
        allv = np.concatenate([allv, v.astype(np.int64)])
        pref = np.concatenate([[0], np.cumsum(allv)])
        r = q.results()
        assert int(r["count"].sum()) == min(W, N)
        assert int(r["sum"].sum()) == int(pref[N] - pref[max(0, N - W)])
        ne = r["count"] > 0
        assert (r["min"][ne] <= r["avg"][ne]).all() and (r["avg"][ne] <= r["max"][ne]).all()
        assert (r["sum"][~ne] == 0).all()
        assert (r["min"][~ne] == INT32_MAX).all() and (r["max"][~ne] == INT32_MIN).all()
        assert (r["avg"][~ne].view(np.uint64) == oracle.NAN_BITS).all()


# --------------------------------------------------------------------------
# AVG rounding: int64 -> double conversion and IEEE division
# --------------------------------------------------------------------------

def test_avg_rounds_like_ieee_double_above_2_pow_53():
    # 2**53 + 1 is not a double: (double)SUM must round it (to nearest even).
    target = 2**53 + 1
    n_full = target // INT32_MAX
    rem = target - n_full * INT32_MAX
    vals = np.full(n_full + 1, INT32_MAX, dtype=np.int32)
    vals[-1] = rem
    q = oracle.Oracle(1, n_full + 1)
    assert q.push(np.zeros(vals.size, np.int32), vals) == 0
    r = q.results()
    assert int(r["sum"][0]) == target
    want = float(target) / float(vals.size)   # CPython: correctly rounded conversion and division
    assert f64_bits(float(r["avg"][0])) == f64_bits(want)
    # For this sum the double-rounded value differs from the correctly rounded
    # exact quotient, so dividing in wider precision would be caught.
    assert want != target / vals.size


def test_avg_division_rounding_small():
    q = oracle.Oracle(3, 10)
    assert q.push(np.array([0, 0, 0, 1, 1, 2], np.int32), np.array([1, 1, 0, -1, 0, 2], np.int32)) == 0
    r = q.results()
    assert f64_bits(float(r["avg"][0])) == f64_bits(2.0 / 3.0)
    assert f64_bits(float(r["avg"][1])) == f64_bits(-0.5)
    assert math.copysign(1.0, float(r["avg"][1])) == -1.0


# --------------------------------------------------------------------------
# Argument handling and poisoning
# --------------------------------------------------------------------------

def test_bad_key_poisons_and_rejects():
    q = oracle.Oracle(4, 8)
    assert q.push(np.array([0, 1], np.int32), np.array([5, 6], np.int32)) == 0
    assert q.push(np.array([2, 4], np.int32), np.array([5, 6], np.int32)) == oracle.EKEY
    assert q.seen == 2
    assert q.push(np.array([0], np.int32), np.array([1], np.int32)) == oracle.EPOISONED
    with pytest.raises(oracle.OracleError):
        q.results()
    q2 = oracle.Oracle(4, 8)
    assert q2.push(np.array([-1], np.int32), np.array([0], np.int32)) == oracle.EKEY


@pytest.mark.parametrize("G,W", [(0, 1), (1, 0), (2**31, 1), (1, 2**31), (-1, 5)])
def test_create_rejects_bad_sizes(G, W):
    with pytest.raises(oracle.OracleError) as ei:
        oracle.Oracle(G, W)
    assert ei.value.status == oracle.EINVAL


def test_group_query_agrees_with_full_results():
    st = streamgen.Stream(50, keys="zipf", s=1.5, seed=3)
    q = oracle.Oracle(50, 400)
    k, v = st.fill(0, 1000)
    q.push(k, v)
    r = q.results()
    for g in range(50):
        s, c, lo, hi, a = q.group(g)
        assert (s, c, lo, hi) == (int(r["sum"][g]), int(r["count"][g]), int(r["min"][g]), int(r["max"][g]))
        assert f64_bits(a) == f64_bits(float(r["avg"][g]))
