"""Pins of the seeded input generator (shared input of the oracle and the CUDA path)."""
import math

import numpy as np
import pytest
from scipy import stats

import streamgen


def test_splitmix64_published_vector():
    # First outputs of SplitMix64 seeded with 1234567, as published with the
    # reference implementation of the generator (Steele, Lea, Flood 2014; Vigna).
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [streamgen.splitmix64(1234567, i) for i in range(5)] == want


def test_fill_is_deterministic_and_split_invariant():
    st = streamgen.Stream(1000, keys="zipf", s=1.2, repermute_every=700, vals="normal", lo=0, hi=999999, seed=9)
    k, v = st.fill(0, 5000)
    st2 = streamgen.Stream(1000, keys="zipf", s=1.2, repermute_every=700, vals="normal", lo=0, hi=999999, seed=9)
    parts = [st2.fill(a, b) for a, b in [(0, 1), (1, 699), (700, 2000), (2700, 2300)]]
    assert (np.concatenate([p[0] for p in parts]) == k).all()
    assert (np.concatenate([p[1] for p in parts]) == v).all()


@pytest.mark.parametrize("s", [0.0, 0.5, 1.0, 1.5, 2.0])
def test_zipf_frequencies_chi_square(s):
    G, n = 50, 200_000
    st = streamgen.Stream(G, keys="zipf", s=s, permute=False, seed=21)
    k, _ = st.fill(0, n)
    p = np.arange(1, G + 1, dtype=np.float64) ** (-s)
    p /= p.sum()
    obs = np.bincount(k, minlength=G)
    chi2 = (((obs - n * p) ** 2) / (n * p)).sum()
    assert stats.chi2.sf(chi2, G - 1) > 1e-4


@pytest.mark.parametrize("s,share", [(1.5, 1 / 2.6058), (2.0, 1 / 1.64492)])
def test_top_key_share_matches_zeta(s, share):
    G, n = 100_000, 1_000_000
    st = streamgen.Stream(G, keys="zipf", s=s, permute=True, seed=2)
    k, _ = st.fill(0, n)
    top = np.bincount(k, minlength=G).max() / n
    assert abs(top - share) < 0.01


def test_permutation_moves_heavy_hitters():
    G = 10_000
    st = streamgen.Stream(G, keys="zipf", s=1.2, permute=True, repermute_every=100_000, seed=4)
    a, _ = st.fill(0, 100_000)
    b, _ = st.fill(100_000, 100_000)
    top_a = np.argmax(np.bincount(a, minlength=G))
    top_b = np.argmax(np.bincount(b, minlength=G))
    assert top_a == st.key_of_rank(0, 0)
    assert top_b == st.key_of_rank(100_000, 0)
    assert top_a != top_b
    perm = [st.key_of_rank(0, r) for r in range(G)]
    assert sorted(perm) == list(range(G))


def test_uniform_keys_and_values_in_range():
    st = streamgen.Stream(1000, keys="uniform", vals="uniform", lo=0, hi=10**6, seed=1)
    k, v = st.fill(0, 200_000)
    assert k.min() == 0 and k.max() == 999
    assert v.min() >= 0 and v.max() < 10**6
    assert stats.chisquare(np.bincount(k, minlength=1000)).pvalue > 1e-4


def test_normal_clipped_moments():
    st = streamgen.Stream(10, keys="uniform", vals="normal", mean=5e5, sd=1e5, lo=0, hi=999_999, seed=8)
    _, v = st.fill(0, 400_000)
    assert abs(v.mean() - (5e5 - 0.5)) < 1e3
    assert abs(v.std() - 1e5) < 1e3
    assert v.min() >= 0 and v.max() <= 999_999


def test_log_uniform_int():
    xs = [streamgen.log_uniform_int(77, i, 100, 10**6) for i in range(20000)]
    assert min(xs) >= 100 and max(xs) <= 10**6
    logs = np.log(np.array(xs, dtype=np.float64))
    assert abs(logs.mean() - (math.log(100) + math.log(10**6)) / 2) < 0.05
