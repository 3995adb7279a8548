"""Synthetic workloads: the stream recipes of the five benchmark configurations.

Only input shapes live here (group counts, window and batch lengths, key and
value distributions, seeds); no aggregation arithmetic.  The paper's own
datasets (Section 5.1: 100M tuples over 40,000 groups, round robin DS1, Zipf
DS2, permuted Zipf DS3, batches of 50K) are not available; these seeded
streams stand in for them with the same structure.
"""
from __future__ import annotations

from dataclasses import dataclass, field

from . import Stream, log_uniform_int, unit_double

ZIPF_SWEEP = (0.0, 0.5, 1.0, 1.5, 2.0)


@dataclass
class QuerySpec:
    """One standing query and the stream that feeds it."""
    name: str
    groups: int
    window: int
    batch: int                 # tuples per push (fixed-batch workloads)
    batches: int               # pushes in the full workload
    stream_kw: dict = field(default_factory=dict)

    def stream(self) -> Stream:
        return Stream(self.groups, **self.stream_kw)

    @property
    def tuples(self) -> int:
        return self.batch * self.batches


def config1() -> QuerySpec:
    """Single query, uniform keys over 1,000 groups, W = B = 10^4, 10^6 tuples."""
    return QuerySpec("uniform_G1e3_W1e4_B1e4", 1000, 10_000, 10_000, 100,
                     dict(keys="uniform", vals="uniform", lo=0, hi=10**6, seed=1))


def config2(s: float) -> QuerySpec:
    """Skew sweep: 10^5 groups, Zipf(s) keys over a permuted ranking, W = B = 10^6,
    10^8 tuples per s."""
    idx = ZIPF_SWEEP.index(s) if s in ZIPF_SWEEP else int(round(s * 10)) + 10
    return QuerySpec("zipf%.1f_G1e5_W1e6_B1e6" % s, 100_000, 1_000_000, 1_000_000, 100,
                     dict(keys="zipf", s=s, permute=True, vals="uniform", lo=0, hi=10**6, seed=2 + idx))


def config3() -> QuerySpec:
    """Drifting skew: 10^6 groups, Zipf(1.2) whose permutation is re-drawn every
    20 batches, normal(5e5, 1e5) values clipped to [0, 10^6), W = 4*10^6,
    B = 2*10^6, 2*10^8 tuples."""
    B = 2_000_000
    return QuerySpec("drift_zipf1.2_G1e6_W4e6_B2e6", 1_000_000, 4_000_000, B, 100,
                     dict(keys="zipf", s=1.2, permute=True, repermute_every=20 * B, vals="normal",
                          mean=5e5, sd=1e5, lo=0, hi=999_999, seed=3))


def multi_query(n_queries: int, seed: int, batches: int, prefix: str) -> list:
    """Standing queries with log-uniform G in [10^2, 10^6], log-uniform W in
    [10^3, 10^7], B = W / 10 and Zipf s uniform in [0, 2]."""
    out = []
    for q in range(n_queries):
        G = log_uniform_int(seed, 4 * q, 100, 10**6)
        W = log_uniform_int(seed, 4 * q + 1, 1000, 10**7)
        s = 2.0 * unit_double(seed, 4 * q + 2)
        B = max(1, W // 10)
        out.append(QuerySpec("%s%d_G%d_W%d_s%.2f" % (prefix, q, G, W, s), G, W, B, batches,
                             dict(keys="zipf", s=s, permute=True, vals="uniform", lo=0, hi=10**6,
                                  seed=1000 * seed + q)))
    return out


def config4() -> list:
    """64 standing queries pushed together, 100 rounds of one batch per query."""
    return multi_query(64, seed=4, batches=100, prefix="batched")


def config5() -> list:
    """256 standing queries of the serving loop (batch sizes drawn per request)."""
    return multi_query(256, seed=5, batches=0, prefix="serve")


def serving_batch_size(query: int, i: int, seed: int = 5) -> int:
    """Size of request i of a serving query: log-uniform in [10^3, 10^6]."""
    return log_uniform_int(seed * 7919 + query, i, 1000, 10**6)


SERVING_TUPLES_PER_S = 2e9   # aggregate arrival rate of the serving configuration


def serving_requests(n_queries: int, duration_s: float, tuples_per_s: float = SERVING_TUPLES_PER_S,
                     seed: int = 5, max_batch: int = 10**6):
    """Requests of the serving loop: a Poisson process of batches whose sizes
    are log-uniform in [10^3, max_batch] (request i of query q has size
    serving_batch_size(q, i) clipped to max_batch); each arrival goes to a
    query drawn uniformly.  The rate makes the expected tuple arrival rate
    tuples_per_s.  Returns (query, index within the query, arrival ns, size)
    as numpy arrays, in arrival order."""
    import numpy as np
    mean = (10**6 - 10**3) / np.log(10**3)          # mean of log-uniform [1e3, 1e6]
    rate = tuples_per_s / mean                       # batches per second
    rng = np.random.Generator(np.random.PCG64(seed))
    expect = int(rate * duration_s * 1.2) + 64
    gaps = rng.exponential(1.0 / rate, size=expect)
    t = np.cumsum(gaps)
    t = t[t < duration_s]
    qs = rng.integers(0, n_queries, size=t.size)
    idx = np.zeros(t.size, np.int64)
    counters = np.zeros(n_queries, np.int64)
    for j, q in enumerate(qs):
        idx[j] = counters[q]
        counters[q] += 1
    sizes = np.array([min(serving_batch_size(int(q), int(i), seed), max_batch) for q, i in zip(qs, idx)], np.int64)
    return qs.astype(np.int64), idx, (t * 1e9).astype(np.int64), sizes


def serving_pool_offset(query: int, i: int, n: int, pool: int) -> int:
    """Start of request i of a query inside the query's pre-generated pool of
    `pool` tuples (requests reuse slices of one pool per query)."""
    span = pool - n + 1
    return 0 if span <= 1 else (i * 2654435761 + query * 40503) % span


# The paper's own workload (Section 5.1): 100M tuples over 40,000 groups in
# batches of 50K, a window of 100 values per group.  DS1 assigns groups
# round robin; DS2 is Zipf with group y more frequent than group z when
# z > y (ranks not permuted; the exponent is not given: 1.0 is used); DS3 is
# DS2 randomly permuted.  Values: uniform [0, 10^6) (not given either).
PAPER_GROUPS, PAPER_WINDOW, PAPER_BATCH, PAPER_TUPLES = 40_000, 100, 50_000, 100_000_000
PAPER_ZIPF_S = 1.0


def paper_dataset(name: str, tuples: int = PAPER_TUPLES, seed: int = 0) -> QuerySpec:
    """DS1, DS2 or DS3 of the paper's experiments as a stream spec."""
    keys = {"DS1": dict(keys="round_robin"),
            "DS2": dict(keys="zipf", s=PAPER_ZIPF_S, permute=False),
            "DS3": dict(keys="zipf", s=PAPER_ZIPF_S, permute=True)}[name]
    kw = dict(keys, vals="uniform", lo=0, hi=10**6, seed=seed + {"DS1": 51, "DS2": 52, "DS3": 53}[name])
    return QuerySpec("%s_G%d_w%d_B%d" % (name, PAPER_GROUPS, PAPER_WINDOW, PAPER_BATCH), PAPER_GROUPS,
                     PAPER_WINDOW, PAPER_BATCH, tuples // PAPER_BATCH, kw)
