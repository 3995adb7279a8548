"""AVG is the fp64 quotient RN(RN(SUM) / COUNT) (Section 2).  The
finalisations take it by integer long division (cq_avg.cuh), so it is
checked two ways: against the device's own fp64 division on drawn pairs
over the whole range of sums and counts (cq_check_avg), and against the
oracle on every path, with groups whose sums run far past 2^32 in both
signs (values at the ends of the int32 range)."""
import numpy as np
import pytest

import paper_1309_0634_b300 as cq
from gpu_util import run_pair
from test_stream_gpu import run_many

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [1, 0x5EED, 2**63 + 12345])
def test_avg_division_matches_fp64_division(seed):
    st, bad = cq.cq_check_avg(1 << 24, seed)
    assert st == cq.CQ_OK
    assert bad == 0


def test_check_avg_arguments():
    assert cq.cq_check_avg(0, 1) == (cq.CQ_OK, 0)
    assert cq.cq_check_avg(-1, 1)[0] == cq.CQ_EINVAL


def _extreme_batches(G, n, count, seed):
    """Keys uniform over G; group g's values sit at the top of the int32
    range when g % 3 == 0, at the bottom when g % 3 == 1, and spread over the
    whole range otherwise, so sums reach about 2^47 in either sign."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        k = rng.integers(0, G, n).astype(np.int32)
        noise = rng.integers(0, 1 << 20, n)
        top = (2**31 - 1) - noise
        bottom = -(2**31) + noise
        spread = rng.integers(-(2**31), 2**31, n)
        v = np.where(k % 3 == 0, top, np.where(k % 3 == 1, bottom, spread)).astype(np.int32)
        out.append((k, v))
    return out


@pytest.mark.parametrize("path", [0, 1, 2, 3])
def test_avg_of_large_sums_every_path(path):
    """Windows of 2^18 tuples over 7 groups: about 37,000 tuples a group, a
    window full of retractions after the fourth push."""
    G, W = 7, 1 << 18
    batches = _extreme_batches(G, 1 << 16, 10, seed=path + 3)
    run_pair(G, W, batches, options={"path": path} if path else None)


def test_avg_of_large_sums_persistent_launch():
    G, W = 7, 1 << 18
    batches = _extreme_batches(G, 1 << 16, 10, seed=9)
    run_many(G, W, batches, calls=[3, 7])
