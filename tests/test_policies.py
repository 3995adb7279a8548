"""The paper's rebalancing policies (Section 4): the oracle pinned on small
cases worked by hand from the algorithms' steps, its invariants, and the
library's host implementation (cqo_rebalance, the step cqo_push runs) equal
to it, move for move, on random batches.  No device is used."""
import numpy as np
import pytest

from oracle import policies as P
import paper_1309_0634_b300 as cq


def keys_of(counts, order=None):
    """A batch with counts[g] tuples of group g, group by group in `order`."""
    order = order if order is not None else sorted(counts)
    out = []
    for g in order:
        out += [g] * counts[g]
    return out


def test_initial_mapping_and_two_pass_reorder():
    m = P.initial_mapping(10, 4)
    assert m == [[0, 1], [2, 3, 4], [5, 6], [7, 8, 9]]
    rng = np.random.default_rng(0)
    keys = rng.integers(0, 10, 200).tolist()
    tpt, ind, order = P.reorder(m, keys)
    own = P.owners(m, 10)
    expect = sorted(range(len(keys)), key=lambda i: (own[keys[i]], i))   # stable by owner
    assert order == expect
    assert ind == [0] + list(np.cumsum([sum(own[k] == t for k in keys) for t in range(4)]))
    assert tpt == [ind[t + 1] - ind[t] for t in range(4)]


def test_none_moves_nothing():
    m = [[0, 1], [2, 3]]
    assert P.rebalance("none", m, keys_of({0: 5000, 1: 1, 2: 1, 3: 1})) == (m, 0)


def test_get_first_ping_pongs_until_the_move_cap():
    # tpt [1600, 20]: g0 (1500) goes to t1; t1 then the most loaded gives its
    # first groups g2, g3 (10 each) and g0 back: four moves = G stops the loop
    m, moves = P.rebalance("getFirst", [[0, 1], [2, 3]], keys_of({0: 1500, 1: 100, 2: 10, 3: 10}))
    assert (m, moves) == ([[1, 2, 3, 0], []], 4)


def test_check_all_moves_the_most_frequent_group():
    # tpt [1400, 10]; g1 (900) is t0's most frequent: [500, 910], balanced
    m, moves = P.rebalance("checkAll", [[0, 1, 2], [3]], keys_of({0: 300, 1: 900, 2: 200, 3: 10}))
    assert (m, moves) == ([[0, 2], [3, 1]], 1)


def test_prob_check_takes_the_first_group_at_its_limit():
    # limit = 0.5 * 1500 / 4 = 187.5: in stream order g1's tuples come first
    counts = {0: 600, 1: 500, 2: 300, 3: 100, 4: 0}
    m, moves = P.rebalance("probCheck", [[0, 1, 2, 3], [4]], keys_of(counts, [1, 0, 2, 3]))
    assert (m, moves) == ([[0, 2, 3], [4, 1]], 1)
    m, moves = P.rebalance("probCheck", [[0, 1, 2, 3], [4]], keys_of(counts, [0, 1, 2, 3]))
    assert (m, moves) == ([[1, 2, 3], [4, 0]], 1)


def test_best_balance_differs_from_check_all():
    # t0: g0 1800, g1 1000, g2 300 (3100); t1: g3 1500.  Gaps after a move:
    # g0 |1300 - 3300| = 2000, g1 |2100 - 2500| = 400, g2 |2800 - 1800| = 1000
    keys = keys_of({0: 1800, 1: 1000, 2: 300, 3: 1500})
    assert P.rebalance("bestBalance", [[0, 1, 2], [3]], keys) == ([[0, 2], [3, 1]], 1)
    # checkAll moves g0 (the most frequent), overshoots, then g3 comes back
    assert P.rebalance("checkAll", [[0, 1, 2], [3]], keys) == ([[1, 2, 3], [0]], 2)


def test_shift_passes_groups_along_the_neighbours():
    # tpt [2000, 100, 50]: tmax 0 < tmin 2, so t0 and t1 pass their last
    # groups up; g1, g3 carry nothing; then g0, g2; then the pair turns and
    # g0 oscillates until six moves (= G)
    m, moves = P.rebalance("shift", [[0, 1], [2, 3], [4, 5]], keys_of({0: 2000, 2: 100, 4: 50}))
    assert (m, moves) == ([[], [0, 1], [2, 3, 4, 5]], 6)


def test_shift_local_is_one_pass_over_neighbours():
    # i = 0: 1500 - 200 > 1000, t0's last group g1 moves up -> [0, 1700, 0];
    # i = 1: 1700 - 0 > 1000, t1's last group g3 (no tuples) moves up
    m, moves = P.rebalance("shiftLocal", [[0, 1], [2, 3], [4, 5]], keys_of({1: 1500, 2: 200}))
    assert (m, moves) == ([[0], [1, 2], [3, 4, 5]], 2)


@pytest.mark.parametrize("policy", P.POLICIES)
def test_every_group_keeps_one_owner(policy):
    rng = np.random.default_rng(1)
    G, T = 97, 8
    m = P.initial_mapping(G, T)
    for _ in range(6):
        keys = (rng.zipf(1.4, 3000) % G).tolist()
        m, _ = P.rebalance(policy, m, keys, threshold=50)
        assert sorted(g for groups in m for g in groups) == list(range(G))


def _random_cases():
    rng = np.random.default_rng(2)
    cases = []
    for policy in P.POLICIES:
        for G, T, n, thr, pot in ((40, 4, 2000, 100, 0.5), (300, 16, 4000, 200, 0.5), (64, 64, 1000, 0, 1.0),
                                  (50, 2, 500, 1000, 0.25), (33, 5, 0, 10, 0.5), (7, 1, 300, 0, 0.5)):
            cases.append((policy, G, T, n, thr, pot, int(rng.integers(1 << 30))))
    return cases


@pytest.mark.parametrize("policy,G,T,n,thr,pot,seed", _random_cases())
def test_library_step_equals_the_oracle(policy, G, T, n, thr, pot, seed):
    """Several consecutive batches, skewed in shifting ways: the library's
    mapping and move count equal the oracle's after every step."""
    rng = np.random.default_rng(seed)
    m_lib = m_ref = P.initial_mapping(G, T)
    for step in range(5):
        s = 1.1 + 0.3 * step
        perm = rng.permutation(G)
        keys = perm[(rng.zipf(s, n) - 1) % G].astype(np.int32) if n else np.zeros(0, np.int32)
        m_ref, moves_ref = P.rebalance(policy, m_ref, keys.tolist(), threshold=thr, pot=pot)
        m_lib, moves_lib = cq.cqo_rebalance(policy, m_lib, keys, threshold=thr, pot=pot)
        assert m_lib == m_ref, (step, policy)
        assert moves_lib == moves_ref, (step, policy)


def test_rebalance_argument_errors():
    m = [[0, 1], [2]]
    with pytest.raises(cq.CQError):
        cq.cqo_rebalance("getFirst", m, np.array([3], np.int32))          # key outside [0, G)
    with pytest.raises(cq.CQError):
        cq.cqo_rebalance("getFirst", [[0, 1], [1]], np.array([0], np.int32))   # a group owned twice
    with pytest.raises(cq.CQError):
        cq.cqo_rebalance("probCheck", m, np.array([0], np.int32), pot=0.0)
