"""The paper's load-balancing policies for its owner-computes GPU kernel
(Section 4, Algorithms getFirst, checkAll, probCheck, bestBalance, shift and
shiftLocal; the CPU side of Section 3.1).

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only ``tests/`` and the
benchmark's CPU legs use it.  Plain Python lists, one step at a time, in the
paper's order and notation, so that a reader can check it against the
algorithms by eye.

Model.  T GPU threads own the G groups; thread t's groups form an ordered
list (the thread-to-group mapping), and every group has exactly one owner
(the group-to-thread mapping).  Initially thread t owns the consecutive ids
[t G / T, (t + 1) G / T) (Section 5.1: an equal number of consecutive
groups).  A batch's tuples per thread, ``tpt``, follow from the mapping.
After a batch, a policy moves groups from loaded to lightly loaded threads;
the moves take effect from the next batch (Section 3.1: a delay of one
iteration).  ``threadThreshold`` defaults to 1000 and ``pot`` to 0.5
(Section 5.1).

Readings where the algorithms leave a choice open:
  - tmax is the thread with the most tuples, tmin the one with the fewest;
    ties go to the lowest thread index;
  - moving group g changes tpt by g's tuples in the current batch;
  - a moved group joins the end of tmin's list (getFirst, checkAll,
    probCheck, bestBalance); shift and shiftLocal keep neighbours' ids in
    order: a group moving down joins the end of the lower thread's list, a
    group moving up joins the front of the upper thread's list;
  - "the tuples of thread t" are the batch's reordered tuples of t's segment
    (its groups when the batch was laid out), in stream order, restricted to
    the groups t still owns at that point of the loop;
  - checkAll and bestBalance break ties by first occurrence in that scan;
    probCheck compares count >= pot * tpt[tmax] / ngroups in IEEE doubles;
  - shift moves every thread's group of one step at the same time (each
    thread's first or last group as the step begins);
  - the while loops also stop when an iteration moves nothing (an empty
    list, or probCheck finding no group at its limit), and after G moves.
"""
from __future__ import annotations

POLICIES = ("none", "getFirst", "checkAll", "probCheck", "bestBalance", "shift", "shiftLocal")


def initial_mapping(G: int, T: int) -> list:
    """Thread t owns groups [t G / T, (t + 1) G / T)."""
    return [list(range(t * G // T, (t + 1) * G // T)) for t in range(T)]


def owners(mapping: list, G: int) -> list:
    own = [-1] * G
    for t, groups in enumerate(mapping):
        for g in groups:
            own[g] = t
    return own


def reorder(mapping: list, keys: list) -> tuple:
    """The two-pass reorder of a batch (Section 3.1): count each thread's
    tuples, then place every tuple after the earlier ones of its thread.
    Returns (tpt, indicator, order) with order[j] the stream index of the
    j-th tuple of the reordered batch and thread t's tuples at
    [indicator[t], indicator[t + 1])."""
    T = len(mapping)
    own = owners(mapping, sum(len(groups) for groups in mapping))
    tpt = [0] * T
    for k in keys:                       # first pass: counts
        tpt[own[k]] += 1
    indicator = [0] * (T + 1)
    for t in range(T):
        indicator[t + 1] = indicator[t] + tpt[t]
    cursor = indicator[:T]
    order = [0] * len(keys)
    for i, k in enumerate(keys):         # second pass: placement
        t = own[k]
        order[cursor[t]] = i
        cursor[t] += 1
    return tpt, indicator, order


def _tmax(tpt):
    best = 0
    for t in range(1, len(tpt)):
        if tpt[t] > tpt[best]:
            best = t
    return best


def _tmin(tpt):
    best = 0
    for t in range(1, len(tpt)):
        if tpt[t] < tpt[best]:
            best = t
    return best


def rebalance(policy: str, mapping: list, keys: list, threshold: int = 1000, pot: float = 0.5) -> tuple:
    """Apply `policy` after a batch with stream keys `keys` laid out by
    `mapping`.  Returns (new mapping, groups moved)."""
    if policy not in POLICIES:
        raise ValueError(policy)
    G = sum(len(groups) for groups in mapping)
    T = len(mapping)
    m = [list(groups) for groups in mapping]
    own = owners(m, G)
    count = [0] * G                      # each group's tuples in this batch
    for k in keys:
        count[k] += 1
    tpt, indicator, order = reorder(mapping, keys)
    if policy == "none" or T < 2:
        return m, 0

    def segment(t):
        """Thread t's tuples in the reordered batch, of groups it still owns."""
        return [keys[order[j]] for j in range(indicator[t], indicator[t + 1]) if own[keys[order[j]]] == t]

    def move(g, src, dst, to_front=False):
        m[src].remove(g)
        if to_front:
            m[dst].insert(0, g)
        else:
            m[dst].append(g)
        own[g] = dst
        tpt[src] -= count[g]
        tpt[dst] += count[g]

    moves = 0
    if policy == "shiftLocal":
        for i in range(T - 1):
            if tpt[i] - tpt[i + 1] > threshold and m[i]:
                move(m[i][-1], i, i + 1, to_front=True)
                moves += 1
            elif tpt[i + 1] - tpt[i] > threshold and m[i + 1]:
                move(m[i + 1][0], i + 1, i)
                moves += 1
        return m, moves

    tmax, tmin = _tmax(tpt), _tmin(tpt)
    while tpt[tmax] - tpt[tmin] > threshold and moves < G:
        moved = 0
        if policy == "getFirst":
            if m[tmax]:
                move(m[tmax][0], tmax, tmin)
                moved = 1
        elif policy in ("checkAll", "bestBalance"):
            seen = []                    # groups in order of first occurrence
            occ = {}
            for g in segment(tmax):
                if g not in occ:
                    occ[g] = 0
                    seen.append(g)
                occ[g] += 1
            chosen = None
            if policy == "checkAll":
                for g in seen:
                    if chosen is None or occ[g] > occ[chosen]:
                        chosen = g
            else:
                for g in seen:
                    gap = abs((tpt[tmax] - occ[g]) - (tpt[tmin] + occ[g]))
                    if chosen is None or gap < best_gap:
                        chosen, best_gap = g, gap
            if chosen is not None:
                move(chosen, tmax, tmin)
                moved = 1
        elif policy == "probCheck":
            ngroups = len(m[tmax])
            if ngroups:
                limit = pot * tpt[tmax] / ngroups
                occ = {}
                for g in segment(tmax):
                    occ[g] = occ.get(g, 0) + 1
                    if occ[g] >= limit:
                        move(g, tmax, tmin)
                        moved = 1
                        break
        elif policy == "shift":
            if tmax > tmin:              # each thread in (tmin, tmax] gives its first group to the one below
                step = [(m[i][0], i, i - 1, False) for i in range(tmin + 1, tmax + 1) if m[i]]
            else:                        # each thread in [tmax, tmin) gives its last group to the one above
                step = [(m[i][-1], i, i + 1, True) for i in range(tmax, tmin) if m[i]]
            for g, src, dst, front in step:
                move(g, src, dst, to_front=front)
            moved = len(step)
        if moved == 0:
            break
        moves += moved
        tmax, tmin = _tmax(tpt), _tmin(tpt)
    return m, moves
