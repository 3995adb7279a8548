"""Placement of independent queries on the ranks of a multi-GPU job (CPU).

The batched and serving workloads shard by query: every query lives on one
rank, no data moves between ranks, and every rank computes the same
placement on its own.  Checked here: each query on exactly one rank, the
longest-processing-time bound on the heaviest rank, and two gloo ranks
arriving at one disjoint cover without exchanging it.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1309_0634_b300 import shard  # noqa: E402


def _batched_weights():
    from streamgen import workloads
    specs = workloads.config4()
    return [shard.round_bytes(sp.groups, sp.window, sp.batch) for sp in specs]


def _serving_weights():
    import paper_1309_0634_b300 as cq
    from streamgen import workloads
    return [cq.cq_footprint_bytes(sp.groups, sp.window) for sp in workloads.config5()]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("which", ["batched", "serving"])
def test_every_query_on_exactly_one_rank_and_balanced(world, which):
    w = _batched_weights() if which == "batched" else _serving_weights()
    parts = shard.assign_queries(w, world)
    assert len(parts) == world
    flat = sorted(q for p in parts for q in p)
    assert flat == list(range(len(w)))                     # a cover, no query twice
    loads = [sum(w[q] for q in p) for p in parts]
    # list scheduling, heaviest first: no rank exceeds the mean by more than one query
    assert max(loads) <= sum(w) / world + max(w) + 1e-6
    assert shard.assign_queries(w, world) == parts         # deterministic


def test_small_hand_case():
    # weights 5, 4, 3, 3, 1 on two ranks: 5 -> r0, 4 -> r1, 3 -> r1 (4 < 5), 3 -> r0, 1 -> r1 (7 < 8)
    assert shard.assign_queries([5, 4, 3, 3, 1], 2) == [[0, 3], [1, 2, 4]]
    # equal weights: memory breaks the tie, then the rank index
    assert shard.assign_queries([1, 1, 1], 2, memory=[10, 1, 1]) == [[0], [1, 2]]
    with pytest.raises(ValueError):
        shard.assign_queries([1], 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = {}
        for which in ("batched", "serving"):
            w = _batched_weights() if which == "batched" else _serving_weights()
            parts = shard.assign_queries(w, world)
            mine = parts[rank]
            everyone = [None] * world
            dist.all_gather_object(everyone, mine)   # only to check the cover; the job itself exchanges nothing
            res[which] = (parts, everyone)
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_compute_one_disjoint_cover():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for which, n in (("batched", 64), ("serving", 256)):
        parts0, seen0 = res[0][which]
        parts1, seen1 = res[1][which]
        assert parts0 == parts1                      # both ranks placed the queries alike
        assert seen0 == seen1 == parts0              # each rank took its own share
        assert not set(parts0[0]) & set(parts0[1])   # disjoint
        assert sorted(parts0[0] + parts0[1]) == list(range(n))
