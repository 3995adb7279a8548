"""Host logic of multi-process runs (CPU, gloo, world size 2).

A query does not shard across GPUs here: ranks run independent replicas of
the workload, and the job's time is the slowest rank's."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    from streamgen import workloads
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import torch
        t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, torch.device("cpu"))
        spec = workloads.config2(1.5)
        spec.stream_kw["seed"] = bench.replica_seed(spec.stream_kw["seed"], rank)
        k, _ = spec.stream().fill(0, 1000)
        out.put((rank, t, bench.job_throughput(10**6, t, world), k.tolist()))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_independent_streams():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, k0), (r1, t1, v1, k1) = res
    assert t0 == t1 == 15.0                      # both ranks see the maximum
    assert v0 == v1 == 2 * 10**6 / 0.015         # all ranks' tuples over the slowest time
    assert not np.array_equal(k0, k1)            # replicas push different streams


def test_reference_arm_prints_once_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--sweep", "0"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["cpu_baseline"]["kind"] == "oracle" and d["value"] > 0
