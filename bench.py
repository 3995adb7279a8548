#!/usr/bin/env python3
"""Benchmark of the per-batch update of a continuous windowed group-by.

Workload: the skew sweep -- one query over G = 10^5 groups with a global
count-based window of W = 10^6 tuples, batches of B = 10^6 tuples whose keys
are Zipf(s) over a randomly permuted ranking, s in {0, 0.5, 1, 1.5, 2},
int32 values uniform in [0, 10^6).  A step is one batch update: the batch is
folded in, the expiring tuples are retracted and SUM/COUNT/MIN/MAX/AVG of
every touched group are rewritten.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]

Per s, after W untimed batches, the K timed batches (distinct, resident in
HBM, 8 MB each, K*8 MB > L2) are pushed back to back through cq_push_many
(one persistent launch) with CUDA events around the call; this is repeated
--runs times (L2 flushed before each run) and the best and the median run
are reported.  The per-batch latency inside the launch comes from the
kernel's own %globaltimer stamps; the latency of a single cq_push of one
batch (L2 flushed before it) is reported beside it.  One JSON line is
printed by rank 0.  Under torchrun every rank runs an independent replica of
the workload (the query does not shard: replicas only), and the slowest
rank's time is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tuples/sec per batch update vs Zipf s (frac of HBM roofline); p99 batch latency"
UNIT = "tuples/s"
FALLBACK_HBM_GBS = 6400.0
L2_FLUSH_BYTES = 512 << 20


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# The sources that define the dominant kernel (the persistent stream push): a recorded
# DRAM traffic figure is valid while these are unchanged.
KERNEL_SOURCES = ("cq_stream.cu", "cq_stream.cuh", "cq_push_dev.cuh", "cq_tags.cuh", "cq_tma.cuh", "cq_internal.h",
                  "cq_avg.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1309_0634_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except Exception:
        return None, None
    if d.get("source_hash") != kernel_source_hash():
        return None, d
    return d, d


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


PATHS = {1: "push_kernel (partitioned, register-staged, one cooperative launch per push)",
         2: "ingest_kernel + finalize_kernel (direct atomics)",
         3: "group_kernel (partitioned, TMA-staged, one cooperative launch per push)",
         4: "stream_kernel (persistent producer/consumer launch over the whole batch sequence, cq_push_many)"}


def replica_seed(seed: int, rank: int) -> int:
    """Seed of a replica's stream: every rank runs an independent replica."""
    return seed + 1000 * rank


def max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's time (the query does not shard: ranks are replicas)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(tuples_per_rank: int, slowest_ms: float, world: int) -> float:
    """Whole-job tuples/s: the tuples all ranks pushed over the slowest rank's time."""
    return world * tuples_per_rank / (slowest_ms / 1e3)


def touched_groups(k_new, k_old, G):
    """U: distinct groups among the pushed and the expiring tuples."""
    a = np.bincount(k_new, minlength=G) > 0
    if k_old is not None:
        a |= np.bincount(k_old, minlength=G) > 0
    return int(a.sum())


def push_bytes(b_eff, expired, U):
    """Algorithmic HBM bytes of one push: new keys+values (8 B), ring write
    (8 B) and expired keys+values (8 B) per tuple, plus 68 B per touched
    group (20 B state read, 20 B state write, 28 B result write)."""
    return 16 * b_eff + 8 * expired + 68 * U


def needed_bytes(b_eff, expired, U, replaces):
    """The same count without the expired tuples when the push replaces the
    whole window: such a push never reads them (every old tuple leaves, and
    the new aggregates are those of the batch alone)."""
    return 16 * b_eff + (0 if replaces else 8 * expired) + 68 * U


def host_cpu():
    """Model name and logical core count of the host."""
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"model": model, "logical_cores": os.cpu_count()}


class OneCore:
    """Pin the calling process to one host core for the oracle's timing."""

    def __enter__(self):
        self.saved = None
        try:
            self.saved = os.sched_getaffinity(0)
            os.sched_setaffinity(0, {min(self.saved)})
        except (AttributeError, OSError):
            self.saved = None
        return self

    def __exit__(self, *exc):
        if self.saved is not None:
            os.sched_setaffinity(0, self.saved)


def run_cpu_baseline(sweep, batches_per_s):
    """The oracle, as it stands, on a bounded sample of the same workload:
    push + full results after every batch, single-threaded, pinned to one
    host core."""
    import oracle
    from streamgen import workloads
    with OneCore():
        return _cpu_baseline(oracle, workloads, sweep, batches_per_s)


def _cpu_baseline(oracle, workloads, sweep, batches_per_s):
    total_t, total_n = 0.0, 0
    for s in sweep:
        spec = workloads.config2(s)
        st = spec.stream()
        o = oracle.Oracle(spec.groups, spec.window)
        for i in range(batches_per_s):
            k, v = st.fill(i * spec.batch, spec.batch)
            t0 = time.perf_counter()
            o.push(k, v)
            o.results()
            total_t += time.perf_counter() - t0
            total_n += spec.batch
    return total_n / total_t, total_t, total_n


def run_reference(args, rank):
    if rank != 0:
        return
    sweep = [float(x) for x in args.sweep.split(",")]
    per_s = max(1, min(args.steps, 40))
    value, secs, n = run_cpu_baseline(sweep, per_s)
    sample = "first %d batches of 10^6 tuples for each s in %s (%d tuples, %.1f s of CPU time)" % (
        per_s, sweep, n, secs)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, n // 10**6),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": config_dict(args, sweep),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(args, sweep):
    return {"workload": "zipf_skew_sweep_G1e5_W1e6_B1e6", "groups": 100_000, "window": 1_000_000,
            "batch": 1_000_000, "zipf_s": sweep, "keys": "Zipf(s) over a permuted ranking",
            "values": "uniform int32 [0, 1e6)", "aggregates": "SUM,COUNT,MIN,MAX,AVG",
            "l2": "batches of a run (K x 8 MB) exceed L2; a 512 MB write flushes it before every run",
            "timed_pushes_per_s": args.steps, "warmup_pushes_per_s": args.warmup, "runs_per_s": args.runs,
            "timing": "CUDA events around one cq_push_many of the K batches (one persistent launch); best run"}


def run_sweep_s(cq, torch, dev, stream, spec, args, rank, flush, dist):
    """One s of the sweep: K timed batches pushed back to back through
    cq_push_many, --runs times; best and median run; per-batch latency from
    the launch's stamps; single-push latency beside it; algorithmic bytes
    from exact touched-group counts."""
    import ctypes
    spec.stream_kw["seed"] = replica_seed(spec.stream_kw["seed"], rank)
    st = spec.stream()
    nb = args.warmup + args.steps
    B, W, G = spec.batch, spec.window, spec.groups
    keys_h = torch.empty((nb, B), dtype=torch.int32, pin_memory=True)
    vals_h = torch.empty((nb, B), dtype=torch.int32, pin_memory=True)
    st.fill_into(0, nb * B, keys_h.data_ptr(), vals_h.data_ptr())
    kn = keys_h.numpy()
    U = [touched_groups(kn[i], kn[i - 1] if i else None, G) for i in range(nb)]
    keys_d = keys_h.to(dev, non_blocking=True)
    vals_d = vals_h.to(dev, non_blocking=True)
    torch.cuda.synchronize()
    q = cq.Query(G, W, cq.CQ_ALL, stream=stream)
    lib = cq.load()
    P = ctypes.c_void_p
    w = args.warmup
    if w:
        assert q.push_many([keys_d[i] for i in range(w)], [vals_d[i] for i in range(w)]) == cq.CQ_OK
    assert q.sync() == cq.CQ_OK
    K = args.steps
    ka = (P * K)(*[keys_d[w + i].data_ptr() for i in range(K)])
    va = (P * K)(*[vals_d[w + i].data_ptr() for i in range(K)])
    na = (ctypes.c_int64 * K)(*([B] * K))
    stamps = torch.empty(2 * K, dtype=torch.int64, device=dev)
    out = cq.cq_many_out(None, None, None, None, None, P(stamps.data_ptr()))
    st0 = q.stats()
    runs = []
    for r in range(args.runs):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(r & 0xFF)            # host enqueues the launch while this runs
        if dist:
            dist.barrier()
        e0.record(stream)
        st_ = lib.cq_push_many(q.handle, K, ka, va, na, ctypes.byref(out))
        e1.record(stream)
        torch.cuda.synchronize()
        if st_ != cq.CQ_OK or q.sync() != cq.CQ_OK:
            raise RuntimeError("cq_push_many failed: %s" % cq.cq_strerror(st_))
        sv = stamps.cpu().numpy().view(np.uint64).astype(np.int64)
        runs.append((e0.elapsed_time(e1), (sv[K:] - sv[:K]) / 1e6))
    st1 = q.stats()
    launches = st1["kernel_launches"] - st0["kernel_launches"]
    path = PATHS.get(st1["last_path"], str(st1["last_path"]))
    times = [t for t, _ in runs]
    best_i = int(np.argmin(times))
    best = max_over_ranks(times[best_i], dist, dev)
    med = float(np.median(times))
    lat = runs[best_i][1]
    # single pushes of one batch (latency of the per-push path), after the runs
    # and three untimed ones (the per-push path's first call sizes its scratch)
    for j in range(3):
        assert q.push(keys_d[w + j], vals_d[w + j]) == cq.CQ_OK
    torch.cuda.synchronize()
    single = []
    for j in range(min(10, K)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(j & 0xFF)
        e0.record(stream)
        assert q.push(keys_d[w + j], vals_d[w + j]) == cq.CQ_OK
        e1.record(stream)
        torch.cuda.synchronize()
        single.append(e0.elapsed_time(e1))
    q.close()
    bytes_ = sum(push_bytes(B, W, U[w + j]) for j in range(K))
    needed = sum(needed_bytes(B, W, U[w + j], B >= W) for j in range(K))
    peak, _ = measured_hbm_peak()
    res = {
        "tuples_per_s": job_throughput(B * K, best, 1 if dist is None else dist.get_world_size()),
        "ms_per_push": best / K, "ms_per_push_median_run": med / K, "runs": len(times),
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "single_push_p50_ms": float(np.percentile(single, 50)), "single_push_p99_ms": float(np.percentile(single, 99)),
        "touched_groups_mean": float(np.mean(U[w:])),
        "alg_bytes_per_push": bytes_ / K, "bytes_needed_per_push": needed / K,
        "frac": bytes_ / (best / 1e3) / 1e9 / peak, "frac_needed": needed / (best / 1e3) / 1e9 / peak,
        "_lat": list(lat), "_single": single, "_launches": launches, "_path": path, "_tuples": B * K,
        "_best_ms": best, "_bytes": bytes_, "_needed": needed,
        "_spec": spec, "_keys_h": keys_h, "_vals_h": vals_h}
    del keys_d, vals_d
    return res


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100, help="timed pushes per Zipf s")
    ap.add_argument("--warmup", type=int, default=3, help="untimed pushes per Zipf s")
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--sweep", default="0,0.5,1,1.5,2")
    ap.add_argument("--runs", type=int, default=5, help="timed runs of the K batches per s (best and median)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-batches", type=int, default=20, help="oracle batches per s for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched-rounds", type=int, default=100, help="timed rounds of the 64-query workload")
    ap.add_argument("--batched-warmup", type=int, default=12)
    ap.add_argument("--serve-seconds", type=float, default=5.0, help="seconds of arrivals of the serving workload")
    ap.add_argument("--no-extra", action="store_true", help="skip every workload beyond the skew sweep")
    ap.add_argument("--extra", default="uniform_small,drifting_skew,batched,paper_workload,serving",
                    help="comma list of the workloads beyond the skew sweep to run")
    ap.add_argument("--owner-batches", type=int, default=100,
                    help="timed batches per (dataset, grid, policy) of the owner-computes ablation")
    ap.add_argument("--paper-tuples", type=int, default=100_000_000,
                    help="tuples of each per-group-window dataset (the paper's 100M)")
    args = ap.parse_args()
    rank, world, local = env_rank()
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import paper_1309_0634_b300 as cq
    from streamgen import workloads

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    sweep = [float(x) for x in args.sweep.split(",")]
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    per_s = {}
    lat_all, single_all = [], []
    total_tuples = 0
    total_ms = 0.0
    total_bytes = 0
    total_needed = 0
    launches = 0
    path = None
    clocks = ClockSampler(local).start() if rank == 0 else None
    for si, s in enumerate(sweep):
        r = run_sweep_s(cq, torch, dev, stream, workloads.config2(s), args, rank, flush, dist)
        if args.e2e_steps and rank == 0 and s == sweep[len(sweep) // 2]:
            r["e2e"] = run_e2e(cq, torch, r.pop("_spec"), r.pop("_keys_h"), r.pop("_vals_h"), args, stream)
        for k in ("_spec", "_keys_h", "_vals_h"):
            r.pop(k, None)
        lat_all.extend(r.pop("_lat"))
        single_all.extend(r.pop("_single"))
        launches += r.pop("_launches")
        path = r.pop("_path")
        total_tuples += r.pop("_tuples")
        total_ms += r.pop("_best_ms")
        total_bytes += r.pop("_bytes")
        total_needed += r.pop("_needed")
        per_s["%.1f" % s] = r
    extra = {}
    wanted = set() if args.no_extra else {w for w in args.extra.split(",") if w}
    if "uniform_small" in wanted:
        extra["uniform_small"] = run_single(cq, torch, dev, stream, workloads.config1(), 3, rank, flush, many=True,
                                            runs=args.runs)
    if "drifting_skew" in wanted:
        extra["drifting_skew"] = run_single(cq, torch, dev, stream, workloads.config3(), 3, rank, flush)
    if "batched" in wanted:
        extra["batched"] = run_batched(cq, torch, dev, stream, args, rank, world, dist)
    if "paper_workload" in wanted:
        extra["paper_workload"] = run_paper(cq, torch, dev, stream, args, rank)
    if "serving" in wanted:
        extra["serving"] = run_serving(cq, torch, dev, args, rank, world, dist)
    clk = clocks.stop() if clocks else None

    peak, peak_kind = measured_hbm_peak()
    achieved = total_bytes / (total_ms / 1e3) / 1e9
    achieved_needed = total_needed / (total_ms / 1e3) / 1e9
    traffic, tinfo = recorded_traffic()
    value = job_throughput(total_tuples, total_ms, world)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    mid = per_s["%.1f" % sweep[len(sweep) // 2]]
    e2e = mid.get("e2e")
    nsteps = args.steps * len(sweep)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / nsteps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": dict(config_dict(args, sweep), parallelism="replicas" if world > 1 else "single"),
        "p50_ms": float(np.percentile(lat_all, 50)), "p99_ms": float(np.percentile(lat_all, 99)),
        "latency": {"what": "per batch inside the persistent launch: first producer start to last consumer "
                            "finish (%globaltimer stamps of the best runs)",
                    "p50_ms": float(np.percentile(lat_all, 50)), "p99_ms": float(np.percentile(lat_all, 99)),
                    "single_push_p50_ms": float(np.percentile(single_all, 50)),
                    "single_push_p99_ms": float(np.percentile(single_all, 99)),
                    "single_push": "one cq_push of one batch, L2 flushed before it, CUDA events"},
        "per_s": per_s,
        "roofline": {"bound": "hbm", "kernel": path,
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak,
                     "bytes_needed_per_push": total_needed / nsteps, "achieved_needed": achieved_needed,
                     "frac_needed": achieved_needed / peak,
                     "traffic": traffic["dram_bytes_per_push"] if traffic else None,
                     "alg_bytes_per_push": total_bytes / nsteps,
                     "timing": "events around back-to-back batches of one persistent launch (best of runs)"},
        "gpu_launches": launches,
        "clocks": clk,
    }
    line.update(extra)
    if e2e:
        line["e2e"] = e2e
    if not args.no_cpu_baseline:
        v, secs, n = run_cpu_baseline(sweep, args.cpu_batches)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
                                "sample": "first %d batches of each s (%d tuples, %.1f s), one pinned core" % (
                                    args.cpu_batches, n, secs)}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


class QueryStream:
    """Host copy of the stream one query of a multi-query workload is fed:
    round r pushes pool batch r mod len(pool).  Gives the keys of any range of
    stream positions, to count touched groups exactly."""

    def __init__(self, keys_pool, batch):
        self.pool = keys_pool      # list of int32 arrays of `batch` keys
        self.B = batch

    def keys(self, a, b):
        out = []
        while a < b:
            r, o = divmod(a, self.B)
            take = min(b - a, self.B - o)
            out.append(self.pool[r % len(self.pool)][o:o + take])
            a += take
        return np.concatenate(out) if out else np.zeros(0, np.int32)


def run_single(cq, torch, dev, stream, spec, warmup, rank, flush, many=False, runs=5):
    """One query over its whole stream (spec.batches pushes), the first
    `warmup` pushes untimed.  many=False: every other push timed alone with
    CUDA events after an L2 flush.  many=True: the remaining batches pushed
    back to back through one cq_push_many, `runs` times on fresh queries,
    best run (per-batch latency from the launch's stamps).  Algorithmic
    bytes use exact touched-group counts."""
    import ctypes
    kw = dict(spec.stream_kw)
    kw["seed"] = replica_seed(kw["seed"], rank)
    st = spec.__class__(spec.name, spec.groups, spec.window, spec.batch, spec.batches, kw).stream()
    nb, B, W, G = spec.batches, spec.batch, spec.window, spec.groups
    keys_h = torch.empty((nb, B), dtype=torch.int32, pin_memory=True)
    vals_h = torch.empty((nb, B), dtype=torch.int32, pin_memory=True)
    st.fill_into(0, nb * B, keys_h.data_ptr(), vals_h.data_ptr())
    kn = keys_h.numpy().reshape(-1)
    keys_d = keys_h.to(dev, non_blocking=True)
    vals_d = vals_h.to(dev, non_blocking=True)
    torch.cuda.synchronize()
    K = nb - warmup
    if many:
        lib = cq.load()
        P = ctypes.c_void_p
        ka = (P * K)(*[keys_d[i].data_ptr() for i in range(warmup, nb)])
        va = (P * K)(*[vals_d[i].data_ptr() for i in range(warmup, nb)])
        na = (ctypes.c_int64 * K)(*([B] * K))
        stamps = torch.empty(2 * K, dtype=torch.int64, device=dev)
        out = cq.cq_many_out(None, None, None, None, None, P(stamps.data_ptr()))
        best, lat, st0, st1 = None, None, None, None
        for r in range(runs):
            q = cq.Query(G, W, cq.CQ_ALL, stream=stream)
            if warmup:
                assert q.push_many([keys_d[i] for i in range(warmup)], [vals_d[i] for i in range(warmup)]) == cq.CQ_OK
            assert q.sync() == cq.CQ_OK
            s0 = q.stats()
            flush.fill_(r & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = lib.cq_push_many(q.handle, K, ka, va, na, ctypes.byref(out))
            e1.record(stream)
            torch.cuda.synchronize()
            if rc != cq.CQ_OK or q.sync() != cq.CQ_OK:
                raise RuntimeError("cq_push_many failed")
            t = e0.elapsed_time(e1)
            if best is None or t < best:
                sv = stamps.cpu().numpy().view(np.uint64).astype(np.int64)
                best, lat, st0, st1 = t, (sv[K:] - sv[:K]) / 1e6, s0, q.stats()
            q.close()
        ms = list(lat)
        t = best
        timing = "CUDA events around one cq_push_many of the %d batches, best of %d runs; latency from stamps" % (
            K, runs)
    else:
        q = cq.Query(G, W, cq.CQ_ALL, stream=stream)
        for i in range(warmup):
            assert q.push(keys_d[i], vals_d[i]) == cq.CQ_OK
        assert q.sync() == cq.CQ_OK
        st0 = q.stats()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        torch.cuda.synchronize()
        for j, i in enumerate(range(warmup, nb)):
            flush.fill_(j & 0xFF)
            ev[j][0].record(stream)
            if q.push(keys_d[i], vals_d[i]) != cq.CQ_OK:
                raise RuntimeError("push failed")
            ev[j][1].record(stream)
        torch.cuda.synchronize()
        assert q.sync() == cq.CQ_OK
        st1 = q.stats()
        ms = [a.elapsed_time(b) for a, b in ev]
        t = sum(ms)
        q.close()
        timing = "every push timed alone with CUDA events after a 512 MB L2 flush"
    total_bytes, total_needed = 0, 0
    for i in range(warmup, nb):
        N = i * B
        lo, hi = max(0, N - W), max(0, N + B - W)
        b_eff = min(B, W)
        touched = np.bincount(kn[N + B - b_eff:N + B], minlength=G) > 0
        if hi > lo:
            touched |= np.bincount(kn[lo:hi], minlength=G) > 0
        U = int(touched.sum())
        total_bytes += push_bytes(b_eff, hi - lo, U)
        total_needed += needed_bytes(b_eff, hi - lo, U, B >= W and N > 0)
    peak, kind = measured_hbm_peak()
    achieved = total_bytes / (t / 1e3) / 1e9
    achieved_needed = total_needed / (t / 1e3) / 1e9
    return {"workload": spec.name, "pushes_timed": K, "tuples_per_s": K * B / (t / 1e3),
            "ms_per_push": t / K, "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
            "flips": st1["flips"] - st0["flips"], "resets": st1["resets"] - st0["resets"],
            "path": PATHS[st1["last_path"]].split(" ")[0], "timing": timing,
            "l2": "flushed before every timed push or run (512 MB write)",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": kind, "unit": "GB/s",
                         "frac": achieved / peak, "alg_bytes_per_push": total_bytes / K,
                         "bytes_needed_per_push": total_needed / K, "frac_needed": achieved_needed / peak}}


def run_batched(cq, torch, dev, stream, args, rank, world=1, dist=None):
    """The batched workload: 64 standing queries (log-uniform G and W, B =
    W / 10, Zipf s uniform in [0, 2]), one group launch per round pushing one
    batch to every query.  Rounds cycle over a pool of distinct batches per
    query (pool > L2); rounds are timed after the windows have filled.
    Under torchrun the queries are split over the ranks (each query on one
    GPU, balanced by its bytes per round; no data exchange), every rank runs
    the rounds of its own queries, and the job's time is the slowest rank's."""
    from streamgen import workloads
    from paper_1309_0634_b300 import shard
    all_specs = workloads.config4()
    parts = shard.assign_queries([shard.round_bytes(sp.groups, sp.window, sp.batch) for sp in all_specs], world,
                                 [cq.cq_footprint_bytes(sp.groups, sp.window) for sp in all_specs])
    mine = parts[rank]
    specs = [all_specs[i] for i in mine]
    npool, warm = 6, max(12, args.batched_warmup)
    qs, kd, vd, host = [], [], [], []
    for qi, sp in enumerate(specs):
        kw = dict(sp.stream_kw)   # a query's stream does not depend on the rank hosting it
        st = sp.__class__(sp.name, sp.groups, sp.window, sp.batch, 0, kw).stream()
        k, v = st.fill(0, npool * sp.batch)
        k = k.reshape(npool, sp.batch)
        v = v.reshape(npool, sp.batch)
        host.append(QueryStream([k[i] for i in range(npool)], sp.batch))
        bpad = (sp.batch + 3) // 4 * 4            # 16-byte aligned batch rows
        kp = np.zeros((npool, bpad), np.int32)
        vp = np.zeros((npool, bpad), np.int32)
        kp[:, :sp.batch] = k
        vp[:, :sp.batch] = v
        kd.append(torch.from_numpy(kp).to(dev)[:, :sp.batch])
        vd.append(torch.from_numpy(vp).to(dev)[:, :sp.batch])
        qs.append(cq.Query(sp.groups, sp.window, cq.CQ_ALL, stream=stream))
    torch.cuda.synchronize()
    # admission: each member is pinned to the group kernel's path and tuned
    # on its own first batch (partition width, heavy-hitter cap, threshold)
    tuned, t_tune = [], time.perf_counter()
    for i, q in enumerate(qs):
        q.set_option("path", 1)
        st_, us = cq.cq_autotune(q.handle, kd[i][0], vd[i][0], specs[i].batch, 2)
        if st_ != cq.CQ_OK:
            raise RuntimeError("autotune failed: %s" % cq.cq_strerror(st_))
        tuned.append({"query": specs[i].name, "partition_bits": q.get_option("partition_bits"),
                      "hot_keys": q.get_option("hot_keys"), "hot_threshold": q.get_option("hot_threshold"),
                      "us_per_push_alone": us})
    t_tune = time.perf_counter() - t_tune
    g = cq.Group(stream)
    B = [sp.batch for sp in specs]

    def round_(r):
        p = r % npool
        st = g.push(qs, [kd[i][p] for i in range(len(qs))], [vd[i][p] for i in range(len(qs))])
        if st != cq.CQ_OK:
            raise RuntimeError("group push failed: %s" % cq.cq_strerror(st))

    for r in range(warm):
        round_(r)
    torch.cuda.synchronize()
    launches0 = g.stats()
    rounds = args.batched_rounds
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(rounds + 1)]
    e0.record(stream)
    for j in range(rounds):
        ev[j].record(stream)
        round_(warm + j)
    ev[rounds].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    total_ms = e0.elapsed_time(e1)
    per_round = [ev[j].elapsed_time(ev[j + 1]) for j in range(rounds)]
    st1 = g.stats()
    # algorithmic bytes of every timed push (exact touched-group counts)
    total_bytes, total_needed, tuples = 0, 0, 0
    for i, sp in enumerate(specs):
        W, b = sp.window, sp.batch
        period = npool * b
        cache = {}
        for j in range(rounds):
            r = warm + j
            N = r * b
            b_eff = min(b, W)
            lo, hi = max(0, N - W), max(0, N + b - W)
            key = (N % period, lo % period, hi - lo)     # the stream repeats with the pool
            if key not in cache:
                new = host[i].keys(N + b - b_eff, N + b)
                old = host[i].keys(lo, hi)
                cache[key] = int(((np.bincount(new, minlength=sp.groups) > 0)
                                  | (np.bincount(old, minlength=sp.groups) > 0)).sum())
            total_bytes += push_bytes(b_eff, hi - lo, cache[key])
            total_needed += needed_bytes(b_eff, hi - lo, cache[key], b >= W and N > 0)
            tuples += b
    for q in qs:
        q.close()
    g.close()
    if dist is not None:
        import torch as _t
        t = _t.tensor([total_bytes, total_needed, tuples], dtype=_t.float64, device=dev)
        dist.all_reduce(t)                                   # job totals (timing-side numbers only)
        total_bytes, total_needed, tuples = float(t[0]), float(t[1]), float(t[2])
        total_ms = max_over_ranks(total_ms, dist, dev)
    peak, kind = measured_hbm_peak()
    achieved = total_bytes / (total_ms / 1e3) / 1e9
    return {"workload": "64 queries, G log-U[1e2,1e6], W log-U[1e3,1e7], B=W/10, Zipf s U[0,2]",
            "sharding": {"ranks": world, "queries_per_rank": [len(x) for x in parts],
                         "how": "each query on one GPU (LPT by bytes per round); no data exchange; "
                                "job time = slowest rank"},
            "autotune": {"what": "cq_autotune per member at admission, path pinned to the group kernel (1); "
                                 "partition width, heavy-hitter cap and threshold chosen per query",
                         "seconds": t_tune, "choices": tuned},
            "rounds": rounds, "warmup_rounds": warm, "tuples_per_round": sum(B),
            "ms_per_round": total_ms / rounds, "p50_ms": float(np.percentile(per_round, 50)),
            "p99_ms": float(np.percentile(per_round, 99)), "tuples_per_s": tuples / (total_ms / 1e3),
            "launches": st1["launches"] - launches0["launches"],
            "graph_launches": st1["graph_launches"] - launches0["graph_launches"],
            "l2": "rounds cycle over %d distinct batches per query (%.0f MB > L2)" % (
                npool, npool * sum(B) * 8 / 1e6),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": kind, "unit": "GB/s",
                         "frac": achieved / peak, "alg_bytes_per_round": total_bytes / rounds,
                         "bytes_needed_per_round": total_needed / rounds,
                         "frac_needed": total_needed / (total_ms / 1e3) / 1e9 / peak}}


def run_serving(cq, torch, dev, args, rank, world=1, dist=None):
    """The serving workload: 256 standing queries (as in the batched one), a
    Poisson stream of requests at 2e9 tuples/s aggregate, batch sizes
    log-uniform in [1e3, 1e6]; each request's tuples are a slice of its
    query's pre-generated device pool.  Latency = completion - arrival.
    Under torchrun the queries are split over the ranks (balanced by device
    footprint; each request is served by its query's rank, no exchange)."""
    from streamgen import workloads
    from paper_1309_0634_b300 import shard
    specs = workloads.config5()
    pool_len = 1 << 20
    qs_, idx, arr, sizes = workloads.serving_requests(len(specs), args.serve_seconds, seed=5)
    parts = shard.assign_queries([cq.cq_footprint_bytes(sp.groups, sp.window) for sp in specs], world)
    mine = set(parts[rank])
    keep = np.array([int(q) in mine for q in qs_], dtype=bool)
    qs_, idx, arr, sizes = qs_[keep], idx[keep], arr[keep], sizes[keep]
    srv = cq.Server(200 << 30)
    served, pools = [], []
    for qi, sp in enumerate(specs):
        if qi not in mine:
            served.append(None)
            pools.append(None)
            continue
        kw = dict(sp.stream_kw)   # a query's stream does not depend on the rank hosting it
        k, v = sp.__class__(sp.name, sp.groups, sp.window, 0, 0, kw).stream().fill(0, pool_len)
        pools.append((torch.from_numpy(k).to(dev), torch.from_numpy(v).to(dev)))
        served.append(srv.admit(sp.groups, sp.window, cq.CQ_ALL, 10**6))
    torch.cuda.synchronize()
    keys, vals, queries = [], [], []
    for q, i, n in zip(qs_, idx, sizes):
        o = workloads.serving_pool_offset(int(q), int(i), int(n), pool_len)
        keys.append(pools[q][0][o:o + n])
        vals.append(pools[q][1][o:o + n])
        queries.append(served[q])
    st = srv.replay(queries, arr, keys, vals)
    if st != cq.CQ_OK:
        raise RuntimeError("serving replay failed: %s" % cq.cq_strerror(st))
    d = srv.stats()
    srv.close()
    offered = float(sizes.sum()) / args.serve_seconds
    achieved = d["tuples"] / d["busy_s"] if d["busy_s"] else 0.0
    sharding = {"ranks": world, "queries_per_rank": [len(x) for x in parts],
                "how": "each query on one GPU (LPT by device footprint); requests served by their query's rank"}
    if dist is not None:
        import torch as _t
        t = _t.tensor([offered, achieved], dtype=_t.float64, device=dev)
        dist.all_reduce(t)
        offered, achieved = float(t[0]), float(t[1])
        p99 = max_over_ranks(d["latency_p99_us"], dist, dev)
        sharding["p99_ms_slowest_rank"] = p99 / 1e3
    return {"workload": "256 queries, Poisson arrivals at 2e9 tuples/s, batches log-U[1e3,1e6]",
            "sharding": sharding,
            "arrival_seconds": args.serve_seconds, "batches": d["completed"], "tuples": d["tuples"],
            "offered_tuples_per_s": offered,
            "achieved_tuples_per_s": achieved,
            "p50_ms": d["latency_p50_us"] / 1e3, "p99_ms": d["latency_p99_us"] / 1e3,
            "max_ms": d["latency_max_us"] / 1e3, "mean_ms": d["latency_mean_us"] / 1e3,
            "launches": d["launches"], "batches_per_launch": d["batches_launched"] / max(1, d["launches"]),
            "reserved_gb": d["reserved_bytes"] / 1e9}


PAPER_GPU_TUPLES_PER_S = 1.25e7   # the paper's GTX 460 on DS2 with its best balancing: about 8 s per 100M tuples


def run_paper(cq, torch, dev, stream, args, rank):
    """The paper's own workload (Section 5.1): 40,000 groups with a window of
    100 values each, batches of 50K, every tuple's window SUM recomputed
    from scratch (once, and ten times for DS2).  All pushes of a dataset are
    timed back to back with CUDA events; the dataset (800 MB for 100M
    tuples) is resident in HBM and larger than L2.  The oracle runs the same
    work on one host core over the first 20 batches."""
    import oracle
    from streamgen import workloads
    out = {"workload": "per-group windows w=100, G=40000, batches of 50K, SUM recomputed per tuple",
           "paper_context_tuples_per_s": PAPER_GPU_TUPLES_PER_S}
    for name, passes in (("DS1", 1), ("DS2", 1), ("DS3", 1), ("DS2", 10)):
        sp = workloads.paper_dataset(name, tuples=args.paper_tuples, seed=replica_seed(0, rank))
        nb, B = sp.batches, sp.batch
        keys_h = torch.empty((nb, B), dtype=torch.int32, pin_memory=True)
        vals_h = torch.empty((nb, B), dtype=torch.int32, pin_memory=True)
        sp.stream().fill_into(0, nb * B, keys_h.data_ptr(), vals_h.data_ptr())
        keys_d = keys_h.to(dev, non_blocking=True)
        vals_d = vals_h.to(dev, non_blocking=True)
        sums = torch.empty(B, dtype=torch.int64, device=dev)
        torch.cuda.synchronize()
        q = cq.GroupWindows(sp.groups, sp.window, passes, stream=stream)
        warm = 3
        for i in range(warm):
            assert q.push(keys_d[i], vals_d[i], sums) == cq.CQ_OK
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = q.stats()["kernel_launches"]
        e0.record(stream)
        for i in range(warm, nb):
            if q.push(keys_d[i], vals_d[i], sums) != cq.CQ_OK:
                raise RuntimeError("per-group window push failed")
        e1.record(stream)
        torch.cuda.synchronize()
        if q.sync() != cq.CQ_OK:
            raise RuntimeError("per-group window push failed")
        ms = e0.elapsed_time(e1)
        tuples = (nb - warm) * B
        launches = q.stats()["kernel_launches"] - l0
        q.close()
        o = oracle.WindowsOracle(sp.groups, sp.window, passes)
        kh, vh = keys_h.numpy(), vals_h.numpy()
        t0 = time.perf_counter()
        for i in range(min(20, nb)):
            o.push(kh[i], vh[i])
        cpu_s = time.perf_counter() - t0
        cpu = min(20, nb) * B / cpu_s
        gpu = tuples / (ms / 1e3)
        out["%s%s" % (name, "" if passes == 1 else "_%dpasses" % passes)] = {
            "passes": passes, "tuples": tuples, "ms": ms, "us_per_batch": 1e3 * ms / (nb - warm),
            "tuples_per_s": gpu, "kernel_launches_per_batch": launches / (nb - warm),
            "oracle_tuples_per_s_1core": cpu, "vs_oracle": gpu / cpu,
            "vs_paper_gpu": gpu / PAPER_GPU_TUPLES_PER_S}
        if passes == 1 and args.owner_batches > 0:
            own = out.setdefault("owner_computes", {
                "what": "the paper's owner-computes kernel with its six host rebalancing policies (Section 4), "
                        "256 threads a block, threadThreshold 1000, pot 0.5; host lay-out and rebalancing "
                        "overlap the previous batch's kernel; wall clock from the first push to the last sync",
                "batches": min(args.owner_batches, nb - warm)})
            own[name] = run_owner(cq, torch, dev, stream, sp, kh, vh, min(args.owner_batches, nb - warm), warm)
        del keys_d, vals_d, keys_h, vals_h
    return out


def run_owner(cq, torch, dev, stream, sp, kh, vh, batches, warm):
    """Owner-computes ablation for one dataset: per grid size and policy, the
    wall time per batch and the throughput normalised to no balance (the
    paper's Tables 1 and 2)."""
    res = {}
    sums = torch.empty(sp.batch, dtype=torch.int64, device=dev)

    def one(grid, policy, device):
        q = cq.OwnerWindows(sp.groups, sp.window, 1, grid=grid, policy=policy, stream=stream, device=device)
        for i in range(warm):
            assert q.push(kh[i], vh[i], sums) == cq.CQ_OK
        assert q.sync() == cq.CQ_OK
        m0 = q.stats()["moves"]
        t0 = time.perf_counter()
        for i in range(warm, warm + batches):
            if q.push(kh[i], vh[i], sums) != cq.CQ_OK:
                raise RuntimeError("owner-computes push failed")
        if q.sync() != cq.CQ_OK:
            raise RuntimeError("owner-computes push failed")
        dt = time.perf_counter() - t0
        st = q.stats()
        q.close()
        return {"us_per_batch": 1e6 * dt / batches, "tuples_per_s": batches * sp.batch / dt,
                "moves": st["moves"] - m0, "host_us_per_batch": st["host_ns"] / 1e3 / st["pushes"]}

    for grid in (4, 64):
        row = {policy: one(grid, policy, False) for policy in cq.CQO_POLICIES}
        # the same policies with the lay-out and the policy loop on the device
        row["device"] = {policy: one(grid, policy, True) for policy in cq.CQO_DEVICE_POLICIES}
        for r in (row, row["device"]):
            base = r["none"]["tuples_per_s"]
            for policy in cq.CQO_POLICIES:
                if policy in r:
                    r[policy]["normalized"] = r[policy]["tuples_per_s"] / base
        res["grid%d" % grid] = row
    return res


def run_e2e(cq, torch, spec, keys_h, vals_h, args, stream):
    """Same pushes through the public host-buffer API: every step copies its
    batch up from pinned host memory (cq_push_host) and reads every group's
    five results back into pinned host memory (cq_results_copy_async), timed
    on the host from the first call to the last result on the host.  Steps
    are issued back to back: a batch's copy up overlaps the push and the
    result read of the step before it, as in a streaming deployment."""
    G = spec.groups
    res = [[torch.empty(G, dtype=dt, pin_memory=True) for dt in (torch.int64, torch.int32, torch.int32, torch.int32,
                                                                  torch.float64)] for _ in range(2)]
    q = cq.Query(spec.groups, spec.window, cq.CQ_ALL, stream=stream)
    n = min(args.e2e_steps, keys_h.shape[0])
    for i in range(min(2, n)):
        cq.cq_push_host(q.handle, keys_h[i], vals_h[i], spec.batch)
        cq.cq_results_copy(q.handle, *res[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(n):
        assert cq.cq_push_host(q.handle, keys_h[i], vals_h[i], spec.batch) == cq.CQ_OK
        assert cq.cq_results_copy_async(q.handle, *res[i & 1]) == cq.CQ_OK
    assert q.sync() == cq.CQ_OK
    dt = time.perf_counter() - t0
    last = res[(n - 1) & 1]
    counts_ok = int(last[1].sum()) == min(spec.window, spec.batch * (n + min(2, n)))   # COUNT adds up to the window
    q.close()
    return {"value": n * spec.batch / dt, "unit": UNIT, "h2d_bytes_per_step": 8 * spec.batch,
            "d2h_bytes_per_step": 28 * G, "steps": n, "timing": "host wall clock, steps pipelined",
            "last_counts_sum_to_window": counts_ok}


if __name__ == "__main__":
    main()
