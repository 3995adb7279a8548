"""Python binding of libcq, the B300 continuous windowed group-by engine.

This module only marshals arguments to the C ABI declared in
``include/cq.h``; every step of the hot path runs in the CUDA kernels of
``libcq.so``.  There is no CPU fallback: if the library was not built, or no
CUDA device is present, the calls raise.

Functions carry the C names (``cq_create``, ``cq_push``, ...).  ``Query`` is a
small convenience wrapper over them for torch tensors and numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcq.so")

CQ_OK, CQ_EINVAL, CQ_ENOMEM, CQ_EKEY, CQ_ECUDA, CQ_ETIMEOUT, CQ_EBUSY, CQ_EPOISONED, CQ_EBUDGET, CQ_ESCRATCH = range(10)
CQ_SUM, CQ_COUNT, CQ_MIN, CQ_MAX, CQ_AVG, CQ_ALL = 1, 2, 4, 8, 16, 31
CQ_OPT_HOT_KEYS, CQ_OPT_HOT_THRESHOLD, CQ_OPT_WARP_AGG = 1, 3, 4
CQ_OPT_CTAS_PER_SM, CQ_OPT_PARTITION_BITS, CQ_OPT_PATH = 5, 7, 8
CQ_OPT_WAIT_LIMIT_US, CQ_OPT_STALL_BATCH, CQ_OPT_STREAM_PRODUCERS = 9, 10, 11

CUDA_STREAM_LEGACY = 0x1   # cudaStreamLegacy
CQ_NOALLOC_SCRATCH_BYTES = 32 << 20

# Every function the C ABI exports (include/cq.h).
EXPORTS = ("cq_create", "cq_footprint_bytes", "cq_push", "cq_push_host", "cq_results", "cq_results_copy",
           "cq_results_copy_async", "cq_sync", "cq_destroy", "cq_strerror", "cq_set_option", "cq_get_option",
           "cq_stats", "cq_hot_list", "cq_trace", "cq_autotune", "cqg_create", "cqg_push", "cqg_sync", "cqg_stats",
           "cqg_destroy", "cq_push_noalloc", "cq_push_many", "cqs_now_ns", "cqs_create", "cqs_admit", "cqs_submit", "cqs_wait",
           "cqs_drain", "cqs_replay", "cqs_stats", "cqs_reset_stats", "cqs_destroy", "cqw_create", "cqw_push",
           "cqw_sync", "cqw_stats", "cqw_destroy", "cqo_create", "cqo_push", "cqo_sync", "cqo_stats", "cqo_mapping",
           "cqo_rebalance", "cqo_destroy", "cq_check_avg")
CQ_TRACE_STAMPS = 8


class cq_result_view(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_int64), ("sum", ctypes.c_void_p), ("count", ctypes.c_void_p),
                ("min", ctypes.c_void_p), ("max", ctypes.c_void_p), ("avg", ctypes.c_void_p)]


class cq_many_out(ctypes.Structure):
    _fields_ = [("sum", ctypes.c_void_p), ("count", ctypes.c_void_p), ("min", ctypes.c_void_p),
                ("max", ctypes.c_void_p), ("avg", ctypes.c_void_p), ("stamps", ctypes.c_void_p)]


class cqs_server_stats(ctypes.Structure):
    _fields_ = [("queries", ctypes.c_int64), ("reserved_bytes", ctypes.c_int64), ("budget_bytes", ctypes.c_int64),
                ("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("tuples", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("batches_launched", ctypes.c_int64),
                ("latency_p50_us", ctypes.c_double), ("latency_p99_us", ctypes.c_double),
                ("latency_max_us", ctypes.c_double), ("latency_mean_us", ctypes.c_double),
                ("busy_s", ctypes.c_double)]


class cqo_stats_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("tuples_seen", "pushes", "moves", "last_moves", "last_max_tpt",
                                              "last_min_tpt", "host_ns")]


CQO_POLICIES = ("none", "getFirst", "checkAll", "probCheck", "bestBalance", "shift", "shiftLocal")
CQO_ON_DEVICE = 16   # lay-out and policy on the device (cqo_create's policy flag)
CQO_DEVICE_POLICIES = CQO_POLICIES[:5]


class cq_query_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("tuples_seen", "window_len", "pushes", "flips", "resets",
                                              "hot_keys", "device_bytes", "kernel_launches", "last_path",
                                              "heavy_folds")]


class CQError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s: %s (status %d)" % (what, cq_strerror(status) if _lib else "?", status))
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libcq.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libcq.so is missing (%s): build it with __graft_entry__.build() "
                           "or python -m paper_1309_0634_b300._build" % path)
    lib = ctypes.CDLL(path)
    c = ctypes
    P = c.c_void_p
    lib.cq_create.restype = c.c_int
    lib.cq_create.argtypes = [c.c_int64, c.c_int64, c.c_uint32, P, c.POINTER(P)]
    lib.cq_footprint_bytes.restype = c.c_int64
    lib.cq_footprint_bytes.argtypes = [c.c_int64, c.c_int64, c.c_uint32]
    lib.cq_push.restype = c.c_int
    lib.cq_push.argtypes = [P, P, P, c.c_int64]
    lib.cq_push_host.restype = c.c_int
    lib.cq_push_host.argtypes = [P, P, P, c.c_int64]
    lib.cq_push_noalloc.restype = c.c_int
    lib.cq_push_noalloc.argtypes = [P, P, P, c.c_int64]
    lib.cq_push_many.restype = c.c_int
    lib.cq_push_many.argtypes = [P, c.c_int, P, P, P, P]
    lib.cq_results.restype = c.c_int
    lib.cq_results.argtypes = [P, c.POINTER(cq_result_view)]
    lib.cq_results_copy.restype = c.c_int
    lib.cq_results_copy.argtypes = [P, P, P, P, P, P]
    lib.cq_results_copy_async.restype = c.c_int
    lib.cq_results_copy_async.argtypes = [P, P, P, P, P, P]
    lib.cq_sync.restype = c.c_int
    lib.cq_sync.argtypes = [P]
    lib.cq_destroy.restype = None
    lib.cq_destroy.argtypes = [P]
    lib.cq_strerror.restype = c.c_char_p
    lib.cq_strerror.argtypes = [c.c_int]
    lib.cq_set_option.restype = c.c_int
    lib.cq_set_option.argtypes = [P, c.c_int, c.c_int64]
    lib.cq_get_option.restype = c.c_int
    lib.cq_get_option.argtypes = [P, c.c_int, c.POINTER(c.c_int64)]
    lib.cq_stats.restype = c.c_int
    lib.cq_stats.argtypes = [P, c.POINTER(cq_query_stats)]
    lib.cq_hot_list.restype = c.c_int
    lib.cq_hot_list.argtypes = [P, c.POINTER(c.c_int32), c.POINTER(c.c_int32), c.c_int, c.POINTER(c.c_int)]
    lib.cq_trace.restype = c.c_int
    lib.cq_trace.argtypes = [P, P, c.c_int64]
    lib.cq_check_avg.restype = c.c_int
    lib.cq_check_avg.argtypes = [c.c_int64, c.c_uint64, c.POINTER(c.c_int64)]
    lib.cqg_create.restype = c.c_int
    lib.cqg_create.argtypes = [P, c.POINTER(P)]
    lib.cqg_push.restype = c.c_int
    lib.cqg_push.argtypes = [P, c.c_int, P, P, P, P, P]
    lib.cqg_sync.restype = c.c_int
    lib.cqg_sync.argtypes = [P]
    lib.cqg_destroy.restype = None
    lib.cqg_destroy.argtypes = [P]
    lib.cqg_stats.restype = c.c_int
    lib.cqg_stats.argtypes = [P, P, P]
    lib.cq_autotune.restype = c.c_int
    lib.cq_autotune.argtypes = [P, P, P, c.c_int64, c.c_int, P]
    lib.cqw_create.restype = c.c_int
    lib.cqw_create.argtypes = [c.c_int64, c.c_int32, c.c_int32, P, c.POINTER(P)]
    lib.cqw_push.restype = c.c_int
    lib.cqw_push.argtypes = [P, P, P, c.c_int64, P]
    lib.cqw_sync.restype = c.c_int
    lib.cqw_sync.argtypes = [P]
    lib.cqw_stats.restype = c.c_int
    lib.cqw_stats.argtypes = [P, P, P, P]
    lib.cqw_destroy.restype = None
    lib.cqw_destroy.argtypes = [P]
    lib.cqo_create.restype = c.c_int
    lib.cqo_create.argtypes = [c.c_int64, c.c_int32, c.c_int32, c.c_int32, c.c_int32, c.c_int64, c.c_double, P,
                               c.POINTER(P)]
    lib.cqo_push.restype = c.c_int
    lib.cqo_push.argtypes = [P, P, P, c.c_int64, P]
    lib.cqo_sync.restype = c.c_int
    lib.cqo_sync.argtypes = [P]
    lib.cqo_stats.restype = c.c_int
    lib.cqo_stats.argtypes = [P, c.POINTER(cqo_stats_t)]
    lib.cqo_mapping.restype = c.c_int
    lib.cqo_mapping.argtypes = [P, P, P]
    lib.cqo_rebalance.restype = c.c_int
    lib.cqo_rebalance.argtypes = [c.c_int32, c.c_int32, c.c_int64, P, P, P, c.c_int64, c.c_int64, c.c_double, P, P,
                                  c.POINTER(c.c_int64)]
    lib.cqo_destroy.restype = None
    lib.cqo_destroy.argtypes = [P]
    lib.cqs_now_ns.restype = c.c_int64
    lib.cqs_now_ns.argtypes = []
    lib.cqs_create.restype = c.c_int
    lib.cqs_create.argtypes = [c.c_int64, P, c.POINTER(P)]
    lib.cqs_admit.restype = c.c_int
    lib.cqs_admit.argtypes = [P, c.c_int64, c.c_int64, c.c_uint32, c.c_int64, c.POINTER(P)]
    lib.cqs_submit.restype = c.c_int
    lib.cqs_submit.argtypes = [P, P, P, P, c.c_int64, c.c_int64, c.POINTER(c.c_int64)]
    lib.cqs_wait.restype = c.c_int
    lib.cqs_wait.argtypes = [P, c.c_int64]
    lib.cqs_drain.restype = c.c_int
    lib.cqs_drain.argtypes = [P]
    lib.cqs_replay.restype = c.c_int
    lib.cqs_replay.argtypes = [P, c.c_int64, P, P, P, P, P]
    lib.cqs_stats.restype = c.c_int
    lib.cqs_stats.argtypes = [P, c.POINTER(cqs_server_stats)]
    lib.cqs_reset_stats.restype = c.c_int
    lib.cqs_reset_stats.argtypes = [P]
    lib.cqs_destroy.restype = None
    lib.cqs_destroy.argtypes = [P]
    _lib = lib
    return lib


def _ptr(x) -> int:
    """Address of a torch tensor, numpy array or integer pointer."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("expected a tensor, an array or an address, got %r" % type(x))


def _check(st: int, what: str) -> int:
    if st != CQ_OK:
        raise CQError(st, what)
    return st


# ---- the C ABI, one function each -------------------------------------------

def cq_strerror(status: int) -> str:
    return load().cq_strerror(int(status)).decode()


def cq_footprint_bytes(groups: int, window: int, aggs: int = CQ_ALL) -> int:
    return int(load().cq_footprint_bytes(int(groups), int(window), int(aggs)))


def cq_create(groups: int, window: int, aggs: int = CQ_ALL, stream: int = 0):
    """Returns (status, handle)."""
    h = ctypes.c_void_p()
    st = load().cq_create(int(groups), int(window), int(aggs), ctypes.c_void_p(int(stream)), ctypes.byref(h))
    return st, h


def cq_push(q, d_keys, d_vals, n: int) -> int:
    return int(load().cq_push(q, ctypes.c_void_p(_ptr(d_keys)), ctypes.c_void_p(_ptr(d_vals)), int(n)))


def cq_push_noalloc(q, d_keys, d_vals, n: int) -> int:
    """cq_push with the kernel's scratch taken from the library's fixed area."""
    return int(load().cq_push_noalloc(q, ctypes.c_void_p(_ptr(d_keys)), ctypes.c_void_p(_ptr(d_vals)), int(n)))


def cq_push_many(q, d_keys, d_vals, n, out=None) -> int:
    """Push len(n) batches in order in one persistent launch: d_keys[j] /
    d_vals[j] (device tensors or addresses) hold batch j's n[j] tuples.
    ``out`` is None or a dict of device tensors: "sum", "count", "min",
    "max", "avg" of len(n) * groups entries (results after every batch)
    and/or "stamps" of 2 * len(n) words."""
    k = len(n)
    P = ctypes.c_void_p
    ka = (P * max(k, 1))(*[_ptr(x) for x in d_keys])
    va = (P * max(k, 1))(*[_ptr(x) for x in d_vals])
    na = (ctypes.c_int64 * max(k, 1))(*[int(x) for x in n])
    o = None
    if out:
        o = cq_many_out(*[P(_ptr(out.get(f))) for f in ("sum", "count", "min", "max", "avg", "stamps")])
    return int(load().cq_push_many(q, int(k), ka, va, na, ctypes.byref(o) if o is not None else None))


def cq_push_host(q, h_keys, h_vals, n: int) -> int:
    return int(load().cq_push_host(q, ctypes.c_void_p(_ptr(h_keys)), ctypes.c_void_p(_ptr(h_vals)), int(n)))


def cq_results(q):
    """Returns (status, cq_result_view) with device pointers."""
    v = cq_result_view()
    st = load().cq_results(q, ctypes.byref(v))
    return st, v


def cq_results_copy(q, h_sum, h_count, h_min, h_max, h_avg) -> int:
    return int(load().cq_results_copy(q, *(ctypes.c_void_p(_ptr(a)) for a in (h_sum, h_count, h_min, h_max, h_avg))))


def cq_results_copy_async(q, h_sum, h_count, h_min, h_max, h_avg) -> int:
    return int(load().cq_results_copy_async(q, *(ctypes.c_void_p(_ptr(a)) for a in (h_sum, h_count, h_min, h_max,
                                                                                      h_avg))))


def cq_sync(q) -> int:
    return int(load().cq_sync(q))


def cq_destroy(q) -> None:
    load().cq_destroy(q)


def cq_set_option(q, opt: int, value: int) -> int:
    return int(load().cq_set_option(q, int(opt), int(value)))


def cq_get_option(q, opt: int):
    v = ctypes.c_int64()
    st = load().cq_get_option(q, int(opt), ctypes.byref(v))
    return st, v.value


def cq_trace(q, d_stamps, slots: int) -> int:
    return int(load().cq_trace(q, ctypes.c_void_p(_ptr(d_stamps)), int(slots)))


def cq_check_avg(n: int, seed: int):
    """(status, mismatches) of the library's AVG division against fp64 over n drawn pairs."""
    out = ctypes.c_int64(0)
    st = int(load().cq_check_avg(int(n), int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(out)))
    return st, int(out.value)


def cqg_create(stream: int = 0):
    """Returns (status, group handle)."""
    h = ctypes.c_void_p()
    st = load().cqg_create(ctypes.c_void_p(int(stream)), ctypes.byref(h))
    return st, h


def cqg_push(g, queries, d_keys, d_vals, n, status=None) -> int:
    """Push batch i to queries[i] for every i in one launch (lists of equal length)."""
    nq = len(queries)
    P = ctypes.c_void_p
    qa = (P * nq)(*[q.handle.value if hasattr(q, "handle") else q.value for q in queries])
    ka = (P * nq)(*[_ptr(x) for x in d_keys])
    va = (P * nq)(*[_ptr(x) for x in d_vals])
    na = (ctypes.c_int64 * nq)(*[int(x) for x in n])
    sa = (ctypes.c_int * nq)() if status is not None else None
    st = int(load().cqg_push(g, nq, qa, ka, va, na, sa))
    if status is not None:
        status[:] = list(sa)
    return st


def cqs_now_ns() -> int:
    return int(load().cqs_now_ns())


def cqs_create(budget_bytes: int, stream=0):
    h = ctypes.c_void_p()
    st = int(load().cqs_create(int(budget_bytes), ctypes.c_void_p(int(stream)), ctypes.byref(h)))
    return st, h


def cqs_admit(s, groups: int, window: int, aggs: int, max_batch: int):
    h = ctypes.c_void_p()
    st = int(load().cqs_admit(s, int(groups), int(window), int(aggs), int(max_batch), ctypes.byref(h)))
    return st, h


def cqs_submit(s, q, d_keys, d_vals, n: int, arrival_ns: int = -1):
    """Returns (status, ticket)."""
    t = ctypes.c_int64(-1)
    st = int(load().cqs_submit(s, q, ctypes.c_void_p(_ptr(d_keys)), ctypes.c_void_p(_ptr(d_vals)), int(n),
                               int(arrival_ns), ctypes.byref(t)))
    return st, t.value


def cqs_wait(s, ticket: int) -> int:
    return int(load().cqs_wait(s, int(ticket)))


def cqs_drain(s) -> int:
    return int(load().cqs_drain(s))


def cqs_replay(s, queries, arrival_ns, d_keys, d_vals, n) -> int:
    """Open-loop replay: batch i goes to queries[i] at arrival_ns[i] ns after the start."""
    nb = len(queries)
    P = ctypes.c_void_p
    qa = (P * nb)(*[q.value if isinstance(q, ctypes.c_void_p) else q for q in queries])
    aa = np.ascontiguousarray(arrival_ns, dtype=np.int64)
    ka = (P * nb)(*[_ptr(x) for x in d_keys])
    va = (P * nb)(*[_ptr(x) for x in d_vals])
    na = np.ascontiguousarray(n, dtype=np.int64)
    return int(load().cqs_replay(s, nb, qa, P(aa.ctypes.data), ka, va, P(na.ctypes.data)))


def cqs_stats(s):
    out = cqs_server_stats()
    st = int(load().cqs_stats(s, ctypes.byref(out)))
    return st, {f: getattr(out, f) for f, _ in cqs_server_stats._fields_}


def cqs_reset_stats(s) -> int:
    return int(load().cqs_reset_stats(s))


def cqs_destroy(s) -> None:
    load().cqs_destroy(s)


def cqg_stats(g):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    st = int(load().cqg_stats(g, ctypes.byref(a), ctypes.byref(b)))
    return st, a.value, b.value


def cq_autotune(q, d_keys, d_vals, n: int, trials: int = 3):
    """Returns (status, mean microseconds per push of the chosen settings)."""
    best = ctypes.c_double()
    st = int(load().cq_autotune(q, ctypes.c_void_p(_ptr(d_keys)), ctypes.c_void_p(_ptr(d_vals)), int(n), int(trials),
                                ctypes.byref(best)))
    return st, best.value


def cqg_sync(g) -> int:
    return int(load().cqg_sync(g))


def cqg_destroy(g) -> None:
    load().cqg_destroy(g)


def cq_stats(q):
    s = cq_query_stats()
    st = load().cq_stats(q, ctypes.byref(s))
    return st, {n: getattr(s, n) for n, _ in cq_query_stats._fields_}


def cq_hot_list(q, cap: int = 128):
    keys = (ctypes.c_int32 * max(cap, 1))()
    counts = (ctypes.c_int32 * max(cap, 1))()
    n = ctypes.c_int(0)
    st = load().cq_hot_list(q, keys, counts, cap, ctypes.byref(n))
    m = min(n.value, cap)
    return st, list(keys[:m]), list(counts[:m]), n.value


# ---- convenience wrapper -----------------------------------------------------

class Query:
    """One continuous query on the current CUDA device.

    ``stream``: a ``torch.cuda.Stream`` / raw ``cudaStream_t`` / None (the
    current torch stream when torch is importable, else a library stream).
    """

    def __init__(self, groups: int, window: int, aggs: int = CQ_ALL, stream=None, **options):
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        if stream == 0:
            # torch reports the legacy default stream as handle 0, which the C
            # ABI reads as "library-owned stream"; name the legacy stream
            # explicitly (cudaStreamLegacy) so pushes stay ordered with torch.
            stream = CUDA_STREAM_LEGACY
        st, h = cq_create(groups, window, aggs, stream)
        _check(st, "cq_create")
        self._h = h
        self.groups, self.window, self.aggs = int(groups), int(window), int(aggs)
        for name, value in options.items():
            self.set_option(name, value)

    _OPTS = {"hot_keys": CQ_OPT_HOT_KEYS, "hot_threshold": CQ_OPT_HOT_THRESHOLD, "warp_agg": CQ_OPT_WARP_AGG,
             "ctas_per_sm": CQ_OPT_CTAS_PER_SM, "partition_bits": CQ_OPT_PARTITION_BITS, "path": CQ_OPT_PATH,
             "wait_limit_us": CQ_OPT_WAIT_LIMIT_US, "stall_batch": CQ_OPT_STALL_BATCH,
             "stream_producers": CQ_OPT_STREAM_PRODUCERS}

    def set_option(self, name: str, value: int) -> None:
        _check(cq_set_option(self._h, self._OPTS[name], value), "cq_set_option(%s)" % name)

    def get_option(self, name: str) -> int:
        st, v = cq_get_option(self._h, self._OPTS[name])
        _check(st, "cq_get_option")
        return v

    @property
    def handle(self):
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None):
            cq_destroy(self._h)
            self._h = None

    __del__ = close

    def push(self, keys, vals) -> int:
        """Push a batch: CUDA tensors go through cq_push, host arrays through cq_push_host."""
        n = int(keys.numel() if hasattr(keys, "numel") else len(keys))
        on_device = hasattr(keys, "is_cuda") and keys.is_cuda
        if on_device:
            return cq_push(self._h, keys, vals, n)
        if hasattr(keys, "numpy"):
            keys, vals = keys.numpy(), vals.numpy()
        keys = np.ascontiguousarray(keys, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.int32)
        self._hold = (keys, vals)  # host arrays must live until the push completes
        return cq_push_host(self._h, keys, vals, n)

    def push_many(self, keys, vals, out=None) -> int:
        """Push a list of device batches (CUDA tensors) in one persistent
        launch (cq_push_many); ``out`` as for cq_push_many."""
        return cq_push_many(self._h, keys, vals, [int(k.numel()) for k in keys], out)

    def push_noalloc(self, keys, vals) -> int:
        """Push a device batch without allocating (cq_push_noalloc)."""
        return cq_push_noalloc(self._h, keys, vals, int(keys.numel()))

    def sync(self) -> int:
        return cq_sync(self._h)

    def results(self) -> dict:
        """Copy every group's SUM, COUNT, MIN, MAX, AVG to host numpy arrays."""
        G = self.groups
        out = dict(sum=np.empty(G, np.int64), count=np.empty(G, np.int32), min=np.empty(G, np.int32),
                   max=np.empty(G, np.int32), avg=np.empty(G, np.float64))
        _check(cq_results_copy(self._h, out["sum"], out["count"], out["min"], out["max"], out["avg"]),
               "cq_results_copy")
        return out

    def stats(self) -> dict:
        st, s = cq_stats(self._h)
        _check(st, "cq_stats")
        return s

    def hot_list(self):
        """(keys, insert counts) of the heavy hitters the next push privatises."""
        st, keys, counts, _ = cq_hot_list(self._h)
        _check(st, "cq_hot_list")
        return keys, counts

    def autotune(self, keys, vals, trials: int = 3) -> float:
        """Pick the fastest tuning settings for batches like (keys, vals)."""
        st, us = cq_autotune(self._h, keys, vals, int(keys.numel()), trials)
        _check(st, "cq_autotune")
        return us


class Group:
    """Pushes one batch to each of several queries in one launch."""

    def __init__(self, stream=None):
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        if stream == 0:
            stream = CUDA_STREAM_LEGACY
        st, h = cqg_create(stream)
        _check(st, "cqg_create")
        self._h = h

    def push(self, queries, keys, vals, status=None) -> int:
        n = [int(k.numel() if hasattr(k, "numel") else len(k)) for k in keys]
        return cqg_push(self._h, queries, keys, vals, n, status)

    def sync(self) -> int:
        return cqg_sync(self._h)

    def stats(self):
        st, launches, graphs = cqg_stats(self._h)
        _check(st, "cqg_stats")
        return {"launches": launches, "graph_launches": graphs}

    def close(self) -> None:
        if getattr(self, "_h", None):
            cqg_destroy(self._h)
            self._h = None

    __del__ = close


class ServedQuery(Query):
    """A query admitted to a Server: the server owns and destroys it."""

    def __init__(self, handle, groups: int, window: int, aggs: int):
        self._h = handle
        self.groups, self.window, self.aggs = int(groups), int(window), int(aggs)

    def close(self) -> None:
        self._h = None

    __del__ = close


class Server:
    """The serving loop: standing queries admitted against a device-memory
    budget, batches submitted over time and pushed by continuous batching."""

    def __init__(self, budget_bytes: int, stream=None):
        if hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        st, h = cqs_create(budget_bytes, stream or 0)
        _check(st, "cqs_create")
        self._h = h
        self.queries = []

    def admit(self, groups: int, window: int, aggs: int = CQ_ALL, max_batch: int = 1 << 20) -> "ServedQuery":
        st, h = cqs_admit(self._h, groups, window, aggs, max_batch)
        _check(st, "cqs_admit")
        q = ServedQuery(h, groups, window, aggs)
        self.queries.append(q)
        return q

    def submit(self, q, keys, vals, arrival_ns: int = -1) -> int:
        st, t = cqs_submit(self._h, q.handle, keys, vals, int(keys.numel()), arrival_ns)
        _check(st, "cqs_submit")
        return t

    def wait(self, ticket: int) -> int:
        return cqs_wait(self._h, ticket)

    def drain(self) -> int:
        return cqs_drain(self._h)

    def replay(self, queries, arrival_ns, keys, vals) -> int:
        return cqs_replay(self._h, [q.handle for q in queries], arrival_ns, keys, vals,
                          [int(k.numel()) for k in keys])

    def stats(self) -> dict:
        st, d = cqs_stats(self._h)
        _check(st, "cqs_stats")
        return d

    def reset_stats(self) -> int:
        return cqs_reset_stats(self._h)

    def close(self) -> None:
        if getattr(self, "_h", None):
            for q in self.queries:
                q.close()
            cqs_destroy(self._h)
            self._h = None

    __del__ = close


class GroupWindows:
    """The paper's own aggregate: one window of ``window`` values per group;
    every pushed tuple's output is its group's window SUM right after it
    entered (recomputed from scratch ``passes`` times)."""

    def __init__(self, groups: int, window: int, passes: int = 1, stream=None):
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        if stream == 0:
            stream = CUDA_STREAM_LEGACY
        h = ctypes.c_void_p()
        _check(int(load().cqw_create(int(groups), int(window), int(passes), ctypes.c_void_p(stream),
                                     ctypes.byref(h))), "cqw_create")
        self._h = h
        self.groups, self.window, self.passes = int(groups), int(window), int(passes)

    def push(self, keys, vals, sums) -> int:
        """keys, vals: device int32 tensors; sums: device int64 tensor of the same length."""
        return int(load().cqw_push(self._h, ctypes.c_void_p(_ptr(keys)), ctypes.c_void_p(_ptr(vals)),
                                   int(keys.numel()), ctypes.c_void_p(_ptr(sums))))

    def sync(self) -> int:
        return int(load().cqw_sync(self._h))

    def stats(self) -> dict:
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(int(load().cqw_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))), "cqw_stats")
        return {"tuples_seen": a.value, "pushes": b.value, "kernel_launches": c.value}

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().cqw_destroy(self._h)
            self._h = None

    __del__ = close


def _csr(mapping):
    """Thread-to-groups lists -> (off, groups) int32 arrays."""
    import numpy as np
    off = np.zeros(len(mapping) + 1, np.int32)
    for t, groups in enumerate(mapping):
        off[t + 1] = off[t] + len(groups)
    flat = np.array([g for groups in mapping for g in groups], np.int32)
    return off, flat


def cqo_rebalance(policy: str, mapping, keys, threshold: int = 1000, pot: float = 0.5):
    """One policy step on the host (no device): returns (new mapping, moves)."""
    import numpy as np
    off, flat = _csr(mapping)
    keys = np.ascontiguousarray(keys, np.int32)
    out_off = np.zeros_like(off)
    out_groups = np.zeros_like(flat)
    moves = ctypes.c_int64()
    st = int(load().cqo_rebalance(CQO_POLICIES.index(policy), len(mapping), int(flat.size), off.ctypes.data,
                                  flat.ctypes.data, keys.ctypes.data, int(keys.size), int(threshold), float(pot),
                                  out_off.ctypes.data, out_groups.ctypes.data, ctypes.byref(moves)))
    _check(st, "cqo_rebalance")
    return [out_groups[out_off[t]:out_off[t + 1]].tolist() for t in range(len(mapping))], moves.value


class OwnerWindows:
    """The paper's owner-computes execution of the per-group windows: owner
    threads (256 per block, ``grid`` blocks) process their groups' tuples in
    order; the host lays batches out and rebalances with ``policy`` (one of
    CQO_POLICIES), or, with ``device=True``, the GPU does both (one of
    CQO_DEVICE_POLICIES).  Outputs as GroupWindows; tuples come from host
    memory."""

    def __init__(self, groups: int, window: int, passes: int = 1, grid: int = 4, policy: str = "probCheck",
                 threshold: int = 1000, pot: float = 0.5, stream=None, device: bool = False):
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        if stream == 0:
            stream = CUDA_STREAM_LEGACY
        h = ctypes.c_void_p()
        code = CQO_POLICIES.index(policy) | (CQO_ON_DEVICE if device else 0)
        _check(int(load().cqo_create(int(groups), int(window), int(passes), int(grid), code, int(threshold),
                                     float(pot), ctypes.c_void_p(stream), ctypes.byref(h))), "cqo_create")
        self._h = h
        self.groups, self.window, self.passes, self.grid, self.policy = int(groups), int(window), int(passes), \
            int(grid), policy
        self.device = bool(device)
        self.threads = 256 * int(grid)

    def push(self, keys, vals, sums) -> int:
        """keys, vals: host int32 numpy arrays; sums: device int64 tensor of the same length."""
        import numpy as np
        keys = np.ascontiguousarray(keys, np.int32)
        vals = np.ascontiguousarray(vals, np.int32)
        return int(load().cqo_push(self._h, keys.ctypes.data, vals.ctypes.data, int(keys.size),
                                   ctypes.c_void_p(_ptr(sums))))

    def sync(self) -> int:
        return int(load().cqo_sync(self._h))

    def stats(self) -> dict:
        s = cqo_stats_t()
        _check(int(load().cqo_stats(self._h, ctypes.byref(s))), "cqo_stats")
        return {n: getattr(s, n) for n, _ in cqo_stats_t._fields_}

    def mapping(self):
        import numpy as np
        off = np.zeros(self.threads + 1, np.int32)
        groups = np.zeros(self.groups, np.int32)
        _check(int(load().cqo_mapping(self._h, off.ctypes.data, groups.ctypes.data)), "cqo_mapping")
        return [groups[off[t]:off[t + 1]].tolist() for t in range(self.threads)]

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().cqo_destroy(self._h)
            self._h = None

    __del__ = close
