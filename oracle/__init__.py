"""CPU oracle for the windowed group-by aggregate.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_1309_0634_b300``) never imports, links or runs it, and it shares no
code with that path.

``oracle.c`` is the plain definition of the query (Section 3 of the paper: a
group-by over (id, attr) tuples aggregating a fixed-size sliding window,
processed in iterations of batches, Section 3.1).  ``oracle_pgw.c`` follows
the paper's own workload step by step: one window of w values per group, the
window's SUM recomputed from scratch after every tuple (Sections 3.2, 5.1).
Both are compiled with the host C compiler on first use.  Every function
below only marshals arguments.

Pinned by ``tests/test_oracle_pins.py`` against closed forms, numpy reductions,
CPython's IEEE arithmetic, invariants and a brute force over the full stream
history; no part of it is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = (os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "oracle_pgw.c"))
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, EKEY, EPOISONED = 0, 1, 2, 3, 7
NAN_BITS = 0x7FF8000000000000


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` (plain C, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(p) for p in _SRCS):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", *_SRCS, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            c = ctypes
            P = c.c_void_p
            lib.oq_create.restype = c.c_int
            lib.oq_create.argtypes = [c.c_int64, c.c_int64, c.POINTER(c.c_void_p)]
            lib.oq_destroy.restype = None
            lib.oq_destroy.argtypes = [P]
            lib.oq_seen.restype = c.c_int64
            lib.oq_seen.argtypes = [P]
            lib.oq_push.restype = c.c_int
            lib.oq_push.argtypes = [P, P, P, c.c_int64]
            lib.oq_results.restype = c.c_int
            lib.oq_results.argtypes = [P, P, P, P, P, P]
            lib.oq_group.restype = c.c_int
            lib.oq_group.argtypes = [P, c.c_int64, P, P, P, P, P]
            lib.ow_create.restype = c.c_int
            lib.ow_create.argtypes = [c.c_int64, c.c_int32, c.c_int32, c.POINTER(c.c_void_p)]
            lib.ow_destroy.restype = None
            lib.ow_destroy.argtypes = [P]
            lib.ow_seen.restype = c.c_int64
            lib.ow_seen.argtypes = [P]
            lib.ow_push.restype = c.c_int
            lib.ow_push.argtypes = [P, P, P, c.c_int64, P]
            lib.ow_group_sum.restype = c.c_int
            lib.ow_group_sum.argtypes = [P, c.c_int64, P, P]
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s failed with status %d" % (what, status))
        self.status = status


class Oracle:
    """One continuous query: ``push`` batches, read ``results`` after any push."""

    def __init__(self, groups: int, window: int):
        self._lib = _load()
        h = ctypes.c_void_p()
        st = self._lib.oq_create(int(groups), int(window), ctypes.byref(h))
        if st != OK:
            raise OracleError(st, "oq_create")
        self._h = h
        self.groups = int(groups)
        self.window = int(window)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oq_destroy(h)
            self._h = None

    @property
    def seen(self) -> int:
        return int(self._lib.oq_seen(self._h))

    def push(self, keys, vals) -> int:
        """Append a batch; returns the status code (0 on success)."""
        keys = np.ascontiguousarray(keys, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.int32)
        if keys.shape != vals.shape:
            raise ValueError("keys and vals differ in length")
        return int(self._lib.oq_push(self._h, keys.ctypes.data, vals.ctypes.data, keys.size))

    def push_ptr(self, keys_ptr: int, vals_ptr: int, n: int) -> int:
        return int(self._lib.oq_push(self._h, ctypes.c_void_p(keys_ptr), ctypes.c_void_p(vals_ptr), int(n)))

    def results(self) -> dict:
        """SUM, COUNT, MIN, MAX, AVG of every group over the current window."""
        G = self.groups
        out = dict(sum=np.empty(G, np.int64), count=np.empty(G, np.int32), min=np.empty(G, np.int32),
                   max=np.empty(G, np.int32), avg=np.empty(G, np.float64))
        st = self._lib.oq_results(self._h, out["sum"].ctypes.data, out["count"].ctypes.data,
                                  out["min"].ctypes.data, out["max"].ctypes.data, out["avg"].ctypes.data)
        if st != OK:
            raise OracleError(st, "oq_results")
        return out

    def group(self, g: int) -> tuple:
        """(sum, count, min, max, avg) of one group, from scratch."""
        s = ctypes.c_int64()
        c = ctypes.c_int32()
        lo = ctypes.c_int32()
        hi = ctypes.c_int32()
        a = ctypes.c_double()
        st = self._lib.oq_group(self._h, int(g), ctypes.addressof(s), ctypes.addressof(c), ctypes.addressof(lo),
                                ctypes.addressof(hi), ctypes.addressof(a))
        if st != OK:
            raise OracleError(st, "oq_group")
        return s.value, c.value, lo.value, hi.value, a.value


class WindowsOracle:
    """The paper's own aggregate: one window of ``window`` values per group;
    ``push`` returns, for every tuple, its group's window SUM right after the
    tuple is inserted (recomputed from scratch ``passes`` times)."""

    def __init__(self, groups: int, window: int, passes: int = 1):
        self._lib = _load()
        h = ctypes.c_void_p()
        st = self._lib.ow_create(int(groups), int(window), int(passes), ctypes.byref(h))
        if st != OK:
            raise OracleError(st, "ow_create")
        self._h = h
        self.groups, self.window, self.passes = int(groups), int(window), int(passes)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.ow_destroy(h)
            self._h = None

    @property
    def seen(self) -> int:
        return int(self._lib.ow_seen(self._h))

    def push(self, keys, vals):
        """Returns (status, per-tuple window sums as int64)."""
        keys = np.ascontiguousarray(keys, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.int32)
        if keys.shape != vals.shape:
            raise ValueError("keys and vals differ in length")
        out = np.zeros(keys.size, np.int64)
        st = int(self._lib.ow_push(self._h, keys.ctypes.data, vals.ctypes.data, keys.size, out.ctypes.data))
        return st, out

    def group_sum(self, g: int) -> tuple:
        """(window sum, values in the window) of group g."""
        s = ctypes.c_int64()
        c = ctypes.c_int32()
        st = self._lib.ow_group_sum(self._h, int(g), ctypes.addressof(s), ctypes.addressof(c))
        if st != OK:
            raise OracleError(st, "ow_group_sum")
        return s.value, c.value
