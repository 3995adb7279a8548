"""Seeded synthetic tuple streams shared by the oracle and the CUDA path.

The module turns (seed, stream index) into (group id, int32 value) tuples and
nothing else: it holds none of the windowed aggregation arithmetic.  The C
source (``streamgen.c``) is compiled on first use with the host C compiler.

The stream shapes follow the paper's datasets (Section 5.1): uniform or
round-robin group ids (DS1), Zipf with the most frequent groups at the
smallest ids (DS2) and a randomly permuted Zipf (DS3), here with an optional
re-draw of the permutation every ``repermute_every`` tuples so the heavy
hitters move.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "streamgen.c")
_LIB = os.path.join(_HERE, "libstreamgen.so")
_lock = threading.Lock()
_lib = None

KEY_UNIFORM, KEY_ZIPF, KEY_ROUND_ROBIN = 0, 1, 2
VAL_UNIFORM, VAL_NORMAL, VAL_INDEX = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile ``libstreamgen.so`` next to its source (host C compiler)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            c = ctypes
            lib.sg_splitmix64_at.restype = c.c_uint64
            lib.sg_splitmix64_at.argtypes = [c.c_uint64, c.c_uint64]
            lib.sg_unit_double.restype = c.c_double
            lib.sg_unit_double.argtypes = [c.c_uint64, c.c_uint64]
            lib.sg_log_uniform_int.restype = c.c_int64
            lib.sg_log_uniform_int.argtypes = [c.c_uint64, c.c_uint64, c.c_int64, c.c_int64]
            lib.sg_create.restype = c.c_void_p
            lib.sg_create.argtypes = [c.c_int64, c.c_int, c.c_double, c.c_int, c.c_int64, c.c_int,
                                      c.c_double, c.c_double, c.c_int64, c.c_int64, c.c_uint64]
            lib.sg_destroy.restype = None
            lib.sg_destroy.argtypes = [c.c_void_p]
            lib.sg_fill.restype = None
            lib.sg_fill.argtypes = [c.c_void_p, c.c_int64, c.c_int64, c.c_void_p, c.c_void_p]
            lib.sg_zipf_pmf.restype = c.c_double
            lib.sg_zipf_pmf.argtypes = [c.c_void_p, c.c_int64]
            lib.sg_key_of_rank.restype = c.c_int32
            lib.sg_key_of_rank.argtypes = [c.c_void_p, c.c_int64, c.c_int64]
            _lib = lib
    return _lib


def splitmix64(seed: int, i: int) -> int:
    """Output number ``i`` (0-based) of SplitMix64 seeded with ``seed``."""
    return int(_load().sg_splitmix64_at(seed & (2**64 - 1), i))


def unit_double(seed: int, i: int) -> float:
    """Uniform double in [0, 1) from draw ``i`` of stream ``seed``."""
    return float(_load().sg_unit_double(seed & (2**64 - 1), i))


def log_uniform_int(seed: int, i: int, lo: int, hi: int) -> int:
    """round(exp(U(ln lo, ln hi))) from draw ``i`` of stream ``seed``."""
    return int(_load().sg_log_uniform_int(seed & (2**64 - 1), i, lo, hi))


class Stream:
    """A deterministic, randomly addressable stream of (key, value) tuples.

    keys: "uniform" | "zipf" | "round_robin"; vals: "uniform" | "normal" | "index".
    ``fill(t0, n)`` returns tuples t0 .. t0+n-1; any split of a range into
    sub-ranges yields the same tuples.
    """

    def __init__(self, groups: int, keys: str = "uniform", s: float = 0.0, permute: bool = True,
                 repermute_every: int = 0, vals: str = "uniform", lo: int = 0, hi: int = 10**6,
                 mean: float = 5e5, sd: float = 1e5, seed: int = 1):
        self.groups = int(groups)
        self.spec = dict(groups=groups, keys=keys, s=s, permute=permute, repermute_every=repermute_every,
                         vals=vals, lo=lo, hi=hi, mean=mean, sd=sd, seed=seed)
        kd = {"uniform": KEY_UNIFORM, "zipf": KEY_ZIPF, "round_robin": KEY_ROUND_ROBIN}[keys]
        vd = {"uniform": VAL_UNIFORM, "normal": VAL_NORMAL, "index": VAL_INDEX}[vals]
        self._lib = _load()
        self._h = self._lib.sg_create(int(groups), kd, float(s), int(bool(permute)), int(repermute_every),
                                      vd, float(mean), float(sd), int(lo), int(hi), seed & (2**64 - 1))
        if not self._h:
            raise ValueError("invalid stream parameters: %r" % (self.spec,))
        self._mu = threading.Lock()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.sg_destroy(h)
            self._h = None

    def fill_into(self, t0: int, n: int, keys_ptr: int, vals_ptr: int) -> None:
        """Write tuples t0 .. t0+n-1 to raw host pointers (int32 arrays)."""
        with self._mu:
            self._lib.sg_fill(self._h, int(t0), int(n), ctypes.c_void_p(keys_ptr), ctypes.c_void_p(vals_ptr))

    def fill(self, t0: int, n: int):
        keys = np.empty(int(n), dtype=np.int32)
        vals = np.empty(int(n), dtype=np.int32)
        if n:
            self.fill_into(t0, n, keys.ctypes.data, vals.ctypes.data)
        return keys, vals

    def zipf_pmf(self):
        """Probability of each rank under the Zipf table (rank 1 first)."""
        return np.array([self._lib.sg_zipf_pmf(self._h, r) for r in range(self.groups)])

    def key_of_rank(self, t: int, r: int) -> int:
        with self._mu:
            return int(self._lib.sg_key_of_rank(self._h, int(t), int(r)))
