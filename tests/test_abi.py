"""The C-ABI library loads and exports every function include/cq.h declares.

Runs without a GPU: only calls that need no CUDA device are made.
"""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1309_0634_b300 as cq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cq.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"CQ_API\s+[\w\s\*]+?\b(cq[gswo]?_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1309_0634_b300 import _build
    _build.build()
    return cq.load()


def test_header_declares_the_abi():
    names = declared_functions()
    assert set(names) == set(cq.EXPORTS), names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.check_output(["nm", "-D", "--defined-only", cq.LIB_PATH]).decode()
    exported = set(re.findall(r"\bT (cq[gswo]?_\w+)", out))
    assert set(declared_functions()) <= exported
    # nothing else leaks out of the library under a cq_ name
    assert exported == set(declared_functions())


def test_build_targets_sm_103a_only():
    from paper_1309_0634_b300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_strerror_and_footprint_need_no_device(lib):
    assert cq.cq_strerror(cq.CQ_OK) == "ok"
    assert "poisoned" in cq.cq_strerror(cq.CQ_EPOISONED)
    assert cq.cq_strerror(99) == "unknown status"
    assert cq.cq_footprint_bytes(0, 10) == -1
    assert cq.cq_footprint_bytes(10, 2**31) == -1
    small = cq.cq_footprint_bytes(1000, 10_000, cq.CQ_SUM | cq.CQ_COUNT)
    full = cq.cq_footprint_bytes(1000, 10_000, cq.CQ_ALL)
    assert 0 < small < full
    # the ring (8 B per window slot) and per-group state dominate
    assert small >= 8 * 10_000 + 28 * 1000


def test_group_and_window_limits_need_no_device(lib):
    """Groups run to 2^30 - 2 (the key 2^30 - 1 pads a run of deltas and the
    bits above carry the retract and front-departure flags); arguments are
    checked before any device call."""
    assert cq.cq_footprint_bytes(2**30 - 2, 10, cq.CQ_SUM) > 0
    assert cq.cq_footprint_bytes(2**30 - 1, 10, cq.CQ_SUM) == -1
    for groups, window, aggs in [(0, 10, cq.CQ_ALL), (2**30 - 1, 10, cq.CQ_ALL), (2**31, 10, cq.CQ_ALL),
                                 (10, 0, cq.CQ_ALL), (10, 2**31, cq.CQ_ALL), (10, 10, 0), (10, 10, 1 << 9)]:
        st, h = cq.cq_create(groups, window, aggs)
        assert st == cq.CQ_EINVAL, (groups, window, aggs)
        assert not h.value
    assert cq.cq_check_avg(-1, 0)[0] == cq.CQ_EINVAL
    assert cq.cq_check_avg(0, 0) == (cq.CQ_OK, 0)


def test_binding_fails_loudly_without_library(tmp_path):
    saved = cq._lib
    try:
        cq._lib = None
        with pytest.raises(RuntimeError, match="libcq.so is missing"):
            cq.load(str(tmp_path / "nope.so"))
    finally:
        cq._lib = saved


def test_null_handle_is_rejected(lib):
    assert lib.cq_push(None, None, None, 1) == cq.CQ_EINVAL
    assert lib.cq_sync(None) == cq.CQ_EINVAL
    st, v = cq.cq_get_option(None, cq.CQ_OPT_PARTITION_BITS)
    assert st == cq.CQ_EINVAL
