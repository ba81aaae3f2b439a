"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/wn.h declares; argument validation that happens before any CUDA call
returns the documented status codes (CPU only, no compute calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def wnlib():
    from paper_2510_25159_gb300 import build as b
    b.build()
    import paper_2510_25159_gb300 as wn
    return wn


def declared_functions():
    src = open(os.path.join(ROOT, "include", "wn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wn_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared_functions()
    for f in ["wn_create_domain", "wn_destroy_domain", "wn_query", "wn_query_batched",
              "wn_query_grid_bitmask", "wn_last_error"]:
        assert f in names


def test_exports_every_declared_symbol(wnlib):
    L = ctypes.CDLL(wnlib.library_path())
    missing = [f for f in declared_functions() if not hasattr(L, f)]
    assert not missing, missing


def test_library_is_sm103a(wnlib):
    from paper_2510_25159_gb300 import build as b
    assert "arch=compute_103a,code=sm_103a" in " ".join(b.ARCH)


def test_validation_codes_without_gpu(wnlib):
    L = wnlib.lib()
    h = ctypes.c_void_p()
    lo = np.array([0, 1], dtype=np.int32)
    bad = np.array([0], dtype=np.int32)
    cp = np.zeros(2, dtype=np.float64)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert L.wn_create_domain(P(lo), 1, P(bad), P(cp), 0.0, 0.0, 0.0, ctypes.byref(h)) == 1
    assert b"degree" in L.wn_last_error()
    assert L.wn_create_domain(P(lo), 1, P(np.array([2], np.int32)), P(np.zeros(6)), -1.0, 0.0, 0.0,
                              ctypes.byref(h)) == 1
    assert L.wn_create_domain(P(lo), 1, P(np.array([1], np.int32)), P(np.array([0.0, 0, np.nan, 1])),
                              0.0, 0.0, 0.0, ctypes.byref(h)) == 1
    wneg = np.array([1.0, -2.0, 1.0])
    assert L.wn_create_domain_rational(P(lo), 1, P(np.array([2], np.int32)), P(np.zeros(6)), P(wneg), 0.0, 0.0,
                                       0.0, ctypes.byref(h)) == 1
    assert b"weights" in L.wn_last_error()
    assert L.wn_set_tuning(3, 0, 0, -1, -1, -1) == 1
    assert L.wn_set_near_tuning(5, 0, 0) == 1 and L.wn_set_near_tuning(31, 0, 0) == 1
    assert L.wn_set_near_tuning(0, 33, 0) == 1 and L.wn_set_near_tuning(0, 0, 40) == 1
    assert L.wn_set_queue_limits(-1, 0) == 1
    assert L.wn_set_flat_records(-1) == 1 and L.wn_set_flat_records(5000) == 1
    assert L.wn_set_grid_tile(12) == 1
    assert L.wn_get_tuning(None, 3) == 1
    assert L.wn_last_escalated(None, 0, None) == 1
    assert L.wn_eval_gap_angle(None, None, None, -1, None) == 1
    assert L.wn_near_work(None) == 1
    assert L.wn_sweep_work(None, 12) == 1
    assert L.wn_grid_triangles(None, 4, 4, 0, 0, None, 0, None, None) == 1
    assert L.wn_query_midpoints(None, None, 3, None, 1, None) == 1
    assert L.wn_query_surfaces(None, None, 1, None, None, None, 1, None) == 1
    assert L.wn_query(None, None, 0, None, None, 1, None) == 1
    assert L.wn_query_grid_bitmask(None, 4, 4, None, None, 1, None) == 1


def test_no_cpu_fallback_in_product():
    """The package never imports the oracle and has no host compute path."""
    pkg = os.path.join(ROOT, "paper_2510_25159_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "wn_oracle" not in text, f
