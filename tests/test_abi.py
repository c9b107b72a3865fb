"""The C ABI library loads and exports every function include/fds.h declares;
argument validation happens before any device work (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fds.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fds_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def fds():
    from paper_2411_18026_gb300 import build
    build.build()
    from paper_2411_18026_gb300 import fds as f
    f.lib()
    return f


def test_exports_every_declared_symbol(fds):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(fds.lib(), n), n


def test_argument_errors_without_gpu(fds):
    L = fds.lib()
    xy = np.zeros((4, 2))
    g = fds.fds_geometry(4, xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1.0)
    out = ctypes.c_void_p()
    assert L.fds_build(ctypes.byref(g), 1.0, 2.0, 1.0, 1e-8, ctypes.byref(out)) == fds.FDS_ERR_ARG   # n < 8
    xy = np.stack([np.cos(np.arange(16)), np.sin(np.arange(16))], 1).copy()
    g = fds.fds_geometry(16, xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1.0)
    assert L.fds_build(ctypes.byref(g), -1.0, 2.0, 1.0, 1e-8, ctypes.byref(out)) == fds.FDS_ERR_ARG  # omega
    assert L.fds_build(ctypes.byref(g), 1.0, 2.0, 0.0, 1e-8, ctypes.byref(out)) == fds.FDS_ERR_ARG   # mu
    assert L.fds_build(ctypes.byref(g), 1.0, 2.0, 1.0, 1.5, ctypes.byref(out)) == fds.FDS_ERR_ARG    # tol
    assert L.fds_build(ctypes.byref(g), 1.0, 2.0, 1.0, 1e-8, None) == fds.FDS_ERR_ARG
    xy[3, 0] = np.nan
    assert L.fds_build(ctypes.byref(g), 1.0, 2.0, 1.0, 1e-8, ctypes.byref(out)) == fds.FDS_ERR_ARG
    assert L.fds_solve(None, None, 1) == fds.FDS_ERR_ARG
    assert L.fds_id_batched(-1, None, None, None, None, 0.1, None, None, None, None, None, 0) == fds.FDS_ERR_ARG
    assert L.fds_lu_batched(0, None, None, None, None, None, None, 0) == fds.FDS_OK
    L.fds_destroy(None)
    assert fds.lib().fds_error_string(-4) == b"singular or non-finite pivot"


def test_fault_injection_arming_without_gpu(fds):
    # host-side faults arm and disarm without touching the device
    L = fds.lib()
    assert L.fds_fault_inject(fds.FDS_FAULT_ALLOC, 0) == fds.FDS_ERR_ARG
    assert L.fds_fault_inject(99, 0) == fds.FDS_ERR_ARG
    assert L.fds_fault_inject(fds.FDS_FAULT_ALLOC, 3) == fds.FDS_OK
    assert L.fds_fault_inject(fds.FDS_FAULT_NAN_BLOCK, 0) == fds.FDS_OK
    assert L.fds_fault_inject(fds.FDS_FAULT_NONE, 0) == fds.FDS_OK


def test_default_library_has_no_bounds_checks(fds):
    import ctypes as C
    n = C.c_int64(-1)
    assert fds.lib().fds_bounds_violations(C.byref(n)) == fds.FDS_ERR_STATE


def test_stage_entries_argument_checks_without_gpu(fds):
    # empty batches return before any device work; the bindings' argument lists match
    L = fds.lib()
    assert L.fds_zgemm_jobs_tc(0, *([None] * 11), None, None, 1, None, 1, 0, 0) == fds.FDS_OK
    assert L.fds_zgemm_jobs_tc(-1, *([None] * 11), None, None, 1, None, 1, 0, 0) == fds.FDS_ERR_ARG
    assert L.fds_zgemm_blocks_tc(0, None, None, None, None, 0, 0) == fds.FDS_OK
