"""Tile autotuner of the batched GEMMs: tuned solves equal untuned ones, the
table covers the sweep's shape classes, and a tuned class is never slower
than the fixed rule it replaces (up to timing noise)."""
import numpy as np
import pytest

import workloads
from gpu_util import fdslib, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_autotuned_solve_equals_fixed_rule(precision):
    torch_cuda()
    fds = fdslib()
    xy = workloads.star(4096, 0.2, 5, rot=0.1)
    omega = workloads.omega_for_kTa(10.0)
    kinds, ang = workloads.plane_wave_set(3)
    fds.fds_autotune_enable(False)
    h = fds.fds_build(xy, omega, 2.0, 1.0, 1e-9, precision=precision)
    F = fds.fds_rhs_plane_wave(h, kinds, ang)
    x0 = fds.fds_solve(h, F)
    h.close()
    fds.fds_autotune_reset()
    fds.fds_autotune_enable(True)
    try:
        h = fds.fds_build(xy, omega, 2.0, 1.0, 1e-9, precision=precision)
        x1 = fds.fds_solve(h, F)     # tunes the classes it meets
        x2 = fds.fds_solve(h, F)     # runs on the table
        h.close()
        rep = fds.fds_autotune_report()
    finally:
        fds.fds_autotune_enable(False)
    assert len(rep) >= 3
    arith = {"c128"} if precision == 0 else {"c64", "ff"}
    assert arith <= {r["arith"] for r in rep} | {"c128"}
    for r in rep:
        assert r["best_us"] <= 1.2 * r["rule_us"] + 2.0, r
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    # same K order in every tile shape: the FP64 solutions agree to rounding;
    # the refined mixed ones to the refinement's accuracy (its residual norms
    # and the forward operator's sums use atomics, so the iterates differ at
    # rounding level from run to run)
    tol = 1e-12 if precision == 0 else 1e-10
    assert rel(x1, x0) <= tol
    assert rel(x2, x0) <= tol
