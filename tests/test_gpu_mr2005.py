"""The Woodbury form of the original Martinsson–Rokhlin elimination
(FDS_VARIANT_MR2005), the method the paper's LU-based variant is compared
with (Sec. 6 introduction): the same compressed system solved through
E_i, F_i, G_i, so its solution equals the LU variant's to rounding; and the
matrix-matrix products it adds to the build (the paper's claim)."""
import numpy as np
import pytest

import workloads
from gpu_util import fdslib, torch_cuda
from oracle import bem

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("l0", [0, 1, 2])
def test_mr2005_exact_without_truncation(l0):
    torch_cuda()
    fds = fdslib()
    xy = workloads.star(256)
    P = bem.phys(2.0, 1.0, 1.0, 3.0)
    F = np.stack([bem.rhs(P, xy, 0, 0.3), bem.rhs(P, xy, 1, 1.9)], 1)
    xd = np.linalg.solve(bem.dense_matrix(P, xy), F)
    h = fds.fds_build(xy, 3.0, 2.0, 1.0, 0.0, leaf_size=32, top_level=l0, variant=fds.FDS_VARIANT_MR2005)
    assert _rel(fds.fds_solve(h, F), xd) < 1e-11
    h.close()


def test_mr2005_equals_lu_variant_and_dense():
    torch_cuda()
    fds = fdslib()
    xy = workloads.star(2048, 0.2, 5, rot=0.3)
    omega = workloads.omega_for_kTa(12.0)
    eps = 1e-9
    P = bem.phys(2.0, 1.0, 1.0, omega)
    kinds, ang = workloads.plane_wave_set(3)
    fds.fds_timing_reset()
    fds.fds_timing_enable(True)
    try:
        hl = fds.fds_build(xy, omega, 2.0, 1.0, eps, leaf_size=32)
        rep_lu = fds.fds_timing_report()
        fds.fds_timing_reset()
        hm = fds.fds_build(xy, omega, 2.0, 1.0, eps, leaf_size=32, variant=fds.FDS_VARIANT_MR2005)
        rep_mr = fds.fds_timing_report()
    finally:
        fds.fds_timing_enable(False)
    F = fds.fds_rhs_plane_wave(hl, kinds, ang)
    xl = fds.fds_solve(hl, F)
    xm = fds.fds_solve(hm, F)
    # same skeletons and compressed system: equal to rounding
    assert _rel(xm, xl) < 1e-10
    xd = np.linalg.solve(bem.dense_matrix(P, xy), F)
    assert _rel(xm, xd) <= 10 * eps
    # the Woodbury form adds E = W A~, V A^{-1}, F = A~ V A^{-1}, G = A^{-1} - E V A^{-1}
    merge = lambda r: sum(v["flops"] for k, v in r.items() if k.startswith("a3."))
    assert "a3.mr2005_products" in rep_mr and "a3.mr2005_products" not in rep_lu
    assert merge(rep_mr) > 1.3 * merge(rep_lu)
    for h in (hl, hm):
        h.close()


def test_mr2005_rejected_with_mixed_precision():
    torch_cuda()
    fds = fdslib()
    with pytest.raises(fds.FdsError) as e:
        fds.fds_build(workloads.star(256), 3.0, 2.0, 1.0, 1e-8, leaf_size=32, precision=fds.FDS_MIXED,
                      variant=fds.FDS_VARIANT_MR2005)
    assert e.value.code == fds.FDS_ERR_ARG
