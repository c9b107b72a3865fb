"""The formulation without the Burton–Miller term on the GPU (Sec. 8.4, eq.
(bie_non_bie): alpha = 0, f = int psi u^I): parity with the oracle's dense
non-BM solve, and the wave intensity |u_1|^2 + |u_2|^2 at x = (1, 0)
(Fig. wave_intensity) near a fictitious frequency of the unit circle, where
only the non-BM solution spikes."""
import numpy as np
import pytest

import disk_modes
import workloads
from gpu_util import fdslib, torch_cuda
from oracle import bem, paomow

pytestmark = pytest.mark.gpu

LAM, MU, RHO = 2.0, 1.0, 1.0


def test_non_bm_matches_oracle_dense_non_bm():
    torch_cuda()
    fds = fdslib()
    xy = workloads.star(1024)
    omega, eps = 2.5, 1e-10
    P = bem.phys(LAM, MU, RHO, omega, alpha=0.0)
    F = np.stack([bem.rhs(P, xy, 0, 0.3), bem.rhs(P, xy, 1, 1.9)], 1)
    xd = np.linalg.solve(bem.dense_matrix(P, xy), F)
    h = fds.fds_build(xy, omega, LAM, MU, eps, leaf_size=32, alpha=0.0)
    # the library's own load vectors of the non-BM system equal the oracle's
    Fg = fds.fds_rhs_plane_wave(h, np.array([0, 1], np.int32), np.array([0.3, 1.9]))
    assert np.linalg.norm(Fg - F) <= 1e-13 * np.linalg.norm(F)
    x = fds.fds_solve(h, F)
    h.close()
    err = np.linalg.norm(x - xd, axis=0) / np.linalg.norm(xd, axis=0)
    assert err.max() <= 10 * eps, err


def test_wave_intensity_spikes_only_without_burton_miller():
    torch_cuda()
    fds = fdslib()
    N = 128
    xy = workloads.circle(N)
    w0 = [w for w, n in disk_modes.eigenfrequencies(4.0, LAM, MU, RHO) if n == 1][0]   # 3.7254
    dev = {}
    for name, alpha in (("non_bm", 0.0), ("bm", None)):
        worst = 0.0
        for w in w0 + np.linspace(-0.01, 0.01, 81):
            h = fds.fds_build(xy, w, LAM, MU, 1e-10, leaf_size=32, alpha=alpha)
            F = fds.fds_rhs_plane_wave(h, np.array([0, 1], np.int32), np.array([0.0, 0.0]))
            x = fds.fds_solve(h, F)
            h.close()
            for j, kind in enumerate((0, 1)):
                u1, u2 = paomow.boundary_displacement(np.array([0.0]), 1.0, LAM, MU, RHO, w, kind, 0.0)
                ref = abs(u1[0]) ** 2 + abs(u2[0]) ** 2
                got = abs(x[0, j]) ** 2 + abs(x[N, j]) ** 2
                worst = max(worst, abs(got - ref) / ref)
        dev[name] = worst
    # discretisation error of the intensity is ~1% at 128 nodes
    assert dev["bm"] < 0.02, dev
    assert dev["non_bm"] > 0.5, dev
