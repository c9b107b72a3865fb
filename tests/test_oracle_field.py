"""Pins of the oracle's field evaluation (Sec. 3, eq. (integ_rep)): from the
exact boundary displacement of the circular cavity it must converge to the
Pao-Mow series off the boundary at the P1 rate, and inside the cavity the
representation must vanish (extinction theorem); from the oracle's own BEM
solution it must reproduce the series too."""
import numpy as np

import workloads
from oracle import bem, paomow

LAM, MU, RHO, OMEGA = 2.0, 1.0, 1.0, 2.0


def _pts(r, th):
    return np.stack([r * np.cos(th), r * np.sin(th)], 1)


def _exact_boundary(N, kind, th0):
    t = 2 * np.pi * np.arange(N) / N
    u1, u2 = paomow.boundary_displacement(t, 1.0, LAM, MU, RHO, OMEGA, kind, th0)
    return np.concatenate([u1, u2])


def test_field_converges_to_pao_mow_at_second_order():
    P = bem.phys(LAM, MU, RHO, OMEGA)
    rng = np.random.default_rng(3)
    r = np.array([1.5, 2.0, 3.0, 1.5, 2.5])
    th = rng.uniform(0, 2 * np.pi, 5)
    for kind in (0, 1):
        ref = np.array(paomow.field(r, th, 1.0, LAM, MU, RHO, OMEGA, kind, 0.3))
        errs = []
        for N in (128, 256, 512):
            f = bem.field(P, workloads.circle(N), _exact_boundary(N, kind, 0.3), kind, 0.3, _pts(r, th))
            errs.append(np.abs(f - ref).max() / np.abs(ref).max())
        assert errs[-1] < 1e-4
        assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


def test_representation_vanishes_inside_the_cavity():
    # extinction: for x in the cavity u^I(x) - int K u ds = 0 with the exact u
    P = bem.phys(LAM, MU, RHO, OMEGA)
    th = np.linspace(0.1, 6.0, 4)
    pts = _pts(np.array([0.2, 0.5, 0.6, 0.3]), th)
    errs = []
    for N in (128, 256):
        f = bem.field(P, workloads.circle(N), _exact_boundary(N, 1, 1.1), 1, 1.1, pts)
        errs.append(np.abs(f).max())
    assert errs[1] < 1e-3 and errs[0] / errs[1] > 3.5, errs


def test_field_from_bem_solution_matches_series():
    N = 256
    P = bem.phys(LAM, MU, RHO, OMEGA)
    xy = workloads.circle(N)
    x = bem.dense_solve(P, xy, bem.rhs(P, xy, 0, 0.7))
    r, th = np.array([1.3, 2.0, 4.0]), np.array([0.0, 2.0, 4.0])
    f = bem.field(P, xy, x, 0, 0.7, _pts(r, th))
    ref = np.array(paomow.field(r, th, 1.0, LAM, MU, RHO, OMEGA, 0, 0.7))
    assert np.abs(f - ref).max() / np.abs(ref).max() < 2e-3
