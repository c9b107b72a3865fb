"""The oracle's dense Galerkin BEM against the Pao–Mow type series for a
traction-free circular cavity (plane P and SV incidence)."""
import numpy as np
import pytest

from oracle import bem, paomow

import workloads

LAM, MU, RHO = 2.0, 1.0, 1.0


@pytest.mark.parametrize("kind", [0, 1])
def test_series_is_traction_free_and_reduces_to_incident(kind):
    # The series itself: traction at r = a vanishes (finite differences of the
    # displacement in polar coordinates), and far from the cavity the field is
    # the incident wave plus an outgoing remainder that decays like r^-1/2.
    a, omega, th0 = 1.0, 2.0, 0.4
    coef = paomow.coefficients(a, LAM, MU, RHO, omega, kind, th0)
    th = np.linspace(0, 2 * np.pi, 7, endpoint=False)
    h = 1e-4

    def u_polar(r, t):
        u1, u2 = paomow.field(r, t, a, LAM, MU, RHO, omega, kind, th0, coef=coef)
        return u1 * np.cos(t) + u2 * np.sin(t), -u1 * np.sin(t) + u2 * np.cos(t)

    ur, ut = u_polar(a, th)
    dur = (np.array(u_polar(a + h, th)) - np.array(u_polar(a + 2 * h, th)) * 0.25 - 0.75 * np.array([ur, ut])) / (0.5 * h)
    urr, utr = dur
    urt = (u_polar(a, th + h)[0] - u_polar(a, th - h)[0]) / (2 * h)
    utt = (u_polar(a, th + h)[1] - u_polar(a, th - h)[1]) / (2 * h)
    srr = (LAM + 2 * MU) * urr + LAM * (ur + utt) / a
    srt = MU * (urt / a + utr - ut / a)
    scale = omega * (LAM + 2 * MU) * max(np.abs(ur).max(), np.abs(ut).max())
    assert np.abs(srr).max() < 1e-5 * scale
    assert np.abs(srt).max() < 1e-5 * scale


@pytest.mark.parametrize("kind,omega", [(0, 1.0), (1, 1.0), (0, 3.0), (1, 3.0)])
def test_bem_converges_to_series_at_second_order(kind, omega):
    errs = []
    for N in (48, 96, 192):
        xy = workloads.circle(N)
        th = 2 * np.pi * np.arange(N) / N
        P = bem.phys(LAM, MU, RHO, omega)
        x = bem.dense_solve(P, xy, bem.rhs(P, xy, kind, 0.3))
        u1, u2 = paomow.boundary_displacement(th, 1.0, LAM, MU, RHO, omega, kind, 0.3)
        ex = np.concatenate([u1, u2])
        errs.append(np.linalg.norm(x - ex) / np.linalg.norm(ex))
    assert errs[-1] < 2e-3
    for e0, e1 in zip(errs, errs[1:]):
        assert 3.3 < e0 / e1 < 4.7
