"""The formulation without the Burton–Miller term (Sec. 8.4, eq.
(bie_non_bie): (D + I_0/2) u = u^I, i.e. alpha = 0), pinned against closed
forms on the unit circle: it is singular exactly at the interior Dirichlet
eigenfrequencies of the elastic disk (the fictitious frequencies), the
Burton–Miller system is not, and away from those frequencies both converge
to the Pao–Mow series."""
import numpy as np
import pytest

import disk_modes
import workloads
from oracle import bem, paomow

LAM, MU, RHO = 2.0, 1.0, 1.0


def _smin(omega, alpha, N=128):
    A = bem.dense_matrix(bem.phys(LAM, MU, RHO, omega, alpha=alpha), workloads.circle(N))
    return np.linalg.svd(A, compute_uv=False)[-1]


def test_disk_eigenfrequencies_closed_form():
    # order 0 includes the torsional modes u_th = J_1(k_T r): k_T a = j_{1,1}
    ev = disk_modes.eigenfrequencies(6.0, LAM, MU, RHO)
    assert any(n == 0 and abs(w - 3.8317059702) < 1e-8 for w, n in ev)
    for w, n in ev:
        assert abs(disk_modes.det(n, w, LAM, MU, RHO)) < 1e-9


def test_non_bm_singular_at_fictitious_frequencies_bm_not():
    ev = disk_modes.eigenfrequencies(6.0, LAM, MU, RHO)
    assert len(ev) >= 4
    ref_non = min(_smin(3.0, 0.0), _smin(4.5, 0.0))
    ref_bm = min(_smin(3.0, None), _smin(4.5, None))
    for w, n in ev:
        # the discrete eigenvalue sits within O(h^2) of the continuous one
        assert _smin(w, 0.0) < 0.03 * ref_non, (w, n)
        assert _smin(w, None) > 0.5 * ref_bm, (w, n)


@pytest.mark.parametrize("kind", [0, 1])
def test_non_bm_converges_to_series_away_from_fictitious_frequencies(kind):
    # omega = 2 lies below the first interior Dirichlet eigenfrequency (3.725)
    omega, errs = 2.0, []
    for N in (48, 96, 192):
        xy = workloads.circle(N)
        th = 2 * np.pi * np.arange(N) / N
        P = bem.phys(LAM, MU, RHO, omega, alpha=0.0)
        x = bem.dense_solve(P, xy, bem.rhs(P, xy, kind, 0.3))
        u1, u2 = paomow.boundary_displacement(th, 1.0, LAM, MU, RHO, omega, kind, 0.3)
        ex = np.concatenate([u1, u2])
        errs.append(np.linalg.norm(x - ex) / np.linalg.norm(ex))
    assert errs[-1] < 2e-3
    for e0, e1 in zip(errs, errs[1:]):
        assert 3.3 < e0 / e1 < 4.7
