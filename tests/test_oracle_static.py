"""Static identities that pin the jump term and the sign of D, and the
hypersingular N, independently of the dynamic kernel details (low frequency).

With n pointing into the cavity (Sec. 2) the elastic double layer of a constant
density equals that constant inside the cavity and 0 in the solid, so on the
boundary D c = c/2 and, in Galerkin form, D_h c = I_0 c / 2; the traction of a
rigid motion vanishes, so N_h applied to translations and to the rotation
(-x_2, x_1) is zero.  Both hold exactly on a polygon with P1 hats."""
import numpy as np

from oracle import bem

import workloads

LAM, MU, RHO = 2.0, 1.0, 1.0
OMEGA = 1e-3


def _mass_rowsum(xy):
    N = len(xy)
    h = np.linalg.norm(np.roll(xy, -1, 0) - xy, axis=1)   # element s: node s -> s+1
    return 0.5 * (np.roll(h, 1) + h)


def _mats(xy):
    A0 = bem.dense_matrix(bem.phys(LAM, MU, RHO, OMEGA, 0.0), xy)       # D + I0/2
    A1 = bem.dense_matrix(bem.phys(LAM, MU, RHO, OMEGA, 1.0), xy)       # D + I0/2 + N
    return A0, A1 - A0


def test_double_layer_of_constants():
    xy = workloads.star(96)
    A0, _ = _mats(xy)
    m = _mass_rowsum(xy)
    N = len(xy)
    for c in (np.array([1.0, 0.0]), np.array([0.3, -0.7])):
        cv = np.concatenate([np.full(N, c[0]), np.full(N, c[1])])
        got = A0 @ cv                       # = D c + I0 c / 2
        want = np.concatenate([m * c[0], m * c[1]])   # = I0 c
        assert np.abs(got - want).max() < 1e-4 * np.abs(want).max()


def test_hypersingular_kills_rigid_motions():
    xy = workloads.tripod(128)
    _, Nm = _mats(xy)
    N = len(xy)
    scale = np.abs(Nm).max()
    for u in (np.concatenate([np.ones(N), np.zeros(N)]),
              np.concatenate([np.zeros(N), np.ones(N)]),
              np.concatenate([-xy[:, 1], xy[:, 0]])):
        assert np.abs(Nm @ u).max() < 1e-5 * scale * np.abs(u).max()
