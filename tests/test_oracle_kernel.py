"""Pins of the oracle's kernel (eq. (funda) and the regularised D/N forms)."""
import numpy as np
import pytest
from scipy.special import hankel1

import kernel_direct as kd
from oracle import bem

LAM, MU, RHO, OMEGA = 2.0, 1.0, 1.0, 1.7


def test_green_satisfies_navier():
    # mu G_ij,kk + (lam+mu) G_kj,ki + rho w^2 G_ij = 0 away from the source
    # (Sec. 2, eq. (bvp1)); central differences, residual must fall as h^2.
    z0 = np.array([0.37, -0.81])

    def G(z):
        return kd.G_tensors(LAM, MU, RHO, OMEGA, z)[0]

    def residual(h):
        e = np.eye(2)
        H = np.zeros((2, 2, 2, 2), complex)  # H[a, b] = d_a d_b G
        for a in range(2):
            for b in range(2):
                H[a, b] = (G(z0 + h * e[a] + h * e[b]) - G(z0 + h * e[a] - h * e[b])
                           - G(z0 - h * e[a] + h * e[b]) + G(z0 - h * e[a] - h * e[b])) / (4 * h * h)
        lap = H[0, 0] + H[1, 1]
        graddiv = np.array([[sum(H[k, i][k, j] for k in range(2)) for j in range(2)] for i in range(2)])
        return np.abs(MU * lap + (LAM + MU) * graddiv + RHO * OMEGA ** 2 * G(z0)).max(), np.abs(MU * lap).max()

    r1, scale = residual(2e-3)
    r2, _ = residual(1e-3)
    assert r2 < 1e-4 * scale
    assert 3.0 < r1 / r2 < 5.0


def test_green_reciprocity_and_symmetry():
    for z in (np.array([0.3, 0.4]), np.array([-1.2, 0.05])):
        G = kd.G_tensors(LAM, MU, RHO, OMEGA, z)[0]
        Gm = kd.G_tensors(LAM, MU, RHO, OMEGA, -z)[0]
        assert np.allclose(G, Gm.T, rtol=1e-14, atol=1e-15)


def test_green_static_limit_normalisation():
    # G - G^s -> const * delta as r -> 0, with the plane-strain Kelvin solution
    # G^s_ij = -[(lam+3mu) delta_ij ln r - (lam+mu) rh_i rh_j] / (4 pi mu (lam+2mu))
    def Gs(z):
        r = np.linalg.norm(z)
        zh = z / r
        return -((LAM + 3 * MU) * np.eye(2) * np.log(r) - (LAM + MU) * np.outer(zh, zh)) / (
            4 * np.pi * MU * (LAM + 2 * MU))

    diffs = []
    for ang in (0.1, 1.3, 2.9):
        z = 1e-5 * np.array([np.cos(ang), np.sin(ang)])
        diffs.append(kd.G_tensors(LAM, MU, RHO, OMEGA, z)[0] - Gs(z))
    for d in diffs[1:]:
        assert np.abs(d - diffs[0]).max() < 1e-6
    assert abs(diffs[0][0, 1]) < 1e-6 and abs(diffs[0][0, 0] - diffs[0][1, 1]) < 1e-6


def _polygon(N=24):
    th = 2 * np.pi * np.arange(N) / N
    return np.stack([1.3 * np.cos(th) + 0.1 * np.cos(3 * th), np.sin(th)], 1)


def _hat_pieces(xy, s):
    N = len(xy)
    out = []
    for e, loc in (((s - 1) % N, 1), (s, 0)):
        a, b = xy[e], xy[(e + 1) % N]
        h = np.linalg.norm(b - a)
        t = (b - a) / h
        out.append((a, t, np.array([-t[1], t[0]]), h, loc))
    return out


def _hat_integral(P, xy, s, t, direct, q=12):
    g, w = np.polynomial.legendre.leggauss(q)
    g, w = 0.5 * (g + 1), 0.5 * w
    acc = np.zeros((2, 2), complex)
    for (a1, t1, n1, h1, A) in _hat_pieces(xy, s):
        for (a2, t2, n2, h2, B) in _hat_pieces(xy, t):
            for si, ws in zip(g, w):
                x = a1 + si * h1 * t1
                Na = si if A == 1 else 1 - si
                dNa = (1 if A == 1 else -1) / h1
                for ti, wt in zip(g, w):
                    y = a2 + ti * h2 * t2
                    Nb = ti if B == 1 else 1 - ti
                    dNb = (1 if B == 1 else -1) / h2
                    ww = ws * wt * h1 * h2
                    if direct:
                        K = kd.KD(LAM, MU, RHO, OMEGA, y - x, n2) + \
                            P._alpha * kd.KN(LAM, MU, RHO, OMEGA, y - x, n1, n2)
                        acc += ww * Na * Nb * K
                    else:
                        K = bem.kernel_blocks(P, y - x, n1, n2)
                        acc += ww * (Na * Nb * K[0] + Na * dNb * K[1] + dNa * Nb * K[2] + dNa * dNb * K[3])
    return acc


@pytest.mark.parametrize("s,t", [(0, 10), (3, 15), (20, 7)])
def test_regularised_equals_direct_on_separated_hats(s, t):
    alpha = 0.3 + 0.8j
    P = bem.phys(LAM, MU, RHO, OMEGA, alpha)
    P._alpha = alpha
    xy = _polygon()
    reg = _hat_integral(P, xy, s, t, direct=False)
    dire = _hat_integral(P, xy, s, t, direct=True)
    assert np.abs(reg - dire).max() < 1e-12 * np.abs(dire).max()
    # and the oracle's own quadrature rule on the same entry
    ent = bem.entries(P, xy, [s], [t])
    assert np.abs(ent - dire).max() < 1e-10 * np.abs(dire).max()


def test_ehat_series_matches_closed_form():
    for z in (0.02, 0.1, 0.4, 0.8, 0.999, 1.0, 1.5):
        closed = (z * hankel1(1, z) + 2j / np.pi) / z ** 2
        assert abs(bem.ehat(z) - closed) < 2e-13 * max(1.0, abs(closed)) + 1e-12 / z ** 2 * 1e-3
    # continuity across the series/closed-form switch
    assert abs(bem.ehat(1 - 1e-12) - bem.ehat(1 + 1e-12)) < 1e-11
