"""Pins of the oracle's element-pair quadrature rule against adaptive
integration of the same regularised integrand (self, adjacent, near, far)."""
import numpy as np
import pytest
from scipy.integrate import quad_vec

from oracle import bem

LAM, MU, RHO = 2.0, 1.0, 1.0


def _poly(N, omega_scale=1.0):
    th = 2 * np.pi * np.arange(N) / N
    r = 1 + 0.2 * np.cos(5 * th)
    return np.stack([r * np.cos(th), r * np.sin(th)], 1)


def _elem(xy, e):
    N = len(xy)
    a, b = xy[e], xy[(e + 1) % N]
    h = np.linalg.norm(b - a)
    t = (b - a) / h
    return a, t, np.array([-t[1], t[0]]), h


def _integrand(P, e, f, sig, tau, z):
    (_, _, n1, h1), (_, _, n2, h2) = e, f
    K = bem.kernel_blocks(P, z, n1, n2)
    Na = np.array([1 - sig, sig]); dNa = np.array([-1, 1]) / h1
    Nb = np.array([1 - tau, tau]); dNb = np.array([-1, 1]) / h2
    out = (np.einsum('a,b,ij->abij', Na, Nb, K[0]) + np.einsum('a,b,ij->abij', Na, dNb, K[1])
           + np.einsum('a,b,ij->abij', dNa, Nb, K[2]) + np.einsum('a,b,ij->abij', dNa, dNb, K[3]))
    return out * h1 * h2


def _gl(q):
    g, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (g + 1), 0.5 * w


def _ref_self(P, E):
    a, t, n, h = E
    gv, wv = _gl(6)   # integrand is polynomial in v for fixed u: exact

    def fu(u):
        acc = np.zeros((2, 2, 2, 2), complex)
        for v, w in zip(gv * (1 - u), wv * (1 - u)):
            acc += w * (_integrand(P, E, E, v, v + u, u * h * t) + _integrand(P, E, E, v + u, v, -u * h * t))
        return acc.ravel()

    val, _ = quad_vec(fu, 0.0, 1.0, epsabs=1e-14, epsrel=1e-13, points=[1e-8, 1e-5, 1e-3, 0.1])
    return val.reshape(2, 2, 2, 2)


def _ref_adjacent(P, e, f, nxt):
    ge, we = _gl(24)
    (_, te, _, he), (_, tf, _, hf) = e, f

    def fxi(xi):
        acc = np.zeros((2, 2, 2, 2), complex)
        for tri in (0, 1):
            for eta, w in zip(ge, we):
                al, be = (xi, xi * eta) if tri == 0 else (xi * eta, xi)
                if nxt:
                    sig, tau, z = 1 - al, be, be * hf * tf + al * he * te
                else:
                    sig, tau, z = al, 1 - be, -be * hf * tf - al * he * te
                acc += w * xi * _integrand(P, e, f, sig, tau, z)
        return acc.ravel()

    val, _ = quad_vec(fxi, 0.0, 1.0, epsabs=1e-14, epsrel=1e-13, points=[1e-6, 1e-3, 0.1])
    return val.reshape(2, 2, 2, 2)


def _ref_regular(P, e, f, split=4, q=16):
    g, w = _gl(q)
    acc = np.zeros((2, 2, 2, 2), complex)
    (a1, t1, _, h1), (a2, t2, _, h2) = e, f
    for s0 in range(split):
        for t0 in range(split):
            for si, ws in zip((s0 + g) / split, w / split):
                for ti, wt in zip((t0 + g) / split, w / split):
                    z = (a2 + ti * h2 * t2) - (a1 + si * h1 * t1)
                    acc += ws * wt * _integrand(P, e, f, si, ti, z)
    return acc


@pytest.mark.parametrize("omega,N", [(1.0, 64), (10.0, 256)])
def test_self_pair(omega, N):
    P = bem.phys(LAM, MU, RHO, omega)
    xy = _poly(N)
    got = bem.pair(P, xy, 5, 5)
    ref = _ref_self(P, _elem(xy, 5))
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("nxt", [1, 0])
def test_adjacent_pair(nxt):
    P = bem.phys(LAM, MU, RHO, 3.0)
    xy = _poly(64)
    e = 9
    f = e + 1 if nxt else e - 1
    got = bem.pair(P, xy, e, f)
    ref = _ref_adjacent(P, _elem(xy, e), _elem(xy, f), nxt)
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("gap", [2, 3, 5, 9, 16, 24])
def test_near_mid_far_pairs(gap):
    P = bem.phys(LAM, MU, RHO, 3.0)
    xy = _poly(64)
    got = bem.pair(P, xy, 20, 20 + gap)
    ref = _ref_regular(P, _elem(xy, 20), _elem(xy, 20 + gap))
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("gap", [24, 40])
def test_far3_pairs_on_a_fine_mesh(gap):
    # 3x3 rule at >= 24 max(h) when k_T max(h) <= 0.02 (here 0.012)
    P = bem.phys(LAM, MU, RHO, 1.0)
    xy = _poly(512)
    got = bem.pair(P, xy, 20, 20 + gap)
    ref = _ref_regular(P, _elem(xy, 20), _elem(xy, 20 + gap))
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()
