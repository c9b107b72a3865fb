"""Pins of the oracle's interpolative decomposition and fast-direct-solver
restatement (Secs. 6–7)."""
import itertools
import os

import numpy as np
import pytest

from oracle import bem, fds

import workloads

HERE = os.path.dirname(os.path.abspath(__file__))


def test_id_recovers_exact_low_rank():
    rng = np.random.default_rng(1)
    m, n, k = 60, 25, 7
    B = rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))
    C = rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))
    Y = B @ C
    kk, perm, T = fds.cpqr_id(Y, 1e-12)
    assert kk == k
    assert np.abs(Y[:, perm[k:]] - Y[:, perm[:k]] @ T).max() < 1e-11 * np.abs(Y).max()
    V = fds.interp_matrix(kk, perm, T, n)
    assert np.abs(Y - Y[:, perm[:k]] @ V).max() < 1e-11 * np.abs(Y).max()


def test_id_truncation_rule_and_residual():
    rng = np.random.default_rng(2)
    m, n = 80, 30
    Uq, _ = np.linalg.qr(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n)))
    Vq, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    s = 10.0 ** (-np.arange(n) / 2.0)
    Y = (Uq * s) @ Vq.conj().T
    for eps in (1e-3, 1e-6, 1e-9):
        k, perm, T = fds.cpqr_id(Y, eps)
        # the k-th pivot passed the test, the next one failed it
        Q, R = np.linalg.qr(Y[:, perm])
        d = np.abs(np.diag(R))
        assert d[k - 1] > eps * d[0]
        if k < n:
            assert d[k] <= eps * d[0] * (1 + 1e-8)
        res = np.linalg.norm(Y[:, perm[k:]] - Y[:, perm[:k]] @ T)
        assert res <= 50 * eps * np.linalg.norm(Y)


def test_id_greedy_pivots_brute_force():
    # each pivot maximises the norm of the column's component orthogonal to the
    # span of the earlier pivots (brute force over all remaining columns)
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((9, 6)) + 1j * rng.standard_normal((9, 6))
    k, perm, _ = fds.cpqr_id(Y, 0.0)
    for j in range(k):
        chosen = list(perm[:j])
        Qb = np.linalg.qr(Y[:, chosen])[0] if chosen else np.zeros((9, 0))
        resid = {c: np.linalg.norm(Y[:, c] - Qb @ (Qb.conj().T @ Y[:, c]))
                 for c in range(6) if c not in chosen}
        best = max(resid.values())
        assert resid[perm[j]] >= best * (1 - 1e-12)


def _setup(N, omega, shape="star", lam=2.0, mu=1.0):
    xy = workloads.star(N) if shape == "star" else workloads.circle(N)
    P = bem.phys(lam, mu, 1.0, omega)
    A = bem.dense_matrix(P, xy)
    F = np.stack([bem.rhs(P, xy, 0, 0.0), bem.rhs(P, xy, 1, 1.1)], 1)
    return xy, P, A, F


@pytest.mark.parametrize("N,leaf,l0", [(96, 24, 0), (96, 24, 1), (128, 16, 2), (128, 16, 1)])
def test_fds_is_exact_when_nothing_is_truncated(N, leaf, l0):
    # eps = 0 keeps every column as a skeleton: U = V = permutations, and
    # eqs. (elim)–(down_comv) become identities, so FDS = dense LU.
    xy, P, A, F = _setup(N, 2.0)
    x = np.linalg.solve(A, F)
    S = fds.FDS(P, xy, 2.0, 1.0, 1.0, 2.0, 0.0, leaf_size=leaf, top_level=l0)
    assert np.linalg.norm(S.solve(F) - x) / np.linalg.norm(x) < 1e-12


@pytest.mark.parametrize("eps", [1e-6, 1e-8, 1e-10])
def test_fds_error_tracks_id_tolerance(eps):
    xy, P, A, F = _setup(256, 4.0)
    x = np.linalg.solve(A, F)
    S = fds.FDS(P, xy, 2.0, 1.0, 1.0, 4.0, eps, leaf_size=32, top_level=1)
    err = np.linalg.norm(S.solve(F) - x) / np.linalg.norm(x)
    assert err <= 10 * eps
    # and it really compressed
    assert S.Atop.shape[0] < 0.85 * 2 * 256


def _table1():
    rows = {}
    with open(os.path.join(HERE, "golden", "paper_table1.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = line.split()
            rows[int(v[0])] = dict(L=int(v[1]), l0=int(v[2]), err={1e-8: float(v[3]), 1e-9: float(v[4]),
                                                                   1e-10: float(v[5])})
    return rows


@pytest.mark.slow
def test_tripod_error_band_of_paper_table1():
    # Same workload as Table 1's first row; the paper leaves alpha, the proxy
    # discretisation and the quadrature unstated, so the check is the decade.
    row = _table1()[400]
    xy = workloads.tripod(400)
    P = bem.phys(1.0, 1.0, 1.0, 2.0)
    f = bem.rhs(P, xy, 0, 0.0)
    x = np.linalg.solve(bem.dense_matrix(P, xy), f)
    for eps in (1e-8, 1e-10):
        S = fds.FDS(P, xy, 1.0, 1.0, 1.0, 2.0, eps, leaf_size=100, top_level=row["l0"], tol_decay=1.0)
        assert S.L == row["L"]
        err = np.linalg.norm(S.solve(f) - x) / np.linalg.norm(x)
        assert row["err"][eps] / 20 < err < row["err"][eps] * 20
