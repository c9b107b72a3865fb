"""Parity of each CUDA stage (kernel evaluation, proxy entries, interpolative
decomposition, batched LU, load vectors) against the oracle on the same inputs."""
import numpy as np
import pytest

import workloads
from gpu_util import dev, fdslib, torch_cuda
from oracle import bem, fds as ofds

pytestmark = pytest.mark.gpu
LAM, MU, RHO = 2.0, 1.0, 1.0


@pytest.mark.parametrize("N,omega", [(200, 5.0), (64, 0.1), (4096, 20.0), (8192, 5.0)])
def test_eval_entries_matches_oracle(N, omega):
    torch = torch_cuda()
    fds = fdslib()
    xy = workloads.star(N)
    rng = np.random.default_rng(N)
    # self, adjacent, near (2-3 apart), mid, far and wrap-around pairs
    base = [0, 1, 2, 3, 5, N - 1, N - 2, N // 2, N // 2 + 1, N // 3]
    rows = np.array(base + list(rng.integers(0, N, 6)), dtype=np.int32)
    cols = np.array(base[::-1] + list(rng.integers(0, N, 5)), dtype=np.int32)
    ref = bem.entries(bem.phys(LAM, MU, RHO, omega), xy, rows, cols)
    out = torch.zeros((2 * len(cols), 2 * len(rows)), dtype=torch.complex128, device="cuda")
    fds.fds_eval_entries(fds.physics(LAM, MU, RHO, omega), dev(torch, xy), dev(torch, rows), dev(torch, cols), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().T
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_eval_cross_matches_oracle():
    torch = torch_cuda()
    fds = fdslib()
    N = 512
    xy = workloads.star(N)
    box = np.arange(100, 164, dtype=np.int32)
    pts = xy[99:165]
    c = 0.5 * (pts.min(0) + pts.max(0))
    R = np.sqrt(((pts - c) ** 2).sum(1)).max()
    m = 64
    th = 2 * np.pi * np.arange(m) / m
    prox = np.stack([c[0] + 1.5 * R * np.cos(th), c[1] + 1.5 * R * np.sin(th)], 1)
    pidx = np.arange(m, dtype=np.int32)
    P = bem.phys(LAM, MU, RHO, 10.0)
    ph = fds.physics(LAM, MU, RHO, 10.0)
    for (X, rows, Y, cols) in ((prox, pidx, xy, box), (xy, box, prox, pidx)):
        ref = bem.cross_entries(P, X, rows, Y, cols, q=4)
        out = torch.zeros((2 * len(cols), 2 * len(rows)), dtype=torch.complex128, device="cuda")
        fds.fds_eval_cross(ph, dev(torch, X), dev(torch, rows), dev(torch, Y), dev(torch, cols), 4, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().T
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def _decaying(rng, m, n, decay):
    k = min(m, n)
    U, _ = np.linalg.qr(rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k)))
    V, _ = np.linalg.qr(rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k)))
    s = decay ** np.arange(k)
    return (U * s) @ V.conj().T


def test_id_batched_matches_oracle():
    torch = torch_cuda()
    fds = fdslib()
    rng = np.random.default_rng(7)
    shapes = [(50, 20), (300, 64), (30, 40), (7, 3), (200, 1), (96, 96)]
    mats = [_decaying(rng, m, n, 0.1) for m, n in shapes]
    tol = 1e-6
    off = np.cumsum([0] + [m * n for m, n in shapes]).astype(np.int64)
    poff = np.cumsum([0] + [n for _, n in shapes]).astype(np.int64)
    toff = np.cumsum([0] + [n * n // 4 + 1 for _, n in shapes]).astype(np.int64)
    Y = np.concatenate([M.T.ravel() for M in mats])             # column-major
    dY = dev(torch, Y)
    d_rank = torch.zeros(len(shapes), dtype=torch.int32, device="cuda")
    d_perm = torch.zeros(int(poff[-1]), dtype=torch.int32, device="cuda")
    d_T = torch.zeros(int(toff[-1]), dtype=torch.complex128, device="cuda")
    fds.fds_id_batched(dev(torch, np.array([m for m, _ in shapes], np.int32)),
                       dev(torch, np.array([n for _, n in shapes], np.int32)), dev(torch, off), dY, tol,
                       d_rank, d_perm, dev(torch, poff), d_T, dev(torch, toff))
    torch.cuda.synchronize()
    rank, perm, T = d_rank.cpu().numpy(), d_perm.cpu().numpy(), d_T.cpu().numpy()
    for b, (M, (m, n)) in enumerate(zip(mats, shapes)):
        k0, p0, T0 = ofds.cpqr_id(M, tol)
        k = int(rank[b])
        assert k == k0
        pb = perm[poff[b]:poff[b] + n]
        assert sorted(pb) == list(range(n))
        assert list(pb[:k]) == list(p0[:k])
        Tb = T[toff[b]:toff[b] + k * (n - k)].reshape(n - k, k).T
        if k and n - k:
            # the order of the non-skeleton columns is free: compare V = [I T] P^T
            Vg = ofds.interp_matrix(k, pb, Tb, n)
            Vo = ofds.interp_matrix(k0, p0, T0, n)
            assert np.abs(Vg - Vo).max() <= 1e-8 * max(1.0, np.abs(Vo).max())
            res = M[:, pb[k:]] - M[:, pb[:k]] @ Tb
            assert np.linalg.norm(res) <= 50 * tol * np.linalg.norm(M)


def test_lu_batched_reconstructs():
    torch = torch_cuda()
    fds = fdslib()
    rng = np.random.default_rng(3)
    sizes = [1, 5, 64, 128, 37]
    As = [rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d)) for d in sizes]
    off = np.cumsum([0] + [d * d for d in sizes]).astype(np.int64)
    poff = np.cumsum([0] + sizes).astype(np.int64)
    dA = dev(torch, np.concatenate([A.T.ravel() for A in As]))
    piv = torch.zeros(int(poff[-1]), dtype=torch.int32, device="cuda")
    info = torch.zeros(len(sizes), dtype=torch.int32, device="cuda")
    fds.fds_lu_batched(dev(torch, np.array(sizes, np.int32)), dev(torch, off), dA, piv, dev(torch, poff), info)
    torch.cuda.synchronize()
    LUall, pv = dA.cpu().numpy(), piv.cpu().numpy()
    assert (info.cpu().numpy() == 0).all()
    for b, (A, d) in enumerate(zip(As, sizes)):
        LU = LUall[off[b]:off[b + 1]].reshape(d, d).T
        L = np.tril(LU, -1) + np.eye(d)
        U = np.triu(LU)
        PA = A.copy()
        for k in range(d):
            p = pv[poff[b] + k]
            assert k <= p < d
            PA[[k, p]] = PA[[p, k]]
        assert np.abs(L @ U - PA).max() <= 1e-12 * np.abs(A).max() * d


def test_lu_batched_reports_singular():
    torch = torch_cuda()
    fds = fdslib()
    A = np.zeros((4, 4), dtype=np.complex128)
    A[0, 0] = 1.0
    dA = dev(torch, A.T.ravel())
    piv = torch.zeros(4, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    fds.fds_lu_batched(dev(torch, np.array([4], np.int32)), dev(torch, np.array([0], np.int64)), dA, piv,
                       dev(torch, np.array([0], np.int64)), info)
    torch.cuda.synchronize()
    assert int(info.cpu()[0]) == 2


def test_rhs_matches_oracle():
    fds = fdslib()
    torch_cuda()
    xy = workloads.tripod(300)
    h = fds.fds_build(xy, 2.0, 1.0, 1.0, 1e-6, leaf_size=64)
    kinds, angles = np.array([0, 1, 0], np.int32), np.array([0.0, 0.4, 2.5])
    got = fds.fds_rhs_plane_wave(h, kinds, angles)
    P = bem.phys(1.0, 1.0, 1.0, 2.0)
    for j in range(3):
        ref = bem.rhs(P, xy, int(kinds[j]), float(angles[j]))
        assert np.abs(got[:, j] - ref).max() <= 1e-13 * np.abs(ref).max()
    h.close()


def test_rhs_coarse_elements_matches_oracle():
    # k h ~ 1: the per-element phase steps take the sincos branch
    fds = fdslib()
    torch_cuda()
    xy = workloads.circle(64)
    h = fds.fds_build(xy, 10.0, 2.0, 1.0, 1e-6, leaf_size=16)
    kinds, angles = np.array([0, 1], np.int32), np.array([0.3, 1.7])
    got = fds.fds_rhs_plane_wave(h, kinds, angles)
    P = bem.phys(2.0, 1.0, 1.0, 10.0)
    for j in range(2):
        ref = bem.rhs(P, xy, int(kinds[j]), float(angles[j]))
        assert np.abs(got[:, j] - ref).max() <= 1e-13 * np.abs(ref).max()
    h.close()


def test_rhs_fine_elements_series_branch_matches_oracle():
    # k h ~ 1e-2: the closed-form Taylor integrals of the phase; 5 waves cover
    # a partial group of the kernel's waves per block
    fds = fdslib()
    torch_cuda()
    xy = workloads.star(4096)
    h = fds.fds_build(xy, 5.0, 2.0, 1.0, 1e-6, leaf_size=64)
    kinds, angles = np.array([0, 1, 1, 0, 1], np.int32), np.array([0.0, 0.4, 2.5, 4.0, 5.9])
    got = fds.fds_rhs_plane_wave(h, kinds, angles)
    P = bem.phys(2.0, 1.0, 1.0, 5.0)
    for j in range(len(kinds)):
        ref = bem.rhs(P, xy, int(kinds[j]), float(angles[j]))
        assert np.abs(got[:, j] - ref).max() <= 1e-13 * np.abs(ref).max()
    h.close()
