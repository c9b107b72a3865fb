"""End-to-end parity of the CUDA fast direct solver against the oracle's dense
Galerkin solve ('Conv') and its FDS restatement."""
import numpy as np
import pytest

import workloads
from gpu_util import fdslib, torch_cuda
from oracle import bem, fds as ofds, paomow

pytestmark = pytest.mark.gpu


def _dense(xy, lam, mu, omega, F):
    P = bem.phys(lam, mu, 1.0, omega)
    return np.linalg.solve(bem.dense_matrix(P, xy), F)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_circle_512_matches_dense_and_series():
    # 512 nodes on the unit circle, lambda=2, mu=1, k_T a = 1, leaf 32,
    # 64 proxy points at 1.5x the cell radius, eps = 1e-10, one plane P wave.
    torch_cuda()
    fds = fdslib()
    lam, mu, omega, eps = 2.0, 1.0, 1.0, 1e-10
    xy = workloads.circle(512)
    h = fds.fds_build(xy, omega, lam, mu, eps, leaf_size=32, top_level=1)
    f = fds.fds_rhs_plane_wave(h, np.array([0], np.int32), np.array([0.0]))[:, 0]
    x = fds.fds_solve(h, f)
    P = bem.phys(lam, mu, 1.0, omega)
    fo = bem.rhs(P, xy, 0, 0.0)
    xd = _dense(xy, lam, mu, omega, fo)
    assert _rel(x, xd) <= 10 * eps
    th = 2 * np.pi * np.arange(512) / 512
    u1, u2 = paomow.boundary_displacement(th, 1.0, lam, mu, 1.0, omega, 0, 0.0)
    assert _rel(x, np.concatenate([u1, u2])) < 1e-4
    st = fds.fds_stats_get(h)
    assert st.levels == 4 and st.top_level == 1
    h.close()


@pytest.mark.parametrize("l0", [0, 1, 2])
def test_exact_without_truncation(l0):
    torch_cuda()
    fds = fdslib()
    xy = workloads.star(256)
    h = fds.fds_build(xy, 3.0, 2.0, 1.0, 0.0, leaf_size=32, top_level=l0)
    P = bem.phys(2.0, 1.0, 1.0, 3.0)
    F = np.stack([bem.rhs(P, xy, 0, 0.3), bem.rhs(P, xy, 1, 1.9)], 1)
    assert _rel(fds.fds_solve(h, F), _dense(xy, 2.0, 1.0, 3.0, F)) < 1e-12
    h.close()


def test_ragged_tree_and_ranks_match_oracle():
    torch_cuda()
    fds = fdslib()
    N, omega, eps = 300, 4.0, 1e-8
    xy = workloads.tripod(N)
    h = fds.fds_build(xy, omega, 1.0, 1.0, eps, leaf_size=32, top_level=1)
    P = bem.phys(1.0, 1.0, 1.0, omega)
    F = np.stack([bem.rhs(P, xy, k, a) for k, a in ((0, 0.0), (1, 0.5), (0, 2.0))], 1)
    x = fds.fds_solve(h, F)
    assert _rel(x, _dense(xy, 1.0, 1.0, omega, F)) <= 10 * eps
    S = ofds.FDS(P, xy, 1.0, 1.0, 1.0, omega, eps, leaf_size=32, top_level=1)
    assert _rel(x, S.solve(F)) <= 10 * eps
    gpu = fds.fds_level_ranks(h, S.L, len(S.levels[S.L]))
    cpu = np.array(S.ranks()[S.L])
    assert np.abs(gpu - cpu).max() <= 1
    h.close()


def test_single_cell_is_dense_solve():
    torch_cuda()
    fds = fdslib()
    xy = workloads.ellipse(40, 2.0, 0.3)
    h = fds.fds_build(xy, 2.0, 2.0, 1.0, 1e-8, leaf_size=64)
    assert fds.fds_stats_get(h).levels == 0
    P = bem.phys(2.0, 1.0, 1.0, 2.0)
    f = bem.rhs(P, xy, 1, 0.2)
    assert _rel(fds.fds_solve(h, f), _dense(xy, 2.0, 1.0, 2.0, f)) < 1e-12
    h.close()


def test_device_solve_many_rhs():
    torch = torch_cuda()
    fds = fdslib()
    xy = workloads.star(1024)
    omega, eps = 10.0, 1e-8
    h = fds.fds_build(xy, omega, 2.0, 1.0, eps, leaf_size=64)
    kinds, angles = workloads.plane_wave_set(150)       # 300 RHS: crosses the 256-column chunk
    dk = torch.from_numpy(kinds).cuda()
    da = torch.from_numpy(angles).cuda()
    d = torch.zeros((len(kinds), 2 * 1024), dtype=torch.complex128, device="cuda")
    fds.fds_rhs_plane_wave_device(h, dk, da, d)
    F = d.cpu().numpy().T.copy()
    fds.fds_solve_device(h, d)
    torch.cuda.synchronize()
    X = d.cpu().numpy().T
    cols = [0, 1, 255, 256, 299]
    ref = _dense(xy, 2.0, 1.0, omega, F[:, cols])
    assert _rel(X[:, cols], ref) <= 10 * eps
    h.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_host_solve_chunks_match_device_solve(precision):
    """The host-buffer solve streams 256-column chunks through two device
    buffers with overlapped copies (600 columns: two full chunks and a ragged
    one); it must give the device solve's result."""
    torch = torch_cuda()
    fds = fdslib()
    prec = fds.FDS_MIXED if precision == "mixed" else fds.FDS_FP64
    xy = workloads.star(1024)
    omega = workloads.omega_for_kTa(5.0)
    h = fds.fds_build(xy, omega, 2.0, 1.0, 1e-9, precision=prec, ir_tol=1e-10)
    rng = np.random.default_rng(5)
    F = rng.standard_normal((2048, 600)) + 1j * rng.standard_normal((2048, 600))
    x_host = fds.fds_solve(h, F)
    st = fds.fds_stats_get(h)
    d = torch.tensor(np.ascontiguousarray(F.T), device="cuda")
    fds.fds_solve_device(h, d)
    torch.cuda.synchronize()
    x_dev = d.cpu().numpy().T
    assert np.abs(x_host - x_dev).max() <= 1e-13 * np.abs(x_dev).max()
    assert st.solve_ms > 0
    if precision == "mixed":
        assert st.ir_residual <= 1e-10
    h.close()
