"""Field evaluation off the boundary (Sec. 3, eq. (integ_rep)) on the GPU
against the oracle on the same boundary data, and through the whole
pipeline against the Pao-Mow series."""
import numpy as np
import pytest

import workloads
from gpu_util import fdslib, torch_cuda
from oracle import bem, paomow

pytestmark = pytest.mark.gpu
LAM, MU, RHO = 2.0, 1.0, 1.0


def _pts(r, th):
    return np.stack([r * np.cos(th), r * np.sin(th)], 1)


def test_field_matches_oracle_on_the_same_boundary_data():
    torch = torch_cuda()
    fds = fdslib()
    N, omega = 512, 3.0
    xy = workloads.star(N)
    h = fds.fds_build(xy, omega, LAM, MU, 1e-8)
    rng = np.random.default_rng(17)
    kinds, angles = np.array([0, 1, 0, 1, 1, 0, 0, 1, 0], np.int32), rng.uniform(0, 2 * np.pi, 9)
    U = rng.standard_normal((9, 2 * N)) + 1j * rng.standard_normal((9, 2 * N))
    # exterior points at 1.3-3 radii and interior points of the cavity (extinction region)
    pts = np.concatenate([_pts(rng.uniform(1.5, 3.0, 12), rng.uniform(0, 2 * np.pi, 12)),
                          _pts(rng.uniform(0.1, 0.5, 4), rng.uniform(0, 2 * np.pi, 4))])
    got = fds.fds_field(h, torch.tensor(U, device="cuda"), kinds, angles, pts)
    P = bem.phys(LAM, MU, RHO, omega)
    for j in range(9):
        ref = bem.field(P, xy, U[j], int(kinds[j]), float(angles[j]), pts)
        assert np.abs(got[:, :, j] - ref).max() <= 1e-11 * np.abs(ref).max(), j
    h.close()


def test_field_of_the_solution_matches_pao_mow():
    torch = torch_cuda()
    fds = fdslib()
    N = 4096
    omega = workloads.omega_for_kTa(5.0)
    xy = workloads.circle(N)
    h = fds.fds_build(xy, omega, LAM, MU, 1e-10)
    kinds, angles = np.array([0, 1], np.int32), np.array([0.3, 1.2])
    F = fds.fds_rhs_plane_wave(h, kinds, angles)
    d = torch.tensor(np.ascontiguousarray(F.T), device="cuda")
    fds.fds_solve_device(h, d)
    r, th = np.linspace(1.2, 3.0, 10), np.linspace(0.0, 6.0, 10)
    got = fds.fds_field(h, d, kinds, angles, _pts(r, th))
    for j in range(2):
        ref = np.array(paomow.field(r, th, 1.0, LAM, MU, RHO, omega, int(kinds[j]), float(angles[j])))
        assert np.abs(got[:, :, j] - ref).max() / np.abs(ref).max() < 1e-4, j
    h.close()


@pytest.mark.parametrize("N,l0", [(8192, 1), (1 << 16, 2)])
def test_compressed_field_matches_direct_summation(N, l0):
    # the tree's skeletons as equivalent sources: the same field as direct
    # summation to the ID tolerance, at exterior points, points a few element
    # lengths off the boundary and points inside the cavity, for random
    # boundary data and for the solution; and far fewer hats per point
    torch = torch_cuda()
    fds = fdslib()
    xy = workloads.star(N)
    omega = workloads.omega_for_kTa(10.0)
    h = fds.fds_build(xy, omega, LAM, MU, 1e-10, top_level=l0)
    rng = np.random.default_rng(29)
    kinds, angles = np.array([0, 1, 1], np.int32), np.array([0.2, 1.0, 4.0])
    th = rng.uniform(0, 2 * np.pi, 8)
    rb = 1.0 + 0.2 * np.cos(5 * th)
    pts = np.concatenate([_pts(rng.uniform(1.3, 3.0, 16), rng.uniform(0, 2 * np.pi, 16)),
                          _pts(rb + 4 * 2 * np.pi / N, th),          # ~4 element lengths outside
                          _pts(rng.uniform(0.1, 0.6, 8), rng.uniform(0, 2 * np.pi, 8))])
    U = rng.standard_normal((3, 2 * N)) + 1j * rng.standard_normal((3, 2 * N))
    F = fds.fds_rhs_plane_wave(h, kinds, angles)
    d = torch.tensor(np.ascontiguousarray(F.T), device="cuda")
    fds.fds_solve_device(h, d)
    for data in (torch.tensor(U, device="cuda"), d):
        ref = fds.fds_field(h, data, kinds, angles, pts)
        fds.fds_timing_reset()
        fds.fds_timing_enable(True)
        got = fds.fds_field(h, data, kinds, angles, pts, compressed=True)
        fds.fds_timing_enable(False)
        hats = fds.fds_timing_report()["f1.field_compressed"]["units"] / len(kinds)
        for j in range(len(kinds)):
            scale = np.abs(ref[:, :, j]).max()
            assert np.abs(got[:, :, j] - ref[:, :, j]).max() <= 1e-7 * scale, (j, np.abs(got - ref).max() / scale)
        assert hats < 0.25 * N * len(pts), hats / (N * len(pts))
    h.close()


def test_compressed_field_of_the_solution_matches_pao_mow():
    torch = torch_cuda()
    fds = fdslib()
    N = 1 << 15
    omega = workloads.omega_for_kTa(10.0)
    h = fds.fds_build(workloads.circle(N), omega, LAM, MU, 1e-10)
    kinds, angles = np.array([0, 1], np.int32), np.array([0.3, 1.2])
    F = fds.fds_rhs_plane_wave(h, kinds, angles)
    d = torch.tensor(np.ascontiguousarray(F.T), device="cuda")
    fds.fds_solve_device(h, d)
    r, th = np.linspace(1.05, 3.0, 12), np.linspace(0.0, 6.0, 12)
    got = fds.fds_field(h, d, kinds, angles, _pts(r, th), compressed=True)
    for j in range(2):
        ref = np.array(paomow.field(r, th, 1.0, LAM, MU, RHO, omega, int(kinds[j]), float(angles[j])))
        assert np.abs(got[:, :, j] - ref).max() / np.abs(ref).max() < 1e-5, j
    h.close()
