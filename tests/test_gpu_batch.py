"""Batched multi-cavity build and solve (concurrent per-cavity streams)
against one-at-a-time builds and the oracle's dense solve."""
import ctypes

import numpy as np
import pytest

import workloads
from gpu_util import fdslib, torch_cuda
from oracle import bem

pytestmark = pytest.mark.gpu


def _cavities(count, seed):
    cav = workloads.random_cavities(count, seed=seed, nmin_log2=9, nmax_log2=11, kta=(1.0, 10.0))
    for c in cav:
        c["omega"] = workloads.omega_for_kTa(c["kTa"])
    return cav


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_batch_matches_single_builds_and_dense():
    torch = torch_cuda()
    fds = fdslib()
    cav = _cavities(7, workloads.SEED + 21)
    tol = 1e-9
    hb = fds.fds_build_batch(cav, 2.0, 1.0, tol, n_streams=4, leaf_size=64)
    kinds, ang = workloads.plane_wave_set(8)     # 16 waves per cavity
    d_rhs, ref = [], []
    for c, h in zip(cav, hb):
        F = fds.fds_rhs_plane_wave(h, kinds, ang)
        hs = fds.fds_build(c["xy"], c["omega"], 2.0, 1.0, tol, leaf_size=64)
        ref.append(fds.fds_solve(hs, F))
        hs.close()
        d_rhs.append(torch.tensor(np.ascontiguousarray(F.T), device="cuda"))
    fds.fds_solve_batch(hb, d_rhs, n_streams=4)
    for c, h, d, x in zip(cav, hb, d_rhs, ref):
        xb = d.cpu().numpy().T
        assert _rel(xb, x) < 1e-11
    # the smallest cavity against the dense Galerkin solve
    i = int(np.argmin([c["N"] for c in cav]))
    P = bem.phys(2.0, 1.0, 1.0, cav[i]["omega"])
    F = fds.fds_rhs_plane_wave(hb[i], kinds[:2], ang[:2])
    xd = np.linalg.solve(bem.dense_matrix(P, cav[i]["xy"]), F)
    assert _rel(fds.fds_solve(hb[i], F), xd) <= 10 * tol
    for h in hb:
        assert fds.fds_handle_stream(h) != 0
        h.close()


def test_batch_mixed_precision():
    torch = torch_cuda()
    fds = fdslib()
    cav = _cavities(4, workloads.SEED + 22)
    hb = fds.fds_build_batch(cav, 2.0, 1.0, 1e-9, n_streams=3, precision=fds.FDS_MIXED, ir_tol=1e-10)
    kinds, ang = workloads.plane_wave_set(3)
    d_rhs, F_list = [], []
    for h in hb:
        F = fds.fds_rhs_plane_wave(h, kinds, ang)
        F_list.append(F)
        d_rhs.append(torch.tensor(np.ascontiguousarray(F.T), device="cuda"))
    fds.fds_solve_batch(hb, d_rhs, n_streams=3)
    for c, h, d, F in zip(cav, hb, d_rhs, F_list):
        h64 = fds.fds_build(c["xy"], c["omega"], 2.0, 1.0, 1e-9)
        assert _rel(d.cpu().numpy().T, fds.fds_solve(h64, F)) < 1e-8
        h64.close()
        h.close()


def test_batch_error_releases_everything():
    torch_cuda()
    fds = fdslib()
    cav = _cavities(3, workloads.SEED + 23)
    cav.insert(1, dict(xy=workloads.circle(5), omega=1.0, N=5))      # too few nodes
    with pytest.raises(fds.FdsError) as e:
        fds.fds_build_batch(cav, 2.0, 1.0, 1e-8, n_streams=2)
    assert e.value.code == fds.FDS_ERR_ARG


@pytest.mark.parametrize("use_graph", [False, True])
def test_level_batched_solve_equals_per_cavity_solves(use_graph):
    # one launch per tree level and phase across cavities of different
    # depths (2^9..2^11 nodes: 3-5 levels below the top) and different
    # numbers of right-hand sides (300 = a full chunk + a ragged one; 1; 0);
    # the same kernels in the same summation order give the same bits
    torch = torch_cuda()
    fds = fdslib()
    cav = _cavities(6, workloads.SEED + 24)
    hb = fds.fds_build_batch(cav, 2.0, 1.0, 1e-9, n_streams=3, leaf_size=64)
    rng = np.random.default_rng(77)
    counts = [300, 16, 1, 0, 40, 257]
    d_rhs, ref = [], []
    for h, nr in zip(hb, counts):
        F = rng.standard_normal((2 * h.n, nr)) + 1j * rng.standard_normal((2 * h.n, nr))
        ref.append(fds.fds_solve(h, F.copy()) if nr else F)
        d_rhs.append(torch.tensor(np.ascontiguousarray(F.T), device="cuda"))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        fds.fds_solve_batch_levels(hb, d_rhs, use_graph=use_graph, stream=s.cuda_stream)
    s.synchronize()
    for d, x, nr in zip(d_rhs, ref, counts):
        if nr:
            assert np.array_equal(d.cpu().numpy().T, x)
    # handles of another precision are refused
    hm = fds.fds_build(cav[0]["xy"], cav[0]["omega"], 2.0, 1.0, 1e-9, precision=fds.FDS_MIXED)
    with pytest.raises(fds.FdsError) as e:
        fds.fds_solve_batch_levels([hm], [d_rhs[0]])
    assert e.value.code == fds.FDS_ERR_ARG
    hm.close()
    for h in hb:
        h.close()
