"""Accuracy of the CUDA solver against the oracle's dense Galerkin solve at
2^12 and 2^13 nodes (tree depths 6 and 7 with 64-node leaves), where the
multi-level error growth of Sec. 8.1 (Table tab:error) shows, and against the
paper's own Table 1 / Table 2 errors on its tripod.

The dense solutions at 2^12-2^13 nodes come from tests/golden/make_dense.py
(oracle only: dense assembly + LU).  Bound: relative L2 error per right-hand
side <= 10 eps, with eps the leaf-level ID tolerance (the largest one used)."""
import os

import numpy as np
import pytest

import workloads
from gpu_util import fdslib, torch_cuda
from oracle import bem

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
EPS = 1e-9


def _golden(N, kta):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_dense", os.path.join(HERE, "golden", "make_dense.py"))
    md = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(md)
    d = np.load(md.path(N, kta))
    return workloads.star(N), workloads.omega_for_kTa(kta), md.load_vectors(N, kta), d["x"]


def _colerr(x, xd):
    return np.linalg.norm(x - xd, axis=0) / np.linalg.norm(xd, axis=0)


@pytest.mark.parametrize("N,kta", [(4096, 10.0), (4096, 20.0), (8192, 10.0), (8192, 20.0)])
def test_fp64_and_mixed_within_10_eps_of_dense(N, kta):
    torch_cuda()
    fds = fdslib()
    xy, omega, F, xd = _golden(N, kta)
    h = fds.fds_build(xy, omega, 2.0, 1.0, EPS)
    e64 = _colerr(fds.fds_solve(h, F), xd)
    h.close()
    assert e64.max() <= 10 * EPS, e64
    hm = fds.fds_build(xy, omega, 2.0, 1.0, EPS, precision=fds.FDS_MIXED, ir_tol=1e-10)
    em = _colerr(fds.fds_solve(hm, F), xd)
    hm.close()
    assert em.max() <= 10 * EPS, em


@pytest.mark.parametrize("N,kta", [(4096, 20.0), (8192, 10.0)])
def test_learned_rank_within_10_eps_of_dense(N, kta):
    torch_cuda()
    fds = fdslib()
    from paper_2411_18026_gb300 import learned
    prm = learned.load_params()
    assert prm is not None
    xy, omega, F, xd = _golden(N, kta)
    h = fds.fds_build(xy, omega, 2.0, 1.0, EPS, precision=fds.FDS_MIXED, ir_tol=1e-10, mlp_params=prm)
    e = _colerr(fds.fds_solve(h, F), xd)
    st = fds.fds_stats_get(h)
    h.close()
    assert st.id_sketched > 0
    assert e.max() <= 10 * EPS, e


def test_single_tolerance_error_grows_with_depth_graded_does_not():
    # the paper's single ID tolerance at every level (tol_decay = 1): the error
    # relative to eps grows with the depth (Sec. 8.1, Table tab:error); with the
    # tolerance halved per level up (the default) it stays below 10 eps
    torch_cuda()
    fds = fdslib()
    ratio = {}
    for N in (4096, 8192):
        xy, omega, F, xd = _golden(N, 10.0)
        for dec in (1.0, 0.5):
            h = fds.fds_build(xy, omega, 2.0, 1.0, EPS, tol_decay=dec)
            ratio[N, dec] = _colerr(fds.fds_solve(h, F), xd).max() / EPS
            h.close()
    assert ratio[8192, 1.0] > 1.5 * ratio[4096, 1.0] and ratio[8192, 1.0] > 10, ratio
    assert ratio[4096, 0.5] <= 10 and ratio[8192, 0.5] <= 10, ratio


@pytest.mark.parametrize("N", [4096, 8192])
def test_single_level_variant_within_eps_of_dense(N):
    # l0 = L - 1 (Sec. 8.1, Table tab:error_single): only the leaves are compressed
    torch_cuda()
    fds = fdslib()
    xy, omega, F, xd = _golden(N, 20.0)
    h = fds.fds_build(xy, omega, 2.0, 1.0, EPS, top_level=-1)
    st = fds.fds_stats_get(h)
    assert st.top_level == st.levels - 1
    e = _colerr(fds.fds_solve(h, F), xd)
    h.close()
    assert e.max() <= 2 * EPS, e


def _table(name):
    rows = {}
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = line.split()
            rows[int(v[0])] = [float(a) if "e" in a else int(a) for a in v[1:]]
    return rows


@pytest.mark.parametrize("N", [400, 800, 1600])
def test_tripod_errors_in_the_band_of_paper_tables(N):
    # the paper's tripod workload (lambda = mu = 1, omega = 2, leaf 100): the
    # multi-level error with the paper's single tolerance within a factor 20
    # of Table 1 (eps 1e-8, 1e-9, 1e-10), and the single-level variant's
    # within a factor 20 of Table 2 (eps 1e-8); the paper leaves alpha, the
    # proxy discretisation and the quadrature unstated, so the check is the band
    torch_cuda()
    fds = fdslib()
    xy = workloads.tripod(N)
    P = bem.phys(1.0, 1.0, 1.0, 2.0)
    f = bem.rhs(P, xy, 0, 0.0)
    x = np.linalg.solve(bem.dense_matrix(P, xy), f)
    t1, t2 = _table("paper_table1.txt")[N], _table("paper_table2.txt")[N]
    for eps, ref in zip((1e-8, 1e-9, 1e-10), t1[2:]):
        h = fds.fds_build(xy, 2.0, 1.0, 1.0, eps, leaf_size=100, top_level=t1[1], tol_decay=1.0)
        assert fds.fds_stats_get(h).levels == t1[0]
        err = np.linalg.norm(fds.fds_solve(h, f) - x) / np.linalg.norm(x)
        h.close()
        assert ref / 20 < err < ref * 20, (N, eps, err, ref)
    h = fds.fds_build(xy, 2.0, 1.0, 1.0, 1e-8, leaf_size=100, top_level=t2[1])
    err = np.linalg.norm(fds.fds_solve(h, f) - x) / np.linalg.norm(x)
    h.close()
    assert t2[2] / 20 < err < t2[2] * 20, (N, err, t2)
