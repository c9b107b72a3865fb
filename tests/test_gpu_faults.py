"""Failure paths with injected faults (fds_fault_inject), every one made on
the host or by withheld work, never by a bad access: a device allocation
that fails in the middle of a build, a NaN in a leaf block, and tensor-core
pipelines whose bounded waits run out because a producer never issues its
copies (or an issuer its MMAs).  Each call returns its error code, and
afterwards the library and the device context give the answers of an
unfaulted run (two builds agree to the compression tolerance: the tile
evaluator's shared-memory atomics add in no fixed order)."""
import time

import numpy as np
import pytest

import workloads
from gpu_util import fdslib, torch_cuda

pytestmark = pytest.mark.gpu

LAM, MU = 2.0, 1.0


@pytest.fixture(autouse=True)
def _disarm():
    yield
    fds = fdslib()
    fds.fds_fault_inject(fds.FDS_FAULT_NONE)


def _problem():
    return workloads.star(2048, 0.2, 5), workloads.omega_for_kTa(10.0)


def _reference(fds, xy, omega, **kw):
    kinds, ang = np.array([0, 1], np.int32), np.array([0.3, 1.2])
    h = fds.fds_build(xy, omega, LAM, MU, 1e-8, **kw)
    F = fds.fds_rhs_plane_wave(h, kinds, ang)
    x = fds.fds_solve(h, F)
    h.close()
    return F, x


def _same(x, xref):
    # eps = 1e-8: two valid builds are within a few eps of each other
    return np.linalg.norm(x - xref) <= 1e-7 * np.linalg.norm(xref)


def test_allocation_failure_mid_build_returns_oom_and_recovers():
    torch = torch_cuda()
    fds = fdslib()
    xy, omega = _problem()
    F, xref = _reference(fds, xy, omega)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    # the 1st, 7th and 40th allocation of a build that makes ~100 of them
    for n in (1, 7, 40):
        fds.fds_fault_inject(fds.FDS_FAULT_ALLOC, n)
        with pytest.raises(fds.FdsError) as e:
            fds.fds_build(xy, omega, LAM, MU, 1e-8)
        assert e.value.code == fds.FDS_ERR_OOM, n
    torch.cuda.synchronize()
    # what the failed builds had allocated was freed
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)
    h = fds.fds_build(xy, omega, LAM, MU, 1e-8)
    x = fds.fds_solve(h, F)
    h.close()
    assert _same(x, xref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nan_in_leaf_block_gives_singular(precision):
    torch_cuda()
    fds = fdslib()
    xy, omega = _problem()
    kw = {} if precision == "fp64" else dict(precision=fds.FDS_MIXED, ir_tol=1e-9)
    F, xref = _reference(fds, xy, omega, **kw)
    fds.fds_fault_inject(fds.FDS_FAULT_NAN_BLOCK)
    with pytest.raises(fds.FdsError) as e:
        fds.fds_build(xy, omega, LAM, MU, 1e-8, **kw)
    assert e.value.code == fds.FDS_ERR_SINGULAR
    # the fault fired once: the next build is clean
    h = fds.fds_build(xy, omega, LAM, MU, 1e-8, **kw)
    x = fds.fds_solve(h, F)
    h.close()
    assert _same(x, xref)


def _blocks(torch, rng, d, nc):
    As = [rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)) for k in d]
    D = int(d.sum())
    X = rng.standard_normal((D, nc)) + 1j * rng.standard_normal((D, nc))
    dA = torch.tensor(np.concatenate([a.T.ravel() for a in As]), device="cuda")
    dX = torch.tensor(np.ascontiguousarray(X.T), device="cuda")
    return As, X, dA, dX


def test_leaf_product_wait_runs_out_then_recovers():
    torch = torch_cuda()
    fds = fdslib()
    rng = np.random.default_rng(3)
    d = np.array([128, 64, 100], np.int32)
    As, X, dA, dX = _blocks(torch, rng, d, 70)
    fds.fds_fault_inject(fds.FDS_FAULT_TC_STALL_FW)
    dY = torch.zeros_like(dX)
    t0 = time.time()
    with pytest.raises(fds.FdsError) as e:
        fds.fds_zgemm_blocks_tc(d, dA, dX, dY)
    assert e.value.code == fds.FDS_ERR_TIMEOUT
    assert time.time() - t0 < 60
    # the device context is usable and the product right again
    dY = torch.zeros_like(dX)
    fds.fds_zgemm_blocks_tc(d, dA, dX, dY)
    got = dY.cpu().numpy().T
    off = np.concatenate([[0], np.cumsum(d)])
    for b, a in enumerate(As):
        r = slice(off[b], off[b + 1])
        assert np.abs(got[r] - a @ X[r]).max() <= 1e-11 * (np.abs(a) @ np.abs(X[r])).max()


def test_complex64_gemm_wait_runs_out_then_recovers():
    torch = torch_cuda()
    fds = fdslib()
    rng = np.random.default_rng(4)
    nb, d, n = 6, 96, 80
    A = (rng.standard_normal((nb, d, d)) + 1j * rng.standard_normal((nb, d, d))).astype(np.complex64)
    B = (rng.standard_normal((nb, d, n)) + 1j * rng.standard_normal((nb, d, n))).astype(np.complex64)
    aoff = np.arange(nb, dtype=np.int64) * d * d
    boff = np.arange(nb, dtype=np.int64) * d * n
    dA = torch.from_numpy(np.ascontiguousarray(A.transpose(0, 2, 1)).view(np.float32).ravel().copy()).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B.transpose(0, 2, 1)).view(np.float32).ravel().copy()).cuda()
    dC = torch.zeros(nb * d * n * 2, dtype=torch.float32, device="cuda")
    fds.fds_fault_inject(fds.FDS_FAULT_TC_STALL_C64)
    t0 = time.time()
    with pytest.raises(fds.FdsError) as e:
        fds.fds_cgemm_c64_batched([d] * nb, [n] * nb, [d] * nb, aoff, boff, boff, dA, dB, dC,
                                  engine=fds.FDS_C64_TENSOR)
    assert e.value.code == fds.FDS_ERR_TIMEOUT
    assert time.time() - t0 < 60
    dC.zero_()
    fds.fds_cgemm_c64_batched([d] * nb, [n] * nb, [d] * nb, aoff, boff, boff, dA, dB, dC, engine=fds.FDS_C64_TENSOR)
    got = dC.cpu().numpy().view(np.complex64).reshape(nb, n, d).transpose(0, 2, 1)
    ref = np.einsum("bij,bjk->bik", A.astype(np.complex128), B.astype(np.complex128))
    assert np.abs(got - ref).max() < 1e-5 * np.abs(ref).max()


def test_mixed_solve_reports_tensor_timeout_then_solves():
    torch_cuda()
    fds = fdslib()
    xy, omega = _problem()
    F, xref = _reference(fds, xy, omega)
    h = fds.fds_build(xy, omega, LAM, MU, 1e-8, precision=fds.FDS_MIXED, ir_tol=1e-9, fw_engine=fds.FDS_FW_TENSOR)
    fds.fds_fault_inject(fds.FDS_FAULT_TC_STALL_FW)
    with pytest.raises(fds.FdsError) as e:
        fds.fds_solve(h, F)
    assert e.value.code == fds.FDS_ERR_TIMEOUT
    # the same handle solves correctly afterwards
    x = fds.fds_solve(h, F)
    h.close()
    assert np.linalg.norm(x - xref) <= 1e-7 * np.linalg.norm(xref)


@pytest.mark.parametrize("spec,code", [("alloc:5", "FDS_ERR_OOM"), ("nan", "FDS_ERR_SINGULAR")])
def test_fault_from_environment(spec, code):
    # FDS_FAULT arms a fault at the first build of a fresh process; the
    # second build of that process is clean
    torch_cuda()
    fds = fdslib()
    import os
    import subprocess
    import sys
    prog = (
        "import numpy as np, workloads\n"
        "from paper_2411_18026_gb300 import fds\n"
        "xy = workloads.star(2048, 0.2, 5)\n"
        "om = workloads.omega_for_kTa(10.0)\n"
        "codes = []\n"
        "for _ in range(2):\n"
        "    try:\n"
        "        fds.fds_build(xy, om, 2.0, 1.0, 1e-8).close(); codes.append(0)\n"
        "    except fds.FdsError as e:\n"
        "        codes.append(e.code)\n"
        "print(codes)\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, FDS_FAULT=spec, PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""))
    out = subprocess.run([sys.executable, "-c", prog], env=env, cwd=root, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip().splitlines()[-1] == str([getattr(fds, code), 0])
