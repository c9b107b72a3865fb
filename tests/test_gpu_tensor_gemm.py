"""The batched complex64 GEMM of the mixed-precision levels on the tensor cores
(tcgen05, three bf16 pieces per operand) and on the FP32 pipe, against the complex128 product of
the same complex64 inputs; and the mixed solve with either engine."""
import numpy as np
import pytest

import workloads
from gpu_util import fdslib, torch_cuda

pytestmark = pytest.mark.gpu

# (m, n, k): single rows/columns, one and several 64-row tiles with ragged
# tails, N tails around the 128- and 256-column tiles, K of 0, below, at and
# above the 16-column stage
SHAPES = [(1, 1, 1), (64, 128, 16), (65, 129, 17), (128, 256, 32), (200, 300, 100), (37, 5, 256),
          (3, 260, 7), (130, 64, 0), (96, 1000, 128), (64, 17, 1)]


def _batch(shapes, opA, seed):
    rng = np.random.default_rng(seed)
    As, Bs, Cs = [], [], []
    for m, n, k in shapes:
        ar, ac = (k, m) if opA else (m, k)
        cplx = lambda r, c: (rng.standard_normal((r, c)) + 1j * rng.standard_normal((r, c))).astype(np.complex64)
        A = cplx(ar, ac)
        A *= np.exp(rng.uniform(-3, 3, (ar, 1))).astype(np.float32)   # rows of very different size
        As.append(A)
        Bs.append(cplx(k, n))
        Cs.append(cplx(m, n))
    return As, Bs, Cs


def _pack(mats):
    off, flat = [], []
    pos = 0
    for M in mats:
        off.append(pos)
        flat.append(np.asfortranarray(M).ravel(order="F"))
        pos += M.size
    return np.array(off, np.int64), np.concatenate(flat) if flat else np.zeros(0, np.complex64)


def _unpack(flat, off, shapes):
    return [flat[o:o + m * n].reshape((m, n), order="F") for o, (m, n) in zip(off, shapes)]


@pytest.mark.parametrize("engine", ["tensor", "simt"])
@pytest.mark.parametrize("opA,alpha,beta", [(0, 1.0, 0.0), (0, -1.0, 1.0), (2, 1.0, 1.0)])
def test_cgemm_matches_complex128_product(engine, opA, alpha, beta):
    torch = torch_cuda()
    fds = fdslib()
    eng = fds.FDS_C64_TENSOR if engine == "tensor" else fds.FDS_C64_SIMT
    As, Bs, Cs = _batch(SHAPES, opA, 7 + opA)
    aoff, af = _pack(As)
    boff, bf = _pack(Bs)
    coff, cf = _pack(Cs)
    dA = torch.from_numpy(af.view(np.float32).copy()).cuda()
    dB = torch.from_numpy(bf.view(np.float32).copy()).cuda()
    dC = torch.from_numpy(cf.view(np.float32).copy()).cuda()
    m = [s[0] for s in SHAPES]
    n = [s[1] for s in SHAPES]
    k = [s[2] for s in SHAPES]
    fds.fds_cgemm_c64_batched(m, n, k, aoff, boff, coff, dA, dB, dC, opA=opA, alpha=alpha, beta=beta, engine=eng)
    got = _unpack(dC.cpu().numpy().view(np.complex64), coff, [(a, b) for a, b, _ in SHAPES])
    for A, B, C, G in zip(As, Bs, Cs, got):
        opAm = A.astype(np.complex128)
        if opA:
            opAm = opAm.conj().T
        ref = alpha * (opAm @ B.astype(np.complex128)) + beta * C.astype(np.complex128)
        # bound: a few fp32 ulps of |op(A)| |B| (+ |C| for the update)
        scale = np.abs(opAm) @ np.abs(B.astype(np.complex128)) + abs(beta) * np.abs(C) + 1e-30
        err = np.abs(G - ref) / scale
        assert err.max() < 2e-6, (A.shape, B.shape, err.max())


def test_cgemm_tensor_agrees_with_simt_on_wide_batch():
    """Many entries of the sweep's leaf shape (128 x 128 times 128 x n)."""
    torch = torch_cuda()
    fds = fdslib()
    nb, d, n = 300, 128, 200
    rng = np.random.default_rng(11)
    A = (rng.standard_normal((nb, d, d)) + 1j * rng.standard_normal((nb, d, d))).astype(np.complex64)
    B = (rng.standard_normal((nb, d, n)) + 1j * rng.standard_normal((nb, d, n))).astype(np.complex64)
    aoff = np.arange(nb, dtype=np.int64) * d * d
    boff = np.arange(nb, dtype=np.int64) * d * n
    dA = torch.from_numpy(np.ascontiguousarray(A.transpose(0, 2, 1)).view(np.float32).ravel().copy()).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B.transpose(0, 2, 1)).view(np.float32).ravel().copy()).cuda()
    out = {}
    for name, eng in (("tensor", fds.FDS_C64_TENSOR), ("simt", fds.FDS_C64_SIMT)):
        dC = torch.zeros(nb * d * n * 2, dtype=torch.float32, device="cuda")
        fds.fds_cgemm_c64_batched([d] * nb, [n] * nb, [d] * nb, aoff, boff, boff, dA, dB, dC, engine=eng)
        out[name] = dC.cpu().numpy().view(np.complex64).reshape(nb, n, d).transpose(0, 2, 1)
    ref = np.einsum("bij,bjk->bik", A.astype(np.complex128), B.astype(np.complex128))
    scale = np.abs(ref).max()
    for name in out:
        assert np.abs(out[name] - ref).max() < 1e-5 * scale, name


@pytest.mark.parametrize("engine", ["tensor", "simt"])
def test_mixed_solve_either_engine(engine):
    """The mixed solve refines to the same answer with either complex64 engine."""
    torch_cuda()
    fdslib()
    from paper_2411_18026_gb300 import fds
    eng = fds.FDS_C64_TENSOR if engine == "tensor" else fds.FDS_C64_SIMT
    N = 4096
    xy = workloads.star(N)
    omega = workloads.omega_for_kTa(10.0)
    kinds, ang = workloads.plane_wave_set(4)
    h64 = fds.fds_build(xy, omega, 2.0, 1.0, 1e-9)
    F = fds.fds_rhs_plane_wave(h64, kinds, ang)
    x64 = fds.fds_solve(h64, F)
    h64.close()
    hm = fds.fds_build(xy, omega, 2.0, 1.0, 1e-9, precision=fds.FDS_MIXED, ir_tol=1e-10, c64_engine=eng,
                       merge_c64=True)
    xm = fds.fds_solve(hm, F)
    st = fds.fds_stats_get(hm)
    hm.close()
    err = np.linalg.norm(xm - x64, axis=0) / np.linalg.norm(x64, axis=0)
    assert err.max() < 1e-8, err.max()
    assert st.ir_iters <= 4
