"""Leaf diagonal blocks of the refinement's forward operator on the tensor
cores (fw_engine = FDS_FW_TENSOR: FP64 blocks and vectors cut into six bf16
slices, 21 slice products accumulated in tensor memory): the refined
solution is the FP64 solver's, on full and ragged leaves, as with the
double-float products it replaces."""
import numpy as np
import pytest

import workloads
from gpu_util import fdslib, torch_cuda

pytestmark = pytest.mark.gpu


def _colmax(a, b):
    return max(np.linalg.norm(a[:, c] - b[:, c]) / np.linalg.norm(b[:, c]) for c in range(b.shape[1]))


@pytest.mark.parametrize("nc", [1, 37, 130])
def test_stage_blocks_match_complex128_product(nc):
    # blocks of 1..128 complex rows, rows spanning 16 decades (per-row
    # exponents), columns of x spanning 8 decades (per-column exponents)
    torch = torch_cuda()
    fds = fdslib()
    rng = np.random.default_rng(41 + nc)
    d = np.array([128, 1, 64, 127, 3, 100, 128, 77], np.int32)
    As = [(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))) * np.logspace(-8, 8, k)[:, None]
          for k in d]
    D = int(d.sum())
    X = (rng.standard_normal((D, nc)) + 1j * rng.standard_normal((D, nc))) * np.logspace(-4, 4, nc)[None, :]
    Y0 = rng.standard_normal((D, nc)) + 1j * rng.standard_normal((D, nc))
    dA = torch.tensor(np.concatenate([a.T.ravel() for a in As]), device="cuda")   # column-major blocks
    dX = torch.tensor(np.ascontiguousarray(X.T), device="cuda")
    dY = torch.tensor(np.ascontiguousarray(Y0.T), device="cuda")
    fds.fds_zgemm_blocks_tc(d, dA, dX, dY)
    got = dY.cpu().numpy().T
    off = np.concatenate([[0], np.cumsum(d)])
    for b, a in enumerate(As):
        r = slice(off[b], off[b + 1])
        prod = a @ X[r]
        scale = np.abs(a) @ np.abs(X[r])            # |A| |x| per entry
        # six 8-bit slices and exact accumulators for the pairs with i + j <= 2:
        # below ~2^-38 of |A| |x|; the float-pair y holds the sum to ~2^-46 of itself
        bound = 2e-11 * scale + 4e-14 * np.abs(Y0[r] + prod)
        excess = np.abs(got[r] - Y0[r] - prod) / bound
        assert excess.max() <= 1.0, (b, excess.max())


@pytest.mark.parametrize("N,leaf,nw", [(8192, 64, 3), (3000, 64, 2), (2048, 40, 140)])
def test_tensor_forward_operator_refines_to_fp64(N, leaf, nw):
    # full 64-node leaves; ragged leaves of 46-47 nodes; 40-node leaves and
    # 280 waves (a full 256-column chunk plus a ragged one, two column tiles)
    torch_cuda()
    fds = fdslib()
    xy = workloads.star(N, 0.2, 5, rot=0.2)
    omega = workloads.omega_for_kTa(10.0)
    kinds, ang = workloads.plane_wave_set(nw)
    h64 = fds.fds_build(xy, omega, 2.0, 1.0, 1e-9, leaf_size=leaf)
    F = fds.fds_rhs_plane_wave(h64, kinds, ang)
    x64 = fds.fds_solve(h64, F)
    h64.close()
    out = {}
    for eng in (fds.FDS_FW_FF, fds.FDS_FW_TENSOR):
        h = fds.fds_build(xy, omega, 2.0, 1.0, 1e-9, leaf_size=leaf, precision=fds.FDS_MIXED, ir_tol=1e-9,
                          fw_engine=eng)
        x = fds.fds_solve(h, F)
        st = fds.fds_stats_get(h)
        out[eng] = (x, st.ir_iters, st.ir_residual)
        h.close()
    xt, it_t, res_t = out[fds.FDS_FW_TENSOR]
    xf, it_f, res_f = out[fds.FDS_FW_FF]
    assert res_t <= 1e-9 and res_f <= 1e-9
    assert abs(it_t - it_f) <= 1
    assert _colmax(xt, x64) < 1e-8
    assert _colmax(xt, xf) < 1e-8
