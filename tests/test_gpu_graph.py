"""CUDA-graph replay of the solve sweep (use_graph): the replayed sweeps give
the solutions of the launch-by-launch sweep, with far fewer host launches,
for FP64 and mixed-precision handles on their own streams (batched builds)
and on a caller's stream."""
import numpy as np
import pytest

import workloads
from gpu_util import fdslib, torch_cuda

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_sweeps_equal_plain_sweeps_batched(precision):
    torch = torch_cuda()
    fds = fdslib()
    cav = workloads.random_cavities(3, seed=workloads.SEED + 31, nmin_log2=11, nmax_log2=12, kta=(2.0, 8.0))
    for c in cav:
        c["omega"] = workloads.omega_for_kTa(c["kTa"])
    kinds, ang = workloads.plane_wave_set(4)
    plain = fds.fds_build_batch(cav, 2.0, 1.0, 1e-9, n_streams=3, precision=precision)
    graph = fds.fds_build_batch(cav, 2.0, 1.0, 1e-9, n_streams=3, precision=precision, use_graph=True)
    # two builds agree to rounding only (atomic sums in the kernel evaluation)
    tol = 1e-11 if precision == 0 else 1e-9
    for hp, hg in zip(plain, graph):
        F = fds.fds_rhs_plane_wave(hp, kinds, ang)
        xp = fds.fds_solve(hp, F)
        dg = [torch.tensor(np.ascontiguousarray(F.T), device="cuda") for _ in range(3)]
        counts = []
        for d in dg:                      # 1st: plain run + capture; 2nd, 3rd: replay
            n0 = fds.fds_launch_count()
            fds.fds_solve_batch([hg], [d], n_streams=1)
            counts.append(fds.fds_launch_count() - n0)
        for d in dg:
            assert _rel(d.cpu().numpy().T, xp) <= tol
        if precision == 0:   # the same graph replayed: the same FP64 result, bit for bit
            assert torch.equal(dg[1], dg[2]) and torch.equal(dg[0], dg[1])
        # (mixed: the refinement's forward operator still launches kernel by kernel)
        assert counts[2] < (0.25 if precision == 0 else 0.8) * counts[0], counts
    for h in plain + graph:
        h.close()


def test_graph_on_a_caller_stream_and_stream_zero_fallback():
    torch = torch_cuda()
    fds = fdslib()
    xy = workloads.star(2048)
    omega = workloads.omega_for_kTa(6.0)
    st = torch.cuda.Stream()
    hg = fds.fds_build(xy, omega, 2.0, 1.0, 1e-9, stream=st, use_graph=True)
    h0 = fds.fds_build(xy, omega, 2.0, 1.0, 1e-9, use_graph=True)   # legacy stream: no capture, plain sweeps
    F = fds.fds_rhs_plane_wave(h0, np.array([0, 1], np.int32), np.array([0.2, 1.4]))
    x0 = fds.fds_solve(h0, F)
    prev = None
    for _ in range(3):
        d = torch.tensor(np.ascontiguousarray(F.T), device="cuda")
        torch.cuda.synchronize()
        fds.fds_solve_device(hg, d, st)
        st.synchronize()
        assert _rel(d.cpu().numpy().T, x0) <= 1e-11
        if prev is not None:
            assert torch.equal(d, prev)
        prev = d
    hg.close()
    h0.close()
