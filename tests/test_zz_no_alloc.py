"""The allocation-free batched LU (fds_lu_batched_noalloc) gives the same
factors and pivots as fds_lu_batched, on two calls in a row.

It exists for callers that cannot allocate device memory when they call the
library (another allocator's callback, a device whose memory a caching
allocator has reserved, a loop that must not synchronise on cudaMalloc).
The file is named to run last in a test session."""
import numpy as np
import pytest

from gpu_util import dev, fdslib, torch_cuda

pytestmark = pytest.mark.gpu


def _batch(rng, sizes):
    As = [rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d)) for d in sizes]
    off = np.cumsum([0] + [d * d for d in sizes]).astype(np.int64)
    poff = np.cumsum([0] + list(sizes)).astype(np.int64)
    flat = np.concatenate([A.T.ravel() for A in As])
    return flat, off, poff


def _run(torch, fds, fn, flat, off, poff, sizes):
    dA = dev(torch, flat)
    piv = torch.zeros(int(poff[-1]), dtype=torch.int32, device="cuda")
    info = torch.full((len(sizes),), -1, dtype=torch.int32, device="cuda")
    fn(dev(torch, np.array(sizes, np.int32)), dev(torch, off), dA, piv, dev(torch, poff), info)
    torch.cuda.synchronize()
    return dA.cpu().numpy(), piv.cpu().numpy(), info.cpu().numpy()


def test_noalloc_lu_matches_allocating_lu_twice():
    torch = torch_cuda()
    fds = fdslib()
    rng = np.random.default_rng(11)
    for sizes in ([3, 64, 17, 128, 1], [40, 7, 96]):
        flat, off, poff = _batch(rng, sizes)
        ref, pref, iref = _run(torch, fds, fds.fds_lu_batched, flat, off, poff, sizes)
        got, pgot, igot = _run(torch, fds, fds.fds_lu_batched_noalloc, flat, off, poff, sizes)
        assert (iref == 0).all() and (igot == 0).all()
        assert (pgot == pref).all()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_noalloc_lu_rejects_oversized_batch():
    torch = torch_cuda()
    fds = fdslib()
    one = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert fds.lib().fds_lu_batched_noalloc(16385, one.data_ptr(), one.data_ptr(), one.data_ptr(),
                                            one.data_ptr(), one.data_ptr(), one.data_ptr(), 0) == fds.FDS_ERR_ARG
