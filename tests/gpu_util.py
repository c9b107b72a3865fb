"""Helpers for the GPU tests: build/load the CUDA library, move arrays."""
import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def fdslib():
    from paper_2411_18026_gb300 import build
    build.build()
    from paper_2411_18026_gb300 import fds
    fds.lib()
    return fds


def dev(torch, a, dtype=None):
    a = np.ascontiguousarray(a)
    t = torch.from_numpy(a)
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()
