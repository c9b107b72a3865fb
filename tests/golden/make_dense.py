"""Write the dense-oracle solutions that the GPU parity tests at 2^12 and 2^13
nodes compare against (too slow to assemble inside every GPU test run).

Calls only the oracle ("Conv" of Sec. 8: dense Galerkin assembly of
A = D + I_0/2 + alpha N and partial-pivot LU, Sec. 4) on seeded star cavities
r = 1 + 0.2 cos 5t (lambda = 2, mu = 1, rho = 1) with one plane P wave
(angle 0.3) and one plane SV wave (angle 1.9).  Output per case:
dense_star_N<nodes>_kta<kTa>.npz with x, the dense solution (2N x 2,
complex128) for the load vectors F = load_vectors(N, kTa).

python tests/golden/make_dense.py [N:kTa ...]    (default: the four cases)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from oracle import bem  # noqa: E402

CASES = [(4096, 10.0), (4096, 20.0), (8192, 10.0), (8192, 20.0)]
WAVES = [(0, 0.3), (1, 1.9)]


def path(N, kta):
    return os.path.join(HERE, "dense_star_N%d_kta%d.npz" % (N, int(kta)))


def load_vectors(N, kta):
    """The oracle's Galerkin load vectors of the two waves (2N x 2)."""
    P = bem.phys(2.0, 1.0, 1.0, workloads.omega_for_kTa(kta))
    xy = workloads.star(N)
    return np.stack([bem.rhs(P, xy, k, a) for k, a in WAVES], 1)


def make(N, kta):
    xy = workloads.star(N)
    P = bem.phys(2.0, 1.0, 1.0, workloads.omega_for_kTa(kta))
    F = load_vectors(N, kta)
    t = time.time()
    x = bem.dense_solve(P, xy, F)
    np.savez(path(N, kta), x=x)
    print("N=%d kTa=%g: %.1f s" % (N, kta, time.time() - t), flush=True)


if __name__ == "__main__":
    cases = [(int(a.split(":")[0]), float(a.split(":")[1])) for a in sys.argv[1:]] or CASES
    for N, kta in cases:
        make(N, kta)
