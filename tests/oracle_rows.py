"""Worker for the full-size residual test: full rows of the oracle's Galerkin
matrix, one node (both components) per call, run in spawned processes."""
import numpy as np

from oracle import bem


def node_rows(args):
    lam, mu, rho, omega, xy, node = args
    P = bem.phys(lam, mu, rho, omega)
    n = len(xy)
    return node, bem.entries(P, xy, np.array([node], np.int32), np.arange(n, dtype=np.int32))
