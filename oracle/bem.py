"""ORACLE — test infrastructure only: dense Galerkin BEM of arXiv 2411.18026.

Thin ctypes front end over ``galerkin.c`` plus the dense solve the paper calls
"Conv" (Sec. 8): assemble the 2N x 2N matrix A = D + I_0/2 + alpha N entry by
entry (Sec. 4), the load vector f (Sec. 4, eq. (gal)), and solve A x = f by
partial-pivot LU (numpy/LAPACK).  The unknown layout is the component-blocked
one of eq. (discre_x): x = (u_1 at nodes 0..N-1, u_2 at nodes 0..N-1).
"""
import ctypes
import numpy as np

from . import build as _build

_lib = None


class Phys(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_double), ("mu", ctypes.c_double), ("rho", ctypes.c_double),
                ("omega", ctypes.c_double), ("alpha_re", ctypes.c_double),
                ("alpha_im", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        P = ctypes.POINTER(Phys)
        _lib.orc_entries.argtypes = [P, dp, ctypes.c_int, ip, ctypes.c_int, ip, ctypes.c_int, dp]
        _lib.orc_cross_entries.argtypes = [P, dp, ctypes.c_int, ip, ctypes.c_int, dp, ctypes.c_int,
                                           ip, ctypes.c_int, ctypes.c_int, dp]
        _lib.orc_rhs.argtypes = [P, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
        _lib.orc_kernel_blocks.argtypes = [P, dp, dp, dp, dp]
        _lib.orc_ehat.argtypes = [ctypes.c_double, dp]
        _lib.orc_pair.argtypes = [P, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        _lib.orc_field.argtypes = [P, dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_double, dp, ctypes.c_int, dp]
        for f in ("orc_entries", "orc_cross_entries", "orc_rhs", "orc_kernel_blocks", "orc_ehat",
                  "orc_pair", "orc_field"):
            getattr(_lib, f).restype = None
    return _lib


def default_alpha(mu, omega, rho=1.0):
    """Burton–Miller coupling alpha = i / (mu k_T): the paper leaves alpha open
    (Sec. 3); uniqueness needs Im(alpha) != 0 and alpha scales as length/mu."""
    kT = omega / np.sqrt(mu / rho)
    return 1j / (mu * kT)


def phys(lam, mu, rho, omega, alpha=None):
    if alpha is None:
        alpha = default_alpha(mu, omega, rho)
    return Phys(lam, mu, rho, omega, float(np.real(alpha)), float(np.imag(alpha)))


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def entries(P, xy, rows, cols):
    """A(rows, cols) on the closed polygon xy (N x 2, counter-clockwise).
    Returns (2 len(rows)) x (2 len(cols)) complex, component-blocked."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.zeros((2 * len(rows), 2 * len(cols)), dtype=np.complex128)
    if len(rows) and len(cols):
        lib().orc_entries(ctypes.byref(P), _dp(xy), len(xy), _ip(rows), len(rows), _ip(cols),
                          len(cols), _dp(out.view(np.float64)))
    return out


def cross_entries(P, X, rows, Y, cols, q=4):
    """Entries between test hats rows[] on polygon X and trial hats cols[] on
    polygon Y (both closed, counter-clockwise), fixed q x q Gauss, no mass."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.zeros((2 * len(rows), 2 * len(cols)), dtype=np.complex128)
    if len(rows) and len(cols):
        lib().orc_cross_entries(ctypes.byref(P), _dp(X), len(X), _ip(rows), len(rows), _dp(Y),
                                len(Y), _ip(cols), len(cols), int(q), _dp(out.view(np.float64)))
    return out


def rhs(P, xy, kind, theta):
    """Galerkin load vector for a plane P (kind 0) or SV (kind 1) wave."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    out = np.zeros(2 * len(xy), dtype=np.complex128)
    lib().orc_rhs(ctypes.byref(P), _dp(xy), len(xy), int(kind), float(theta),
                  _dp(out.view(np.float64)))
    return out


def field(P, xy, u, kind, theta, pts):
    """Displacement at points off the boundary (Sec. 3, eq. (integ_rep)) from
    the boundary solution u (2N complex) of a plane P (kind 0) or SV (kind 1)
    wave.  pts: (npts, 2).  Returns (2, npts) complex."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.complex128)
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    out = np.zeros(2 * len(pts), dtype=np.complex128)
    lib().orc_field(ctypes.byref(P), _dp(xy), len(xy), _dp(u.view(np.float64)), int(kind), float(theta),
                    _dp(pts), len(pts), _dp(out.view(np.float64)))
    return out.reshape(2, len(pts))


def kernel_blocks(P, z, nx, ny):
    """The four 2x2 regularised kernel blocks at one point pair."""
    out = np.zeros((4, 2, 2), dtype=np.complex128)
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (z, nx, ny)]
    lib().orc_kernel_blocks(ctypes.byref(P), _dp(a[0]), _dp(a[1]), _dp(a[2]),
                            _dp(out.view(np.float64)))
    return out


def ehat(z):
    out = np.zeros(2)
    lib().orc_ehat(float(z), _dp(out))
    return out[0] + 1j * out[1]


def pair(P, xy, ie, jf):
    """Element-pair integral I[A][B][i][j] under the project's quadrature rule."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    out = np.zeros((2, 2, 2, 2), dtype=np.complex128)
    lib().orc_pair(ctypes.byref(P), _dp(xy), len(xy), int(ie), int(jf), _dp(out.view(np.float64)))
    return out


def dense_matrix(P, xy):
    n = len(xy)
    idx = np.arange(n, dtype=np.int32)
    return entries(P, xy, idx, idx)


def dense_solve(P, xy, F):
    """'Conv' of Sec. 8: dense assembly + partial-pivot LU solve.  F: (2N,) or
    (2N, nrhs) load vectors; returns the nodal displacements, same layout."""
    A = dense_matrix(P, xy)
    return np.linalg.solve(A, F)
