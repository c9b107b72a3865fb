"""Interior Dirichlet eigenfrequencies of an elastic disk (closed form), the
fictitious frequencies of the direct boundary integral equation without the
Burton–Miller term (Sec. 8.4, eq. (bie_non_bie)).

Derivation (Navier equation of Sec. 2 inside the disk r < a, potentials
u = grad phi + curl(psi e3), phi = A J_n(k_L r) e^{in th},
psi = B J_n(k_T r) e^{in th}, regular at r = 0):
  u_r(a)  = A k_L J_n'(k_L a) + B (i n / a) J_n(k_T a)
  u_th(a) = A (i n / a) J_n(k_L a) - B k_T J_n'(k_T a)
u = 0 on r = a has a nonzero solution when the 2 x 2 determinant vanishes:
  det_n(omega) = (n / a)^2 J_n(k_L a) J_n(k_T a) - k_L k_T J_n'(k_L a) J_n'(k_T a).
At such an omega the traction t of the eigenfunction gives a single-layer
potential that vanishes outside the cavity, so I/2 + D (the operator of
eq. (bie_non_bie) for the exterior) is singular there as well.
"""
import numpy as np
from scipy.optimize import brentq
from scipy.special import jv, jvp


def det(n, omega, lam=2.0, mu=1.0, rho=1.0, a=1.0):
    kL, kT = omega / np.sqrt((lam + 2 * mu) / rho), omega / np.sqrt(mu / rho)
    return (n / a) ** 2 * jv(n, kL * a) * jv(n, kT * a) - kL * kT * jvp(n, kL * a) * jvp(n, kT * a)


def eigenfrequencies(omega_max, lam=2.0, mu=1.0, rho=1.0, a=1.0, nmax=12, step=1e-3):
    """All interior Dirichlet eigenfrequencies in (0, omega_max] with their
    order n >= 0 (orders +-n give the same omega), sorted by omega."""
    out = []
    w = np.arange(step, omega_max + step, step)
    for n in range(nmax + 1):
        d = det(n, w, lam, mu, rho, a)
        for i in np.nonzero(np.sign(d[:-1]) * np.sign(d[1:]) < 0)[0]:
            out.append((brentq(lambda x: det(n, x, lam, mu, rho, a), w[i], w[i + 1], xtol=1e-13), n))
    return sorted(out)
