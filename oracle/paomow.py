"""ORACLE — test infrastructure only: series solution for a traction-free
circular cavity of radius a under a plane P or SV wave (Pao–Mow type).

Derived here from the Navier equation of Sec. 2 in polar coordinates (time
factor exp(-i w t), matching H^(1) in eq. (funda)): u = grad phi + curl(psi e3),
phi = sum_n f_n(r) e^{in th}, psi = sum_n g_n(r) e^{in th} with Bessel/Hankel
radial parts; sigma_rr = sigma_rth = 0 at r = a gives a 2x2 system per order n:
  sigma_rr  = mu [ -kT^2 f - 2 f'/r + 2 n^2 f / r^2 + 2 i n (g'/r - g/r^2) ]
  sigma_rth = mu [ 2 i n (f'/r - f/r^2) + 2 g'/r + (kT^2 - 2 n^2/r^2) g ]
  u_r = f' + (i n / r) g,  u_th = (i n / r) f - g'.
Incident P: u^I = d exp(i kL d.x) (phi^I = exp(i kL d.x)/(i kL));
incident SV: u^I = d_perp exp(i kT d.x) (psi^I = (i/kT) exp(i kT d.x)),
d = (cos th0, sin th0), d_perp = (-sin th0, cos th0).
"""
import numpy as np
from scipy.special import jv, jvp, hankel1, h1vp


def _wavenumbers(lam, mu, rho, omega):
    return omega / np.sqrt((lam + 2 * mu) / rho), omega / np.sqrt(mu / rho)


def _incident(n, kind, theta0, kL, kT, r):
    ph = np.exp(-1j * n * theta0)
    if kind == 0:
        cf = (1j ** n) * ph / (1j * kL)
        return cf * jv(n, kL * r), cf * kL * jvp(n, kL * r), 0.0 * r, 0.0 * r
    cg = (1j / kT) * (1j ** n) * ph
    return 0.0 * r, 0.0 * r, cg * jv(n, kT * r), cg * kT * jvp(n, kT * r)


def coefficients(a, lam, mu, rho, omega, kind=0, theta0=0.0, nmax=None):
    kL, kT = _wavenumbers(lam, mu, rho, omega)
    if nmax is None:
        nmax = int(np.ceil(kT * a)) + 30
    coef = {}
    r = a
    for n in range(-nmax, nmax + 1):
        fI, fIp, gI, gIp = _incident(n, kind, theta0, kL, kT, r)
        HL, HLp = hankel1(n, kL * r), kL * h1vp(n, kL * r)
        HT, HTp = hankel1(n, kT * r), kT * h1vp(n, kT * r)

        def srr(f, fp, g, gp):
            return mu * (-kT ** 2 * f - 2 * fp / r + 2 * n * n * f / r ** 2 + 2j * n * (gp / r - g / r ** 2))

        def srt(f, fp, g, gp):
            return mu * (2j * n * (fp / r - f / r ** 2) + 2 * gp / r + (kT ** 2 - 2 * n * n / r ** 2) * g)

        M = np.array([[srr(HL, HLp, 0, 0), srr(0, 0, HT, HTp)],
                      [srt(HL, HLp, 0, 0), srt(0, 0, HT, HTp)]])
        b = -np.array([srr(fI, fIp, gI, gIp), srt(fI, fIp, gI, gIp)])
        coef[n] = np.linalg.solve(M, b)
    return coef


def field(r, th, a, lam, mu, rho, omega, kind=0, theta0=0.0, nmax=None, coef=None):
    """Total displacement (u1, u2) at polar points (r >= a, th).  By default the
    series runs to |n| = ceil(k_T max(a, r)) + 30: the incident wave's
    Bessel expansion at radius r needs orders beyond k r."""
    kL, kT = _wavenumbers(lam, mu, rho, omega)
    if coef is None:
        if nmax is None:
            nmax = int(np.ceil(kT * max(a, float(np.max(r))))) + 30
        coef = coefficients(a, lam, mu, rho, omega, kind, theta0, nmax)
    r = np.asarray(r, dtype=np.float64) * np.ones_like(np.asarray(th, dtype=np.float64))
    th = np.asarray(th, dtype=np.float64) * np.ones_like(r)
    ur = np.zeros(r.shape, dtype=np.complex128)
    ut = np.zeros(r.shape, dtype=np.complex128)
    for n, (A, B) in coef.items():
        fI, fIp, gI, gIp = _incident(n, kind, theta0, kL, kT, r)
        f = fI + A * hankel1(n, kL * r)
        fp = fIp + A * kL * h1vp(n, kL * r)
        g = gI + B * hankel1(n, kT * r)
        gp = gIp + B * kT * h1vp(n, kT * r)
        e = np.exp(1j * n * th)
        ur += (fp + 1j * n / r * g) * e
        ut += (1j * n / r * f - gp) * e
    return ur * np.cos(th) - ut * np.sin(th), ur * np.sin(th) + ut * np.cos(th)


def boundary_displacement(theta_pts, a, lam, mu, rho, omega, kind=0, theta0=0.0, nmax=None):
    return field(a, theta_pts, a, lam, mu, rho, omega, kind, theta0, nmax)
