"""Direct (unregularised) elastodynamic kernels for the oracle pins.

Written straight from eq. (funda) and the traction operator of Sec. 2:
G_kl(z) = i/(4 mu) [H0(kT r) d_kl + kT^-2 d_k d_l (H0(kT r) - H0(kL r))],
double-layer kernel K^D_ij = C_jpkq n^y_p d_q G_ik(z) and hypersingular kernel
K^N_ij = -C_iakb C_jplq n^x_a n^y_p d_b d_q G_kl(z), with z = y - x.  Radial
derivatives use (r^-1 d/dr)^m H0(kr) = (-k/r)^m H_m(kr).
"""
import numpy as np
from scipy.special import hankel1

D2 = np.eye(2)


def elastic_tensor(lam, mu):
    C = np.zeros((2, 2, 2, 2))
    for i in range(2):
        for p in range(2):
            for j in range(2):
                for q in range(2):
                    C[i, p, j, q] = lam * D2[i, p] * D2[j, q] + mu * (D2[i, j] * D2[p, q] + D2[i, q] * D2[p, j])
    return C


def radial_derivs(k, z):
    """H0(k|z|) and its Cartesian derivative tensors of order 1..4."""
    r = np.linalg.norm(z)
    Dm = [(-k / r) ** m * hankel1(m, k * r) for m in range(5)]
    d = D2
    f1 = z * Dm[1]
    f2 = d * Dm[1] + np.outer(z, z) * Dm[2]
    f3 = np.zeros((2, 2, 2), complex)
    f4 = np.zeros((2, 2, 2, 2), complex)
    for a in range(2):
        for b in range(2):
            for c in range(2):
                f3[a, b, c] = (d[a, b] * z[c] + d[a, c] * z[b] + d[b, c] * z[a]) * Dm[2] + z[a] * z[b] * z[c] * Dm[3]
                for e in range(2):
                    f4[a, b, c, e] = ((d[a, b] * d[c, e] + d[a, c] * d[b, e] + d[a, e] * d[b, c]) * Dm[2]
                                      + (d[a, b] * z[c] * z[e] + d[a, c] * z[b] * z[e] + d[a, e] * z[b] * z[c]
                                         + d[b, c] * z[a] * z[e] + d[b, e] * z[a] * z[c] + d[c, e] * z[a] * z[b]) * Dm[3]
                                      + z[a] * z[b] * z[c] * z[e] * Dm[4])
    return Dm[0], f1, f2, f3, f4


def wavenumbers(lam, mu, rho, omega):
    return omega / np.sqrt((lam + 2 * mu) / rho), omega / np.sqrt(mu / rho)


def G_tensors(lam, mu, rho, omega, z):
    kL, kT = wavenumbers(lam, mu, rho, omega)
    T = radial_derivs(kT, z)
    L = radial_derivs(kL, z)
    a = 1j / (4 * mu)
    G = a * (T[0] * D2 + (T[2] - L[2]) / kT ** 2)
    G1 = a * (np.einsum('kl,q->klq', D2, T[1]) + (T[3] - L[3]) / kT ** 2)
    G2 = a * (np.einsum('kl,bq->klbq', D2, T[2]) + (T[4] - L[4]) / kT ** 2)
    return G, G1, G2


def KD(lam, mu, rho, omega, z, ny):
    C = elastic_tensor(lam, mu)
    _, G1, _ = G_tensors(lam, mu, rho, omega, z)
    return np.einsum('jpkq,p,ikq->ij', C, ny, G1)


def KN(lam, mu, rho, omega, z, nx, ny):
    C = elastic_tensor(lam, mu)
    _, _, G2 = G_tensors(lam, mu, rho, omega, z)
    return -np.einsum('iakb,jplq,a,p,klbq->ij', C, C, nx, ny, G2)
