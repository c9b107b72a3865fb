"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

Holds none of the method's arithmetic: only boundary node coordinates of the
cavity shapes, material/frequency parameters and incident-wave angle lists.
Node order is counter-clockwise, uniform in the curve parameter theta.

Shapes
  circle:  r = a
  star:    r(theta) = 1 + e cos(m theta)                (default e=0.2, m=5)
  tripod:  the scatterer of the paper's numerical examples (Sec. 8, Fig.
           (tripod)): ((1 + 0.3 cos 3t) cos t, (1 + 0.3 cos 3t) sin t) / 1.3
  ellipse: semi-axes (aspect, 1) scaled to unit mean radius, rotated
"""
import numpy as np

SEED = 20241127


def circle(N, a=1.0):
    th = 2.0 * np.pi * np.arange(N) / N
    return np.stack([a * np.cos(th), a * np.sin(th)], 1)


def star(N, e=0.2, m=5, rot=0.0):
    th = 2.0 * np.pi * np.arange(N) / N
    r = 1.0 + e * np.cos(m * th)
    return np.stack([r * np.cos(th + rot), r * np.sin(th + rot)], 1)


def tripod(N, r=1.0, a=0.3, b=3):
    th = 2.0 * np.pi * np.arange(N) / N
    rr = r + a * np.cos(b * th)
    return np.stack([rr * np.cos(th) / (1 + a), rr * np.sin(th) / (1 + a)], 1)


def ellipse(N, aspect=2.0, rot=0.0):
    th = 2.0 * np.pi * np.arange(N) / N
    s = 1.0 / np.sqrt(aspect)
    x, y = aspect * s * np.cos(th), s * np.sin(th)
    c, d = np.cos(rot), np.sin(rot)
    return np.stack([c * x - d * y, d * x + c * y], 1)


def random_cavities(count, seed=SEED + 2, nmin_log2=12, nmax_log2=15, kta=(1.0, 20.0)):
    """Many-cavity workload: ellipses (aspect U[1,4], random rotation) or stars
    (e ~ U[0,0.3], m ~ U{3..8}), 50/50; node counts uniform in
    [2^nmin_log2, 2^nmax_log2]; k_T a uniform in kta.  Returns a list of dicts."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        N = int(rng.integers(1 << nmin_log2, (1 << nmax_log2) + 1))
        k = float(rng.uniform(*kta))
        if rng.random() < 0.5:
            asp = float(rng.uniform(1.0, 4.0))
            rot = float(rng.uniform(0, np.pi))
            out.append(dict(kind="ellipse", N=N, kTa=k, xy=ellipse(N, asp, rot)))
        else:
            e = float(rng.uniform(0.0, 0.3))
            m = int(rng.integers(3, 9))
            rot = float(rng.uniform(0, 2 * np.pi))
            out.append(dict(kind="star", N=N, kTa=k, xy=star(N, e, m, rot)))
    return out


def mlp_init(seed=SEED + 5, nin=16, nh=64):
    """Initial parameters of the learned-rank network (Glorot-uniform weights,
    zero biases) followed by an identity input normalisation (mu 0, sd 1):
    the flat layout W1, b1, W2, b2, w3, b3, mu, sd, float64."""
    rng = np.random.default_rng(seed)

    def glorot(fan_out, fan_in):
        a = np.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-a, a, (fan_out, fan_in))

    parts = [glorot(nh, nin).ravel(), np.zeros(nh), glorot(nh, nh).ravel(), np.zeros(nh), glorot(1, nh).ravel(),
             np.zeros(1), np.zeros(nin), np.ones(nin)]
    return np.concatenate(parts)


def minibatch_order(n, batch, epochs, seed=SEED + 6):
    """Sample order of minibatch training: per epoch a seeded permutation of
    range(n), truncated to whole batches."""
    rng = np.random.default_rng(seed)
    per = (n // batch) * batch
    return np.concatenate([rng.permutation(n)[:per] for _ in range(epochs)]).astype(np.int32)


def plane_wave_set(n_per_kind):
    """Alternating P (kind 0) and SV (kind 1) plane waves at uniform angles:
    returns (kinds[int32], angles[float64]) of length 2*n_per_kind."""
    th = 2.0 * np.pi * np.arange(n_per_kind) / n_per_kind
    kinds = np.tile(np.array([0, 1], dtype=np.int32), n_per_kind)
    angles = np.repeat(th, 2)
    return kinds, angles


def material(lam=2.0, mu=1.0, rho=1.0):
    return dict(lam=lam, mu=mu, rho=rho)


def omega_for_kTa(kTa, mu=1.0, rho=1.0, a=1.0):
    """omega with k_T a = kTa (c_T = sqrt(mu/rho))."""
    return kTa * np.sqrt(mu / rho) / a
