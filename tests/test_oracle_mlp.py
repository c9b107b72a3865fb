"""Pins of the learned-rank network oracle (oracle/mlp.py): closed-form
forward values, central finite differences for the gradient, Adam's
bias-corrected first step, and descent on a learnable target."""
import numpy as np

from oracle import mlp


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, scale, mlp.NPARAM)
    q = mlp.unpack(p)
    q["mu"][:] = rng.normal(0.0, 1.0, mlp.NIN)
    q["sd"][:] = rng.uniform(0.5, 2.0, mlp.NIN)
    return p


def test_layout_sizes():
    assert mlp.NTRAIN == 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1
    assert mlp.NPARAM == mlp.NTRAIN + 32


def test_forward_closed_form():
    # W1 = first 16 unit rows, W2 = identity, w3 = e_0: y = tanh(tanh(u_0)) + b3
    p = np.zeros(mlp.NPARAM)
    q = mlp.unpack(p)
    for i in range(16):
        q["W1"][i, i] = 1.0
    q["W2"][:] = np.eye(64)
    q["w3"][0] = 1.0
    q["b3"][0] = 0.25
    q["sd"][:] = 2.0
    q["mu"][:] = 1.0
    X = np.array([[3.0] + [0.0] * 15, [-1.0] + [5.0] * 15])
    y, _ = mlp.forward(p, X)
    u0 = (X[:, 0] - 1.0) / 2.0
    assert np.allclose(y, np.tanh(np.tanh(u0)) + 0.25, rtol=0, atol=1e-15)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(7)
    p = _params(3)
    X = rng.normal(0.0, 1.5, (9, mlp.NIN))
    t = rng.uniform(0.0, 1.0, 9)
    L, g = mlp.loss_grad(p, X, t)
    # every parameter block, several entries each
    o = 0
    for name, n in mlp.SIZES:
        for k in sorted(set([o, o + n // 2, o + n - 1])):
            h = 1e-6
            pp, pm = p.copy(), p.copy()
            pp[k] += h
            pm[k] -= h
            fd = (mlp.loss_grad(pp, X, t)[0] - mlp.loss_grad(pm, X, t)[0]) / (2 * h)
            assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])), (name, k, fd, g[k])
        o += n
    assert g.shape == (mlp.NTRAIN,)
    assert L > 0


def test_adam_first_step_has_magnitude_lr():
    # bias correction makes the first step lr * g / (|g| + eps) per coordinate
    p = _params(5)
    g = np.linspace(-2.0, 3.0, mlp.NTRAIN)
    g[g == 0] = 1.0
    p1, m, v = mlp.adam(p, g, np.zeros(mlp.NTRAIN), np.zeros(mlp.NTRAIN), 1, 0.01)
    step = p[:mlp.NTRAIN] - p1[:mlp.NTRAIN]
    assert np.allclose(step, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    assert np.array_equal(p1[mlp.NTRAIN:], p[mlp.NTRAIN:])     # normalisation untouched


def test_training_fits_a_smooth_target():
    rng = np.random.default_rng(11)
    X = rng.normal(0.0, 1.0, (256, mlp.NIN))
    t = 0.5 + 0.3 * np.tanh(X[:, 0] - 0.5 * X[:, 3])
    p = _params(13, scale=0.1)
    q = mlp.unpack(p)
    q["mu"][:] = 0.0
    q["sd"][:] = 1.0
    order = np.concatenate([rng.permutation(256) for _ in range(40)])
    p2, losses = mlp.train(p, X, t, order, 32, 3e-3)
    assert losses[-20:].mean() < 0.05 * losses[:5].mean()
    # deterministic given the order
    p3, _ = mlp.train(p, X, t, order, 32, 3e-3)
    assert np.array_equal(p2, p3)
