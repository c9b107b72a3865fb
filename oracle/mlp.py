"""Oracle for the learned-rank predictor: a 16 -> 64 -> 64 -> 1 perceptron
with tanh hidden units, mean-squared-error loss and Adam updates, in float64
numpy with plain loops over the layers.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline may import this module.

The network predicts, for one (cell, component) of a tree level, the
fraction k / n of the component's DOFs that the interpolative decomposition
keeps (Sec. 7.2 rank); the CUDA training and inference kernels are checked
against this restatement.  Parameter layout (flat float vector, the same on
both sides):

    W1 [64 x 16] row-major | b1 [64] | W2 [64 x 64] | b2 [64] | w3 [64] | b3 [1]
    followed by the (untrained) input normalisation mu [16] | sd [16]

Forward:  u = (x - mu) / sd,  h1 = tanh(W1 u + b1),  h2 = tanh(W2 h1 + b2),
          y = w3 . h2 + b3.
Loss:     L = (1/B) sum_b (y_b - t_b)^2 over a batch.
Adam (Kingma & Ba 2015, Algorithm 1): m <- b1 m + (1-b1) g,
          v <- b2 v + (1-b2) g^2, p <- p - lr (m / (1-b1^s)) / (sqrt(v / (1-b2^s)) + eps).
"""
import numpy as np

NIN, NH = 16, 64
SIZES = [("W1", NH * NIN), ("b1", NH), ("W2", NH * NH), ("b2", NH), ("w3", NH), ("b3", 1)]
NTRAIN = sum(n for _, n in SIZES)          # trained parameters
NPARAM = NTRAIN + 2 * NIN                  # + normalisation


def unpack(p):
    """Views of the parameter vector by name."""
    out, o = {}, 0
    for name, n in SIZES:
        out[name] = p[o:o + n]
        o += n
    out["mu"] = p[o:o + NIN]
    out["sd"] = p[o + NIN:o + 2 * NIN]
    out["W1"] = out["W1"].reshape(NH, NIN)
    out["W2"] = out["W2"].reshape(NH, NH)
    return out


def forward(p, X):
    """Predictions y[B] and the hidden activations for a batch X[B, 16]."""
    q = unpack(np.asarray(p, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    U = (X - q["mu"]) / q["sd"]
    H1 = np.tanh(U @ q["W1"].T + q["b1"])
    H2 = np.tanh(H1 @ q["W2"].T + q["b2"])
    y = H2 @ q["w3"] + q["b3"][0]
    return y, (U, H1, H2)


def loss_grad(p, X, t):
    """Mean-squared-error loss and its gradient with respect to the trained
    parameters (back-propagation through the two tanh layers)."""
    q = unpack(np.asarray(p, dtype=np.float64))
    y, (U, H1, H2) = forward(p, X)
    B = len(y)
    r = y - np.asarray(t, dtype=np.float64)
    L = float(np.mean(r * r))
    dy = 2.0 * r / B                              # dL/dy
    g_w3 = H2.T @ dy
    g_b3 = np.array([dy.sum()])
    dH2 = np.outer(dy, q["w3"]) * (1.0 - H2 * H2)  # through tanh
    g_W2 = dH2.T @ H1
    g_b2 = dH2.sum(0)
    dH1 = (dH2 @ q["W2"]) * (1.0 - H1 * H1)
    g_W1 = dH1.T @ U
    g_b1 = dH1.sum(0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, g_b3])
    return L, g


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update of the trained parameters (step counts from 1)."""
    p = np.array(p, dtype=np.float64)
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    p[:NTRAIN] -= lr * mh / (np.sqrt(vh) + eps)
    return p, m, v


def train(p, X, t, order, batch, lr):
    """Minibatch Adam over the sample order given (a flat index list whose
    length is a multiple of the batch size); returns parameters and the loss
    of every step."""
    p = np.array(p, dtype=np.float64)
    m = np.zeros(NTRAIN)
    v = np.zeros(NTRAIN)
    losses = []
    for s in range(len(order) // batch):
        idx = order[s * batch:(s + 1) * batch]
        L, g = loss_grad(p, X[idx], t[idx])
        p, m, v = adam(p, g, m, v, s + 1, lr)
        losses.append(L)
    return p, np.array(losses)
