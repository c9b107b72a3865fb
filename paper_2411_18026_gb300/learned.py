"""Training data and training of the learned skeleton-rank network through the
library's C ABI (marshalling only: features come from the build kernels, the
gradient and Adam steps from the library's training kernels).

collect(cavities, ...)   -> features [rows, 16] (float32), rank fractions [rows]
train(features, fracs)   -> parameter vector (FDS_MLP_NPARAM float32) for
                            fds_build(..., mlp_params=...)
"""
import numpy as np

from . import fds


def collect(cavities, tol, leaf_size=64, lam=2.0, mu=1.0, rho=1.0):
    """Build every cavity (dicts with 'xy' and 'kTa') with the adaptive ID and
    return the recorded features and k / n of every (cell, component)."""
    feats, fracs = [], []
    for c in cavities:
        omega = c["kTa"] * np.sqrt(mu / rho)
        h = fds.fds_build(c["xy"], omega, lam, mu, tol, rho=rho, leaf_size=leaf_size, record_features=True)
        f, r = fds.fds_features_get(h)
        h.close()
        feats.append(f)
        fracs.append(r)
    return np.concatenate(feats), np.concatenate(fracs)


def train(features, fracs, init, order, batch=256, lr=2e-3, stream=None):
    """Adam training on the GPU.  init: initial parameters (its normalisation
    part is replaced by the features' mean and standard deviation); order:
    minibatch sample order (see workloads.minibatch_order).  Returns
    (parameters float32, per-step losses)."""
    import torch
    p = np.array(init, dtype=np.float64)
    mu = features.mean(0)
    sd = features.std(0)
    sd[sd < 1e-6] = 1.0
    p[fds.FDS_MLP_NTRAIN:fds.FDS_MLP_NTRAIN + 16] = mu
    p[fds.FDS_MLP_NTRAIN + 16:] = sd
    d_p = torch.tensor(p, dtype=torch.float32, device="cuda")
    d_X = torch.tensor(np.ascontiguousarray(features, dtype=np.float32), device="cuda")
    d_t = torch.tensor(np.ascontiguousarray(fracs, dtype=np.float32), device="cuda")
    d_o = torch.tensor(np.ascontiguousarray(order, dtype=np.int32), device="cuda")
    d_l = torch.zeros(len(order) // batch, dtype=torch.float32, device="cuda")
    fds.fds_mlp_train(d_p, d_X, d_t, d_o, batch, lr, d_l, stream)
    torch.cuda.synchronize()
    return d_p.cpu().numpy(), d_l.cpu().numpy()
