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


PARAMS_FILE = __import__("os").path.join(__import__("os").path.dirname(__file__), "rank_mlp_params.npy")


def load_params(path=PARAMS_FILE):
    """The parameter vector trained by `python -m paper_2411_18026_gb300.learned`
    (float32, FDS_MLP_NPARAM), or None if it has not been trained."""
    import os
    if not os.path.exists(path):
        return None
    p = np.load(path)
    return p if p.size == fds.FDS_MLP_NPARAM else None


def main(argv=None):
    """Train the rank network on seeded random cavities (ellipses and stars,
    2^12..2^16 nodes, k_T a in [1, 20], leaf tolerance 1e-9 and 1e-8 with the
    default per-level tolerance, leaf 64) and save the parameters next to this
    module."""
    import argparse
    import sys
    import time
    ap = argparse.ArgumentParser(prog="python -m paper_2411_18026_gb300.learned")
    ap.add_argument("--count", type=int, default=2000, help="training cavities")
    ap.add_argument("--nmax-log2", type=int, default=16, help="largest training cavity: 2^n nodes")
    ap.add_argument("--epochs", type=int, default=0, help="passes over the samples (0: enough for --steps)")
    ap.add_argument("--steps", type=int, default=30000, help="Adam steps when --epochs is 0")
    ap.add_argument("--out", default=PARAMS_FILE)
    a = ap.parse_args(argv)
    sys.path.insert(0, __import__("os").path.dirname(__import__("os").path.dirname(__file__)))
    import workloads
    from . import build
    build.build()
    t0 = time.time()
    cav = workloads.random_cavities(a.count, seed=workloads.SEED + 4, nmin_log2=12, nmax_log2=a.nmax_log2)
    half = len(cav) // 2
    F1, r1 = collect(cav[:half], 1e-9)
    F2, r2 = collect(cav[half:], 1e-8)
    F, r = np.concatenate([F1, F2]), np.concatenate([r1, r2])
    t1 = time.time()
    epochs = a.epochs or max(1, -(-a.steps * 256 // len(F)))
    order = workloads.minibatch_order(len(F), 256, epochs)
    p, losses = train(F, r, workloads.mlp_init(), order, batch=256, lr=2e-3)
    np.save(a.out, p.astype(np.float32))
    print("samples %d, collect %.1fs, train %.1fs, loss %.3e -> %.3e, saved %s" %
          (len(F), t1 - t0, time.time() - t1, losses[:10].mean(), losses[-50:].mean(), a.out))


if __name__ == "__main__":
    main()
