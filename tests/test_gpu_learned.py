"""Learned skeleton-rank network: CUDA inference / gradient / Adam kernels
against the oracle restatement (oracle/mlp.py), training determinism, the
recorded training data, and the learned-rank build (sketched ID with adaptive
fallback) against the adaptive build and the dense oracle solve."""
import numpy as np
import pytest

import workloads
from gpu_util import fdslib, torch_cuda
from oracle import bem, mlp

pytestmark = pytest.mark.gpu


def _params(seed):
    p = workloads.mlp_init(seed)
    rng = np.random.default_rng(seed + 1)
    q = mlp.unpack(p)
    q["mu"][:] = rng.normal(0.0, 1.0, 16)
    q["sd"][:] = rng.uniform(0.5, 2.0, 16)
    q["b1"][:] = rng.normal(0.0, 0.1, 64)
    q["b2"][:] = rng.normal(0.0, 0.1, 64)
    q["b3"][:] = 0.3
    return p


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(0.0, 1.5, (n, 16))
    t = 0.4 + 0.2 * np.tanh(X[:, 1] - 0.3 * X[:, 5])
    return X, t


def test_forward_matches_oracle():
    torch = torch_cuda()
    fds = fdslib()
    p = _params(1)
    X, _ = _data(1000, 2)           # ragged last CTA
    d_p = torch.tensor(p, dtype=torch.float32, device="cuda")
    d_X = torch.tensor(X, dtype=torch.float32, device="cuda")
    d_y = torch.empty(1000, dtype=torch.float32, device="cuda")
    fds.fds_mlp_forward(d_p, d_X, d_y)
    y_ref, _ = mlp.forward(p.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64))
    assert np.abs(d_y.cpu().numpy() - y_ref).max() <= 2e-5 * max(1.0, np.abs(y_ref).max())


@pytest.mark.parametrize("n", [1, 37, 256, 777])
def test_loss_gradient_matches_oracle(n):
    torch = torch_cuda()
    fds = fdslib()
    p = _params(3)
    X, t = _data(n, 4)
    p32 = p.astype(np.float32).astype(np.float64)
    L_ref, g_ref = mlp.loss_grad(p32, X.astype(np.float32).astype(np.float64), t.astype(np.float32))
    d_p = torch.tensor(p, dtype=torch.float32, device="cuda")
    d_X = torch.tensor(X, dtype=torch.float32, device="cuda")
    d_t = torch.tensor(t, dtype=torch.float32, device="cuda")
    d_g = torch.empty(fds.FDS_MLP_NTRAIN, dtype=torch.float32, device="cuda")
    d_L = torch.empty(1, dtype=torch.float32, device="cuda")
    fds.fds_mlp_loss_grad(d_p, d_X, d_t, d_g, d_L)
    g = d_g.cpu().numpy()
    assert abs(d_L.item() - L_ref) <= 1e-5 * max(1.0, L_ref)
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
    # repeated call: bit-identical (deterministic reduction)
    d_g2 = torch.empty_like(d_g)
    fds.fds_mlp_loss_grad(d_p, d_X, d_t, d_g2, d_L)
    assert torch.equal(d_g, d_g2)


def test_adam_step_matches_oracle():
    torch = torch_cuda()
    fds = fdslib()
    rng = np.random.default_rng(9)
    p = _params(5)
    g = rng.normal(0, 1, fds.FDS_MLP_NTRAIN)
    m = rng.normal(0, 0.1, fds.FDS_MLP_NTRAIN)
    v = rng.uniform(0, 0.1, fds.FDS_MLP_NTRAIN)
    d_p = torch.tensor(p, dtype=torch.float32, device="cuda")
    d_g = torch.tensor(g, dtype=torch.float32, device="cuda")
    d_m = torch.tensor(m, dtype=torch.float32, device="cuda")
    d_v = torch.tensor(v, dtype=torch.float32, device="cuda")
    fds.fds_mlp_adam(d_p, d_g, d_m, d_v, 7, 1e-3)
    p_ref, m_ref, v_ref = mlp.adam(p.astype(np.float32).astype(np.float64), g.astype(np.float32), m.astype(np.float32),
                                   v.astype(np.float32), 7, 1e-3)
    assert np.abs(d_p.cpu().numpy() - p_ref).max() <= 1e-6
    assert np.abs(d_m.cpu().numpy() - m_ref).max() <= 1e-6
    assert np.abs(d_v.cpu().numpy() - v_ref).max() <= 1e-6


def test_training_is_deterministic_and_follows_oracle():
    torch = torch_cuda()
    fds = fdslib()
    X, t = _data(512, 6)
    p0 = workloads.mlp_init(7)
    order = workloads.minibatch_order(512, 64, 3)
    res = []
    for _ in range(2):
        d_p = torch.tensor(p0, dtype=torch.float32, device="cuda")
        d_X = torch.tensor(X, dtype=torch.float32, device="cuda")
        d_t = torch.tensor(t, dtype=torch.float32, device="cuda")
        d_o = torch.tensor(order, dtype=torch.int32, device="cuda")
        d_l = torch.zeros(len(order) // 64, dtype=torch.float32, device="cuda")
        fds.fds_mlp_train(d_p, d_X, d_t, d_o, 64, 3e-3, d_l)
        res.append((d_p.cpu().numpy(), d_l.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    p_ref, l_ref = mlp.train(p0.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64),
                             t.astype(np.float32).astype(np.float64), order, 64, 3e-3)
    # same loss curve (float32 vs float64 arithmetic)
    assert np.abs(res[0][1] - l_ref).max() <= 1e-3 * l_ref.max()
    assert res[0][1][-5:].mean() < 0.5 * res[0][1][:3].mean()


def test_recorded_features():
    torch_cuda()
    fds = fdslib()
    xy = workloads.star(2048)
    tol = 1e-8
    h = fds.fds_build(xy, workloads.omega_for_kTa(10.0), 2.0, 1.0, tol, leaf_size=64, record_features=True)
    F, r = fds.fds_features_get(h)
    st = fds.fds_stats_get(h)
    # every (cell, component) of levels L..l0+1 with DOFs
    assert len(F) == st.features_recorded > 2 * (2048 // 64)
    assert np.all((r > 0) & (r <= 1))
    assert set(np.unique(F[:, 2])) == {0.0, 1.0}
    # log10 of the level's ID tolerance: tol at the leaves, halved per level up
    assert np.allclose(F[:, 13], np.log10(tol) + F[:, 0] * np.log10(0.5), atol=1e-5)
    leaf = F[:, 0] == 0
    assert np.all(F[leaf, 14] == 1.0) and np.allclose(F[leaf, 1], np.log2(64))
    # ranks recorded equal the level ranks the build reports
    L = st.levels
    k = fds.fds_level_ranks(h, L, 2048 // 64)
    assert np.allclose(r[:2 * (2048 // 64)].reshape(-1, 2) * 64, k)
    h.close()


def _trained(fds):
    from paper_2411_18026_gb300 import learned
    cav = workloads.random_cavities(10, seed=workloads.SEED + 11, nmin_log2=10, nmax_log2=12, kta=(2.0, 12.0))
    F, r = learned.collect(cav, 1e-8, leaf_size=32)
    order = workloads.minibatch_order(len(F), 128, 60)
    p, losses = learned.train(F, r, workloads.mlp_init(), order, batch=128, lr=3e-3)
    return p, losses, F, r


def test_learned_build_matches_adaptive_and_dense():
    torch_cuda()
    fds = fdslib()
    p, losses, F, r = _trained(fds)
    assert losses[-20:].mean() < 0.2 * losses[:5].mean()
    # unseen cavity
    xy = workloads.star(1024, 0.15, 4, rot=0.3)
    omega = workloads.omega_for_kTa(7.0)
    tol = 1e-8
    ha = fds.fds_build(xy, omega, 2.0, 1.0, tol, leaf_size=32)
    hl = fds.fds_build(xy, omega, 2.0, 1.0, tol, leaf_size=32, mlp_params=p)
    st = fds.fds_stats_get(hl)
    assert st.id_sketched + st.id_fallback > 0
    assert st.id_sketched >= 0.5 * (st.id_sketched + st.id_fallback)
    P = bem.phys(2.0, 1.0, 1.0, omega)
    Fr = np.stack([bem.rhs(P, xy, 0, 0.2), bem.rhs(P, xy, 1, 2.5)], 1)
    xa = fds.fds_solve(ha, Fr)
    xl = fds.fds_solve(hl, Fr)
    xd = np.linalg.solve(bem.dense_matrix(P, xy), Fr)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(xa, xd) <= 10 * tol
    assert rel(xl, xd) <= 10 * tol
    ha.close()
    hl.close()


def test_untrained_prediction_falls_back():
    # a network predicting rank 0 everywhere: every sketch is too small to
    # reveal the rank, so every ID falls back and the result is the adaptive one
    torch_cuda()
    fds = fdslib()
    p = np.zeros(fds.FDS_MLP_NPARAM)
    p[fds.FDS_MLP_NTRAIN + 16:] = 1.0     # sd = 1
    xy = workloads.star(512)
    omega = workloads.omega_for_kTa(5.0)
    ha = fds.fds_build(xy, omega, 2.0, 1.0, 1e-8, leaf_size=32)
    hl = fds.fds_build(xy, omega, 2.0, 1.0, 1e-8, leaf_size=32, mlp_params=p, sketch_extra=1)
    st = fds.fds_stats_get(hl)
    assert st.id_sketched == 0 and st.id_fallback > 0
    for l in range(st.top_level + 1, st.levels + 1):
        nb = 1 << l
        assert np.array_equal(fds.fds_level_ranks(ha, l, nb), fds.fds_level_ranks(hl, l, nb))
    ha.close()
    hl.close()


def _id_ms(fds, xy, omega, tol, params):
    fds.fds_timing_reset()
    fds.fds_timing_enable(True)
    h = fds.fds_build(xy, omega, 2.0, 1.0, tol, leaf_size=64, mlp_params=params)
    fds.fds_timing_enable(False)
    rep = fds.fds_timing_report()
    st = fds.fds_stats_get(h)
    ms = sum(v["ms"] for k, v in rep.items() if k.startswith("a2."))
    return h, ms, st


def test_trained_network_gains_over_adaptive_id():
    # The trained network sizes the sketch; the gain is the ID time against the
    # adaptive CPQR (same tolerance), at an accuracy that stays within 10 eps
    # of the adaptive build's solution.  A network predicting k = n (sketch of
    # n + extra rows) isolates what the prediction adds to the sketch.
    torch_cuda()
    fds = fdslib()
    from paper_2411_18026_gb300 import learned
    p = learned.load_params()
    if p is None:
        p, _, _, _ = _trained(fds)
    full = np.zeros(fds.FDS_MLP_NPARAM)
    full[fds.FDS_MLP_NTRAIN - 1] = 1.0            # b3 = 1: predicts k / n = 1
    full[fds.FDS_MLP_NTRAIN + 16:] = 1.0
    xy = workloads.star(1 << 16, 0.25, 6, rot=0.7)
    omega = workloads.omega_for_kTa(12.0)
    tol = 1e-8
    for _ in range(2):      # warm-up (first launches load the kernels)
        ha, ms_a, _ = _id_ms(fds, xy, omega, tol, None)
        ha.close()
    ha, ms_a, st_a = _id_ms(fds, xy, omega, tol, None)
    hl, ms_l, st_l = _id_ms(fds, xy, omega, tol, p)
    hf, ms_f, st_f = _id_ms(fds, xy, omega, tol, full)
    print("ID ms: adaptive %.2f, sketch k=n %.2f (fallback %d), learned %.2f (sketched %d, fallback %d)"
          % (ms_a, ms_f, st_f.id_fallback, ms_l, st_l.id_sketched, st_l.id_fallback))
    assert st_l.id_fallback <= 0.2 * (st_l.id_sketched + st_l.id_fallback)
    assert ms_l < ms_a
    # the sketch keeps a few more skeleton columns than the adaptive ID
    ka = sum(st_a.skeleton_dofs[l] for l in range(st_a.top_level + 1, st_a.levels + 1))
    kl = sum(st_l.skeleton_dofs[l] for l in range(st_l.top_level + 1, st_l.levels + 1))
    print("skeleton DOFs: adaptive %d, learned %d (+%.1f%%)" % (ka, kl, 100.0 * (kl - ka) / ka))
    assert 0.95 * ka <= kl <= 1.25 * ka
    kinds, ang = workloads.plane_wave_set(2)
    F = fds.fds_rhs_plane_wave(ha, kinds, ang)
    xa = fds.fds_solve(ha, F)
    xl = fds.fds_solve(hl, F)
    # two compressions at the same tolerances: with the per-level graded
    # tolerance both stay within a few tol of the Galerkin solution
    err = np.linalg.norm(xl - xa) / np.linalg.norm(xa)
    print("learned vs adaptive solution: %.2e" % err)
    assert err <= 100 * tol
    for h in (ha, hl, hf):
        h.close()
