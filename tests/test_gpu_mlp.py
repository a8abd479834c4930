"""The MLP-seeded secular solve on the GPU.

* features, analytic estimates, inference, initialisation, gradient and
  Adam step of the library's kernels against the FP64 oracle
  (oracle/mlp.py, itself pinned by finite differences and closed forms):
  gradient relative error <= 1e-3 per parameter block in FP32;
* harvesting does not change the SVD;
* a network trained by the library's own kernels on harvests of n = 2048
  uniform (seed 4) and graded (seed 5) bidiagonals starts the roots of
  n = 4096 problems closer: fewer root-finder iterations, and the SVD still
  meets the FP64 tolerances against the oracle (the root finder finishes
  every root to the same stopping rule).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import check
from oracle import merge
from oracle import mlp as M
from paper_2508_11467_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bdc():
    from paper_2508_11467_gb300 import bdc as b
    from paper_2508_11467_gb300 import build
    build.build()
    b.lib()
    return b


def _secular_problem(N, seed, tiny=()):
    rng = np.random.default_rng(seed)
    d = np.concatenate([[0.0], np.sort(rng.uniform(0.05, 3.0, N - 1))])
    z = rng.normal(size=N)
    for k in tiny:
        z[k] = 1e-9 * np.sign(z[k])
    return d, z


def _rand_feats(rng, S):
    X = np.empty((S, M.N_IN))
    X[:, :3] = rng.normal(size=(S, 3)) * 4.0 - 3.0
    X[:, 3:5] = rng.normal(size=(S, 2))
    X[:, 5:7] = rng.normal(size=(S, 2)) * 4.0 - 6.0
    X[:, 7:9] = rng.normal(size=(S, 2))
    X[:, 9] = rng.normal(size=S) * 5.0
    X[:, 10] = rng.uniform(0.0, 1.0, S)
    return X


def test_counts(bdc):
    assert bdc.mlp_param_count() == M.N_PARAMS
    assert bdc.mlp_feature_count() == M.N_IN


@pytest.mark.parametrize("N", [2, 3, 12, 300])
def test_features_match_oracle(bdc, N):
    d, z = _secular_problem(N, 10 + N, tiny=(1,) if N > 2 else ())
    F, yq = bdc.mlp_features(torch.from_numpy(d).cuda(), torch.from_numpy(z).cuda())
    F, yq = F.cpu().numpy(), yq.cpu().numpy()
    R = M.all_features(d, z)
    assert F.shape == R.shape
    np.testing.assert_allclose(F, R, rtol=1e-5, atol=2e-4)
    yr = np.array([M.analytic(d, z, i) for i in range(N - 1)])
    np.testing.assert_allclose(yq, yr, rtol=1e-9, atol=1e-9)


def test_init_statistics(bdc):
    rng = np.random.default_rng(0)
    X = _rand_feats(rng, 5000)
    y = rng.normal(size=5000) * 2 + 0.5
    Xt = torch.from_numpy(X.astype(np.float32)).cuda()
    yt = torch.from_numpy(y.astype(np.float32)).cuda()
    P = bdc.mlp_init(Xt, yt, seed=7).cpu().numpy().astype(np.float64)
    X32 = X.astype(np.float32).astype(np.float64)
    k = M.N_IN
    np.testing.assert_allclose(P[0:k], X32.mean(axis=0), rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(P[k:2 * k], 1.0 / X32.std(axis=0), rtol=1e-4)
    p = M.unpack(P)
    assert np.all(p["b1"] == 0) and np.all(p["b2"] == 0)
    assert np.all(p["W3"] == 0) and p["b3"] == 0      # untrained: g = 0
    assert np.abs(p["W1"]).max() <= np.sqrt(6 / (M.N_IN + 64)) and np.abs(p["W2"]).max() <= np.sqrt(6 / 128)
    assert np.std(p["W1"]) > 0.1   # U(-a, a), a = 0.29: std a/sqrt(3)
    P2 = bdc.mlp_init(Xt, yt, seed=7).cpu().numpy()
    P3 = bdc.mlp_init(Xt, yt, seed=8).cpu().numpy()
    assert np.array_equal(P2, P.astype(np.float32)) and not np.array_equal(P3[M.OFF_W1:], P2[M.OFF_W1:])


def _trained_like_params(bdc, rng, S=3000):
    X = _rand_feats(rng, S)
    y = np.tanh(X[:, 0] - X[:, 1]) * 3 + 0.2 * X[:, 2]
    Xt = torch.from_numpy(X.astype(np.float32)).cuda()
    yt = torch.from_numpy(y.astype(np.float32)).cuda()
    P = bdc.mlp_init(Xt, yt, seed=1)
    # move away from the symmetric start so every block has signal
    k = M.OFF_W1
    P[k:] += torch.from_numpy(rng.normal(size=M.N_PARAMS - k).astype(np.float32) * 0.05).cuda()
    return P, X, y


def test_predict_matches_oracle(bdc):
    rng = np.random.default_rng(1)
    P, X, _ = _trained_like_params(bdc, rng)
    yh = bdc.mlp_predict(P, torch.from_numpy(X.astype(np.float32)).cuda()).cpu().numpy()
    ref, _ = M.forward(P.cpu().numpy().astype(np.float64), X.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(yh, ref, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("S,huber", [(50, 0.0), (1000, 0.25), (20000, 0.25), (3000, 0.0)])
def test_grad_matches_oracle(bdc, S, huber):
    """GPU backward vs the FP64 chain rule: one partial block (S = 50), a
    ragged multi-block case, and more 64-sample blocks than CTAs; squared
    and Huber loss."""
    rng = np.random.default_rng(S)
    P, X, y = _trained_like_params(bdc, rng, S)
    g, loss = bdc.mlp_grad(P, torch.from_numpy(X.astype(np.float32)).cuda(),
                           torch.from_numpy(y.astype(np.float32)).cuda(), huber=huber)
    g = g.cpu().numpy().astype(np.float64)
    L, G = M.loss_and_grad(P.cpu().numpy().astype(np.float64), X.astype(np.float32).astype(np.float64),
                           y.astype(np.float32).astype(np.float64), huber)
    assert float(loss.item()) == pytest.approx(L, rel=1e-4)
    assert np.all(g[:M.OFF_W1] == 0.0)
    for a, b in [(M.OFF_W1, M.OFF_B1), (M.OFF_B1, M.OFF_W2), (M.OFF_W2, M.OFF_B2), (M.OFF_B2, M.OFF_W3),
                 (M.OFF_W3, M.OFF_B3), (M.OFF_B3, M.N_PARAMS)]:
        rel = np.linalg.norm(g[a:b] - G[a:b]) / max(np.linalg.norm(G[a:b]), 1e-30)
        assert rel <= 1e-3, (a, b, rel)


def test_grad_deterministic(bdc):
    rng = np.random.default_rng(5)
    P, X, y = _trained_like_params(bdc, rng, 7000)
    Xt = torch.from_numpy(X.astype(np.float32)).cuda()
    yt = torch.from_numpy(y.astype(np.float32)).cuda()
    g1, l1 = bdc.mlp_grad(P, Xt, yt)
    g2, l2 = bdc.mlp_grad(P, Xt, yt)
    assert torch.equal(g1, g2) and torch.equal(l1, l2)


def test_adam_matches_oracle(bdc):
    rng = np.random.default_rng(2)
    P = rng.normal(size=M.N_PARAMS).astype(np.float32)
    G = rng.normal(size=M.N_PARAMS).astype(np.float32)
    G[:M.OFF_W1] = 0
    m = (rng.normal(size=M.N_PARAMS) * 0.1).astype(np.float32)
    v = (rng.uniform(0, 0.1, M.N_PARAMS)).astype(np.float32)
    Pt, Gt, mt, vt = (torch.from_numpy(a.copy()).cuda() for a in (P, G, m, v))
    bdc.mlp_adam(Pt, Gt, mt, vt, 3, 2e-3)
    # the kernel takes its hyper-parameters as FP32 values
    f32 = lambda v: float(np.float32(v))
    P1, m1, v1 = M.adam_step(P.astype(np.float64), G.astype(np.float64), m.astype(np.float64),
                             v.astype(np.float64), 3, f32(2e-3), f32(0.9), f32(0.999), f32(1e-8))
    np.testing.assert_allclose(mt.cpu().numpy(), m1, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(vt.cpu().numpy(), v1, rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(Pt.cpu().numpy(), P1, rtol=1e-5, atol=1e-6)
    assert np.array_equal(Pt.cpu().numpy()[:M.OFF_W1], P[:M.OFF_W1])


def test_harvest_does_not_change_the_svd(bdc):
    d, e = inputs.uniform(1500, 3)
    dt, et = torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda()
    H = bdc.Harvest(1 << 16)
    S1, U1, VT1, _ = bdc.svd(dt, et)
    S2, U2, VT2, _ = bdc.svd_harvest(dt, et, H)
    assert torch.equal(S1, S2) and torch.equal(U1, U2) and torch.equal(VT1, VT2)
    F, y = H.data()
    assert 0 < F.shape[0] <= H.cap
    F, y = F.cpu().numpy(), y.cpu().numpy()
    assert np.all(np.isfinite(F)) and np.all(np.abs(F) <= 40) and np.all(np.isfinite(y))
    assert np.all((F[:, 10] >= 0) & (F[:, 10] < 1))
    # a second call appends; a small capacity counts past the end without writing
    bdc.svd_harvest(dt, et, H)
    assert int(H.count.item()) == 2 * F.shape[0]
    Hs = bdc.Harvest(10)
    bdc.svd_harvest(dt, et, Hs)
    assert int(Hs.count.item()) == F.shape[0] and Hs.size() == 10


@pytest.fixture(scope="module")
def trained(bdc):
    """Harvest n = 2048 uniform (seed 4) and graded (seed 5), train with the
    library's kernels."""
    H = bdc.Harvest(1 << 20)
    for kind, seed in [("uniform", 4), ("graded", 5)]:
        d, e = inputs.make(kind, 2048, seed)
        bdc.svd_harvest(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda(), H)
    F, r = H.data()
    P, losses = bdc.mlp_train(F, r, steps=1500, lr=3e-3, seed=0)
    torch.cuda.synchronize()
    return P, losses.cpu().numpy(), F, r


def test_training_lowers_the_loss(bdc, trained):
    P, losses, F, r = trained
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.8 * losses[0], (losses[0], losses[-1])
    # the trained correction shrinks the median error of the analytic start
    g = bdc.mlp_predict(P, F)
    e0 = float(r.abs().median())
    e1 = float((g - r).abs().median())
    print(f"median |y - y_q| {e0:.3f}  median |y - y_q - g| {e1:.3f}")
    assert e1 < e0


@pytest.mark.parametrize("seed_mode", ["analytic", "mlp"])
def test_seeded_roots_equal_plain_roots(bdc, trained, seed_mode):
    P = trained[0]
    d, z = _secular_problem(1500, 3)
    dt, zt = torch.from_numpy(d).cuda(), torch.from_numpy(z).cuda()
    o0, t0, w0, it0, i0 = bdc.secular_solve_ex(dt, zt)
    o1, t1, w1, it1, i1 = bdc.secular_solve_ex(dt, zt, seed=seed_mode, mlp=P)
    assert int(i0.item()) == 0 and int(i1.item()) == 0
    w0, w1 = w0.cpu().numpy(), w1.cpu().numpy()
    # the same bar as the plain solve: a few ulps against the bisection
    # oracle, and the returned (org, tau) satisfy the secular equation
    _, _, wr = merge.secular_roots(d, z)
    eps = np.finfo(float).eps
    assert np.max(np.abs(w1 - wr) / wr) <= 64 * eps
    assert np.max(np.abs(w1 - w0) / w0) <= 64 * eps
    f, scale = merge.secular_f(d, z, o1.cpu().numpy(), t1.cpu().numpy())
    assert np.all(np.abs(f) <= 64 * eps * scale)
    # the origin is the nearer pole (away from the interval midpoints)
    o1n = o1.cpu().numpy()
    pos = (w1[:-1] ** 2 - d[:-1] ** 2) / (d[1:] ** 2 - d[:-1] ** 2)
    far = np.abs(pos - 0.5) > 1e-6
    assert np.all(o1n[:-1][far] == np.where(pos[far] < 0.5, np.arange(len(d) - 1)[far], np.arange(1, len(d))[far]))
    it0, it1 = it0.cpu().numpy(), it1.cpu().numpy()
    assert np.all(it1 >= 0)
    print(f"{seed_mode}: iterations per root plain {it0.mean():.3f}  seeded {it1.mean():.3f}")


@pytest.mark.parametrize("kind,seed", [("uniform", 0), ("graded", 1)])
def test_mlp_svd_parity_and_fewer_iterations(bdc, trained, kind, seed):
    """The gain: iterations per root of the plain start, the analytic start
    alone and the trained network, on n = 4096 problems the network was not
    trained on; and the seeded SVD meets the FP64 bar against the oracle."""
    P = trained[0]
    n = 4096
    d, e = inputs.make(kind, n, seed)
    dt, et = torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda()
    stats = {}
    for mode in ("plain", "analytic", "mlp"):
        bdc.profile_begin()
        # FP64 starts only: the FP32 pre-iterations would hide the start's effect
        S, U, VT, info = bdc.svd(dt, et, seed=mode, mlp=P if mode == "mlp" else None, fp32_start=False)
        prof = bdc.profile_end()
        assert info == 0
        stats[mode] = (prof["secular"]["iters"], prof["secular"]["roots"], S, U, VT)
    r0 = stats["plain"][1]
    assert all(stats[m][1] == r0 > 0 for m in stats)
    ipr = {m: stats[m][0] / r0 for m in stats}
    print(f"{kind}: iterations per root " + "  ".join(f"{m} {v:.3f}" for m, v in ipr.items()))
    # with the FP64 root finder alone the learned start saves >= 15% of the
    # iterations against the midpoint start; against its own analytic prior
    # it is reported, not claimed (the network corrects y_q by ~0.04 in logit,
    # too little to remove a step of the rational iteration)
    assert ipr["mlp"] <= 0.85 * ipr["plain"], ipr
    assert ipr["mlp"] <= 1.02 * ipr["analytic"], ipr
    # parity of the seeded run with the FP64 oracle (same bar as the plain path)
    _, _, S, U, VT = stats["mlp"]
    s = S.cpu().numpy()
    tol = 1e-13 * n
    assert check.sigma_rel_err(s, oracle.sigma_only(d, e)) <= tol
    assert oracle.residual(d, e, s, U.cpu().numpy(), VT.cpu().numpy()) <= tol
    for X in (U, VT.t()):
        G = X.t() @ X
        G.diagonal().sub_(1.0)
        assert float(torch.linalg.norm(G)) <= tol
    # singular values agree with the plain solve to rounding
    s0 = stats["plain"][2].cpu().numpy()
    assert np.max(np.abs(s - s0)) <= 64 * np.finfo(float).eps * s0[0]


@pytest.mark.parametrize("kind,seed", [("uniform", 0), ("graded", 1)])
def test_shipped_configuration_has_no_start_to_gain(bdc, trained, kind, seed):
    """With the FP32 pre-iterations (the default) every start rule needs
    the same FP64 work: each root takes one pole-sum evaluation at its start
    and at least one more that confirms the step, and the FP32 phase already
    brings every start to ~2^-17, so plain, analytic and learned starts all
    land at ~1.1 FP64 iterations per root (2.1 evaluations).  The learned
    start does not pay in this configuration; this test records that."""
    P = trained[0]
    d, e = inputs.make(kind, 4096, seed)
    dt, et = torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda()
    ipr = {}
    for mode in ("plain", "analytic", "mlp"):
        bdc.profile_begin()
        _, _, _, info = bdc.svd(dt, et, seed=mode, mlp=P if mode == "mlp" else None)
        prof = bdc.profile_end()
        assert info == 0
        ipr[mode] = prof["secular"]["iters"] / prof["secular"]["roots"]
    print(f"{kind} (FP32 pre-iterations): FP64 iterations per root " +
          "  ".join(f"{m} {v:.3f}" for m, v in ipr.items()))
    assert all(1.0 <= v <= 1.35 for v in ipr.values()), ipr
    assert max(ipr.values()) <= 1.06 * min(ipr.values()), ipr


def test_mlp_with_mixed_products(bdc, trained):
    P = trained[0]
    d, e = inputs.uniform(4096, 0)
    S, U, VT, info = bdc.svd(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda(), prec="exact",
                             seed="mlp", mlp=P)
    assert info == 0
    s = S.cpu().numpy()
    assert oracle.residual(d, e, s, U.cpu().numpy(), VT.cpu().numpy()) <= 1e-12
    assert check.sigma_rel_err(s, oracle.sigma_only(d, e)) <= 1e-13 * 4096


def test_mlp_save_load_roundtrip(bdc, trained, tmp_path):
    P = trained[0]
    path = tmp_path / "mlp.bin"
    bdc.mlp_save(P, str(path))
    Q = bdc.mlp_load(str(path))
    assert torch.equal(P, Q)
