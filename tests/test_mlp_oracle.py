"""Pins of the root-start oracle (oracle/mlp.py) against things other than
itself: central finite differences for the backward pass, hand-derived
feature values, scale invariance, the closed-form root of a two-pole
secular equation (where the analytic estimate is exact), the exactness of
the far-pole moment estimate for a single far pole, and the sign rule of
Adam's first step."""
import numpy as np
import pytest

from oracle import merge
from oracle import mlp as M


def _rand_params(rng, scale=0.5):
    P = rng.uniform(-scale, scale, M.N_PARAMS)
    P[M.OFF_MEAN:M.OFF_MEAN + M.N_IN] = rng.normal(size=M.N_IN)
    P[M.OFF_ISTD:M.OFF_ISTD + M.N_IN] = rng.uniform(0.5, 2.0, M.N_IN)
    return P


def test_layout():
    assert M.N_PARAMS == 22 + 64 * 11 + 64 + 64 * 64 + 64 + 64 + 1 == 5015


@pytest.mark.parametrize("huber", [0.0, 0.3])
def test_backward_matches_central_differences(huber):
    rng = np.random.default_rng(0)
    P = _rand_params(rng)
    X = rng.normal(size=(7, M.N_IN))
    y = rng.normal(size=7)
    L, G = M.loss_and_grad(P, X, y, huber)
    assert L == pytest.approx(M.loss(P, X, y, huber), rel=1e-15)
    # every block: a few indices of W1, b1, W2, b2, W3 and b3
    idx = list(rng.choice(np.arange(M.OFF_W1, M.OFF_B1), 6, replace=False))
    idx += list(rng.choice(np.arange(M.OFF_B1, M.OFF_W2), 4, replace=False))
    idx += list(rng.choice(np.arange(M.OFF_W2, M.OFF_B2), 8, replace=False))
    idx += list(rng.choice(np.arange(M.OFF_B2, M.OFF_W3), 4, replace=False))
    idx += list(rng.choice(np.arange(M.OFF_W3, M.OFF_B3), 4, replace=False))
    idx += [M.OFF_B3]
    h = 1e-6
    for k in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[k] += h
        Pm[k] -= h
        fd = (M.loss(Pp, X, y, huber) - M.loss(Pm, X, y, huber)) / (2 * h)
        assert abs(fd - G[k]) <= 1e-7 * max(1.0, abs(fd)), (k, fd, G[k])
    # the normalisation is not trained
    assert np.all(G[:M.OFF_W1] == 0.0)


def test_features_hand_example():
    # d = [0, 1, 3, 4], z = [1, 2, 1, 0.5], root 1 in (1, 3):
    # D2 = 9 - 1 = 8, gaps (1, 2, 1), rho = 1 + 4 + 1 + 0.25 = 6.25,
    # midpoint m = 2: near = 1/(0 - 4) + 0.25/(16 - 4) = -11/48, no far poles
    d = np.array([0.0, 1.0, 3.0, 4.0])
    z = np.array([1.0, 2.0, 1.0, 0.5])
    assert M.background(d, z, 1) == pytest.approx((-11 / 48, 0.0), rel=1e-15, abs=0)
    f = M.features(d, z, 1)
    want = [np.log(4 / 8), np.log(1 / 8), np.log(6.25 / 8), np.log(1 / 2), np.log(1 / 2),
            np.log(1 / 8), np.log(0.25 / 8), np.arcsinh(-11 / 48), 0.0, M.analytic(d, z, 1), 1 / 3]
    np.testing.assert_allclose(f, want, rtol=1e-15, atol=1e-15)
    # ends: root 0 has no left neighbour, root 2 no right one
    f0 = M.features(d, z, 0)
    assert f0[3] == 0.0 and f0[5] == -40.0 and f0[10] == 0.0
    f2 = M.features(d, z, 2)
    assert f2[4] == 0.0 and f2[6] == -40.0


def test_analytic_solves_the_frozen_quadratic():
    # y_q's t satisfies c - a/t + b/(1-t) = 0 with c = 1 + near + far
    rng = np.random.default_rng(4)
    N = 60
    d = np.concatenate([[0.0], np.sort(rng.uniform(0.1, 2.0, N - 1))])
    z = rng.normal(size=N)
    for i in (0, 5, 30, N - 2):
        D2 = (d[i + 1] - d[i]) * (d[i + 1] + d[i])
        a, b = z[i] ** 2 / D2, z[i + 1] ** 2 / D2
        c = 1.0 + sum(M.background(d, z, i))
        y = M.analytic(d, z, i)
        t = 1.0 / (1.0 + np.exp(-y))
        s = 1.0 / (1.0 + np.exp(y))
        scale = abs(c) + a / t + b / s
        assert abs(c - a / t + b / s) <= 1e-12 * scale


def test_far_estimate_exact_for_one_far_pole():
    # root 0 of an 11-pole problem: poles 2..9 are near, pole 10 is the only
    # far one, so the moment estimate is its exact term
    rng = np.random.default_rng(5)
    d = np.concatenate([[0.0], np.sort(rng.uniform(0.1, 2.0, 10))])
    z = rng.normal(size=11)
    m = 0.5 * (d[0] + d[1])
    near, far = M.background(d, z, 0)
    assert far == pytest.approx(z[10] ** 2 / (d[10] ** 2 - m * m), rel=1e-14)
    assert near == pytest.approx(sum(z[j] ** 2 / (d[j] ** 2 - m * m) for j in range(2, 10)), rel=1e-13)


def test_features_scale_invariant_and_clamped():
    rng = np.random.default_rng(1)
    N = 40
    d = np.concatenate([[0.0], np.sort(rng.uniform(0.1, 2.0, N - 1))])
    z = rng.normal(size=N)
    F = M.all_features(d, z)
    for c in (1e-5, 3.0, 1e7):
        np.testing.assert_allclose(M.all_features(c * d, c * z), F, rtol=1e-12, atol=1e-12)
    z2 = z.copy()
    z2[5] = 1e-30
    F2 = M.all_features(d, z2)
    assert F2[5, 0] == -40.0 and F2[4, 1] == -40.0
    assert np.all(np.abs(F2) <= 40.0)


def test_two_pole_closed_form():
    # N = 2, d = (0, d1): w^2 solves u^2 - (d1^2 + rho) u + z0^2 d1^2 = 0;
    # root 0 is the smaller solution, in (0, d1^2).  With no other pole the
    # analytic estimate is exact and the training target is 0.
    for d1, z0, z1 in [(1.0, 0.3, 0.4), (2.5, 1.0, 1e-3), (0.7, 1e-4, 2.0)]:
        rho = z0 * z0 + z1 * z1
        b = d1 * d1 + rho
        u = 2 * z0 * z0 * d1 * d1 / (b + np.sqrt(b * b - 4 * z0 * z0 * d1 * d1))
        t = u / (d1 * d1)
        y = np.log(t / (1 - t))
        d = np.array([0.0, d1])
        z = np.array([z0, z1])
        om = np.array([np.sqrt(u), 0.0])
        assert M.logit(d, om, 0) == pytest.approx(y, rel=1e-10, abs=1e-12)
        assert M.analytic(d, z, 0) == pytest.approx(y, rel=1e-10, abs=1e-10)
        # and the oracle's own secular roots land on the same position
        org, tau, om2 = merge.secular_roots(d, z)
        assert M.logit(d, om2, 0) == pytest.approx(y, rel=1e-9, abs=1e-9)
        assert abs(M.target(d, z, om2, 0)) <= 1e-8


def test_adam_first_step_is_lr_times_sign():
    rng = np.random.default_rng(2)
    P = _rand_params(rng)
    G = rng.normal(size=M.N_PARAMS)
    k = M.OFF_W1
    G[:k] = 0.0
    P1, m, v = M.adam_step(P, G, np.zeros_like(P), np.zeros_like(P), 1, 1e-3, eps=1e-30)
    np.testing.assert_allclose(P1[k:], P[k:] - 1e-3 * np.sign(G[k:]), rtol=0, atol=1e-15)
    assert np.all(P1[:k] == P[:k])
    np.testing.assert_allclose(m[k:], 0.1 * G[k:])
    np.testing.assert_allclose(v[k:], 0.001 * G[k:] ** 2)


def test_forward_linear_limit():
    # with tiny weights tanh is linear: yhat ~ b3 + W3 (W2 (W1 xn + b1) + b2)
    rng = np.random.default_rng(3)
    P = _rand_params(rng, scale=1e-4)
    X = rng.normal(size=(5, M.N_IN))
    p = M.unpack(P)
    Xn = (X - p["mean"]) * p["istd"]
    lin = ((Xn @ p["W1"].T + p["b1"]) @ p["W2"].T + p["b2"]) @ p["W3"] + p["b3"]
    y, _ = M.forward(P, X)
    np.testing.assert_allclose(y, lin, rtol=0, atol=1e-14)
