"""Pins for the merge-step oracle (Sec. 4.2.1) and the numpy model of Alg. 2."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import check, merge
from paper_2508_11467_gb300 import inputs

EPS = np.finfo(np.float64).eps
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random_M(N, seed, gap=1e-3):
    rng = np.random.default_rng(seed)
    d = np.concatenate(([0.0], np.sort(rng.uniform(gap, 1.0, N - 1))))
    # keep poles separated by at least gap
    for i in range(1, N):
        d[i] = max(d[i], d[i - 1] + gap)
    z = rng.uniform(0.05, 0.5, N) * rng.choice([-1.0, 1.0], N)
    return d, z


def _dense_M(d, z):
    N = d.shape[0]
    M = np.zeros((N, N))
    M[0, :] = z
    M[np.arange(1, N), np.arange(1, N)] = d[1:]
    return M


@pytest.mark.parametrize("N,seed", [(1, 0), (2, 1), (5, 2), (40, 3), (200, 4)])
def test_secular_roots_are_singular_values_of_M(N, seed):
    d, z = _random_M(N, seed)
    org, tau, omega = merge.secular_roots(d, z)
    # library pin: singular values of the dense M (Eq. diag-one-side-M)
    ref = np.sort(np.linalg.svd(_dense_M(d, z), compute_uv=False))
    assert np.max(np.abs(omega - ref)) <= 8 * N * EPS * ref[-1]
    # interlacing d_i < w_i < d_{i+1}
    assert np.all(omega > d) and np.all(omega[:-1] < d[1:])
    # the origin is the nearer pole
    assert np.all(np.abs(tau) <= 0.5 * np.concatenate((np.diff(d), [np.inf])) * (1 + 1e-12))
    f, scale = merge.secular_f(d, z, org, tau)
    assert np.all(np.abs(f) <= 64 * N * EPS * scale)


def test_secular_roots_near_tiny_weight_poles_first_order():
    # A pole d_o with a tiny weight z_o has a root w with x = w^2 - d_o^2
    # = z_o^2 / g(d_o) up to a relative O(x) term, where g is f without the
    # z_o term (Eq. M-svd-val: z_o^2 / (d_o^2 - w^2) + g(w) = 0); so
    # tau = w - d_o = x / (w + d_o) ~ x / (2 d_o).  The bisection oracle
    # resolves these offsets (1e-38 .. 1e-20) to their own relative accuracy.
    rng = np.random.default_rng(11)
    N = 200
    d = np.concatenate(([0.0, 2.2654e-11, 3.1e-10, 6.2e-9], np.sort(rng.uniform(1e-3, 1.0, N - 4))))
    for i in range(5, N):
        d[i] = max(d[i], d[i - 1] + 1e-4)
    z = rng.uniform(0.05, 0.5, N) * rng.choice([-1.0, 1.0], N)
    z[0], z[1], z[2], z[3] = 0.104, -8.82e-15, 6.6e-12, 3.3e-13
    z[50], z[51] = 3e-13, -2e-14
    org, tau, omega = merge.secular_roots(d, z)
    for o in (1, 2, 3, 50, 51):
        rest = np.arange(N) != o
        g = 1.0 + np.sum(z[rest] ** 2 / ((d[rest] - d[o]) * (d[rest] + d[o])))
        x = z[o] ** 2 / g
        tau_pred = x / (2.0 * d[o])
        i = (o - 1) if x < 0 else o               # the root on that side of d_o
        assert org[i] == o
        assert abs(tau[i] - tau_pred) <= 1e-12 * abs(tau_pred)
    f, scale = merge.secular_f(d, z, org, tau)
    assert np.all(np.abs(f) <= 64 * N * EPS * scale)


@pytest.mark.parametrize("z1", [1e-3, 1e-8, 1e-12])
def test_last_root_with_tiny_weight_closed_form(z1):
    """Two poles d = (0, 1), z = (z0, z1) with z1^2 below eps: the last root
    omega = 1 + tau sits within an ulp of its pole.  Closed form: x = omega^2
    - 1 solves x^2 + (1 - z0^2 - z1^2) x - z1^2 = 0 (the characteristic
    polynomial of M^T M for M = [[z0, z1], [0, 1]]), whose positive root,
    written without cancellation, is 2 z1^2 / (b + sqrt(b^2 + 4 z1^2)),
    b = 1 - z0^2 - z1^2; tau = x / (1 + sqrt(1 + x))."""
    z0 = 1e-20
    d, z = np.array([0.0, 1.0]), np.array([z0, z1])
    org, tau, omega = merge.secular_roots(d, z)
    b = 1.0 - z0 * z0 - z1 * z1
    x = 2.0 * z1 * z1 / (b + np.sqrt(b * b + 4.0 * z1 * z1))
    t = x / (1.0 + np.sqrt(1.0 + x))
    assert org[-1] == 1
    assert abs(tau[-1] - t) <= 4 * EPS * t
    # and the vectors of M built from it are orthonormal (no zero denominator)
    zt = merge.lowner_ztilde(d, z, org, tau)
    UM, VM = merge.m_vectors(d, zt, org, tau)
    assert check.orth_err(UM) <= 8 * EPS and check.orth_err(VM) <= 8 * EPS


def test_lowner_reproduces_z_when_separated():
    d, z = _random_M(60, 9, gap=1e-2)
    org, tau, _ = merge.secular_roots(d, z)
    zt = merge.lowner_ztilde(d, z, org, tau)
    assert np.all(np.sign(zt) == np.sign(z))
    normM = np.linalg.norm(_dense_M(d, z), 2)
    assert np.max(np.abs(zt - z)) <= 1e3 * 60 * EPS * normM


def test_lowner_roots_are_exact_for_ztilde():
    # omega are (to rounding) the exact roots of the secular equation of z~
    d, z = _random_M(80, 10, gap=1e-3)
    org, tau, _ = merge.secular_roots(d, z)
    zt = merge.lowner_ztilde(d, z, org, tau)
    f, scale = merge.secular_f(d, zt, org, tau)
    assert np.all(np.abs(f) <= 64 * 80 * EPS * scale)


@pytest.mark.parametrize("N,seed", [(1, 1), (3, 2), (64, 5), (300, 6)])
def test_m_vectors_orthonormal_and_exact(N, seed):
    d, z = _random_M(N, seed, gap=1e-4)
    org, tau, omega = merge.secular_roots(d, z)
    zt = merge.lowner_ztilde(d, z, org, tau)
    UM, VM = merge.m_vectors(d, zt, org, tau)
    assert check.orth_err(UM) <= 16 * N * EPS
    assert check.orth_err(VM) <= 16 * N * EPS
    Mt = _dense_M(d, zt)
    # M~ v_i = w_i u_i (Eq. M-svd-vec)
    R = Mt @ VM - UM * omega[None, :]
    assert np.linalg.norm(R) <= 16 * N * EPS * np.linalg.norm(Mt)


def test_deflation_cases_n3_golden():
    with open(os.path.join(GOLDEN, "deflation_n3.json")) as fh:
        g = json.load(fh)
    for case in g["cases"]:
        d = np.array(case["d"])
        z = np.array(case["z"])
        tol = merge.deflation_tol(d, 0.5, 0.5)
        assert tol == 8 * EPS * max(np.max(np.abs(d)), 0.5)
        out = merge.deflate(d, z, tol)
        assert out["keep"].tolist() == case["keep"], case["name"]
        assert out["defl"].tolist() == case["defl"], case["name"]
        assert np.allclose(out["dval"], case["dval"], rtol=0, atol=0), case["name"]
        if case["z0_is_tol"]:
            assert out["zkeep"][0] == tol
            assert np.allclose(out["zkeep"][1:], case["zkeep_tail"], rtol=0, atol=0)
        else:
            assert np.allclose(out["zkeep"], case["zkeep"], rtol=1e-15, atol=0), case["name"]
        if "rot" in case:
            kind, p, q, c, s = out["rots"][0]
            r = case["rot"]
            assert (kind, p, q) == (r["kind"], r["p"], r["q"])
            assert abs(c - r["c"]) <= 2 * EPS and abs(s - r["s"]) <= 2 * EPS


def test_deflation_is_backward_stable():
    # P M Q = [[M1, 0], [0, D]] + O(tol): rebuild from the deflated pieces
    rng = np.random.default_rng(12)
    N = 30
    d = np.concatenate(([0.0], np.sort(rng.uniform(0, 1, N - 1))))
    d[5] = d[4] + 1e-17          # close pair
    d[1] = 3e-17                 # close to d_0 = 0
    z = rng.uniform(-0.5, 0.5, N)
    z[9] = 1e-18                 # small z
    tol = merge.deflation_tol(d, 0.5, 0.5)
    out = merge.deflate(d, z, tol)
    I = np.eye(N)
    Wr, Vr = merge.apply_rotations(out["rots"], I, I)
    M = _dense_M(d, z)
    # rotated basis: M = Wr Mdef Vr^T with Mdef block diagonal after reordering
    Mdef = Wr.T @ M @ Vr
    keep, defl = out["keep"], out["defl"]
    target = np.zeros((N, N))
    target[np.ix_(keep, keep)] = _dense_M(d[keep], out["zkeep"])
    target[defl, defl] = out["dval"]
    assert np.linalg.norm(Mdef - target) <= 8 * tol
    assert set(keep.tolist()) | set(defl.tolist()) == set(range(N))
    assert 9 in defl.tolist() and 1 in defl.tolist() and 4 in defl.tolist()


@pytest.mark.parametrize("kind,n,leaf", [("uniform", 33, 16), ("uniform", 256, 16), ("graded", 256, 16),
                                         ("clustered", 256, 16), ("ones", 100, 8), ("uniform", 257, 32)])
def test_numpy_bdc_model_matches_qr(kind, n, leaf):
    d, e = inputs.make(kind, n, {"uniform": 0, "graded": 1, "clustered": 2, "ones": 0}[kind])
    s, U, VT = merge.bdc_svd(d, e, leaf)
    ref = oracle.sigma_only(d, e)
    assert check.sigma_rel_err(s, ref) <= 1e-13 * n
    assert oracle.residual(d, e, s, U, VT) <= 1e-13 * n
    assert check.orth_err(U) <= 1e-13 * n
    assert check.orth_err(VT.T) <= 1e-13 * n


def test_numpy_bdc_full_deflation():
    d, _ = inputs.uniform(64, 5)
    e = np.zeros(63)
    s, U, VT = merge.bdc_svd(d, e, 8)
    # every merge deflates fully; only the scaling by max|d| rounds
    assert np.max(np.abs(s - np.sort(d)[::-1])) <= 2 * EPS * np.max(d)
    assert oracle.residual(d, e, s, U, VT) <= 4 * EPS
