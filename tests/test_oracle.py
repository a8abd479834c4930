"""Pins for the FP64 QR oracle against facts that do not come from it.

Closed forms, invariants, special cases, a library SVD (LAPACK via numpy),
Sturm bisection (a different algorithm), and exact characteristic
polynomials (sympy) on tiny integer matrices.
"""
import numpy as np
import pytest

import oracle
from oracle import check
from paper_2508_11467_gb300 import inputs

EPS = np.finfo(np.float64).eps


def closed_form_ones(n):
    k = np.arange(1, n + 1)
    return 2.0 * np.cos(k * np.pi / (2 * n + 1))


@pytest.mark.parametrize("n", [1, 2, 3, 8, 64, 256])
def test_closed_form_d_e_one(n):
    # d = e = 1: B B^T is tridiag(1; 2,...,2,1... ) with eigenvalues 4cos^2(k pi/(2n+1))
    d, e = inputs.ones(n)
    ex = closed_form_ones(n)
    s = oracle.sigma_only(d, e)
    assert np.max(np.abs(s - ex)) <= 8 * n * EPS
    s2, U, VT = oracle.bdsqr(d, e)
    assert np.max(np.abs(s2 - ex)) <= 8 * n * EPS
    assert oracle.residual(d, e, s2, U, VT) <= 8 * n * EPS
    if n <= 64:
        st = oracle.sturm_sigma(d, e)
        assert np.max(np.abs(st - ex)) <= 8 * EPS * 2.0


def test_n1_and_n2_closed_forms():
    s, U, VT = oracle.bdsqr(np.array([-3.0]), np.zeros(0))
    assert s[0] == 3.0 and abs(U[0, 0] * VT[0, 0] * 3.0 - (-3.0)) == 0.0
    rng = np.random.default_rng(5)
    for _ in range(50):
        a, b, c = rng.uniform(-2, 2, 3)
        s = oracle.sigma_only(np.array([a, c]), np.array([b]))
        # s1^2 + s2^2 = a^2 + b^2 + c^2 and s1 s2 = |a c| (trace/determinant of B^T B)
        assert abs(s[0] ** 2 + s[1] ** 2 - (a * a + b * b + c * c)) <= 16 * EPS * (a * a + b * b + c * c)
        assert abs(s[0] * s[1] - abs(a * c)) <= 16 * EPS * (a * a + b * b + c * c)
        assert s[0] >= s[1] >= 0.0


def test_diagonal_input_gives_sorted_abs():
    rng = np.random.default_rng(7)
    d = rng.uniform(-2, 2, 40)
    e = np.zeros(39)
    s, U, VT = oracle.bdsqr(d, e)
    assert np.array_equal(s, np.sort(np.abs(d))[::-1])
    # U and V are signed permutations
    assert np.allclose(np.abs(U).sum(axis=0), 1.0) and np.allclose(np.abs(VT).sum(axis=1), 1.0)
    assert oracle.residual(d, e, s, U, VT) <= 4 * EPS


@pytest.mark.parametrize("kind,n", [("uniform", 200), ("graded", 256), ("clustered", 128)])
def test_against_lapack(kind, n):
    d, e = inputs.make(kind, n, {"uniform": 0, "graded": 1, "clustered": 2}[kind])
    ref = np.linalg.svd(oracle.dense(d, e), compute_uv=False)
    s, U, VT = oracle.bdsqr(d, e)
    assert check.sigma_rel_err(s, ref) <= 4 * n * EPS
    assert oracle.residual(d, e, s, U, VT) <= 4 * n * EPS
    assert check.orth_err(U) <= 4 * n * EPS
    assert check.orth_err(VT.T) <= 4 * n * EPS
    assert check.e_svd(d, e, s, U, VT) <= 4 * n * EPS


@pytest.mark.parametrize("k", [-1033, -700, 480])
def test_power_of_two_scaling_against_lapack(k):
    """sigma(2^k B) = 2^k sigma(B): the oracle on B scaled by 2^k (k = -1033
    puts every entry below the normal range) against LAPACK on the same
    entries scaled back to order one (exact).  Subnormal outputs keep the
    spacing 2^-1074, which the tolerance adds."""
    n = 60
    d, e = inputs.uniform(n, 31)
    ds, es = np.ldexp(d, k), np.ldexp(e, k)
    du, eu = np.ldexp(ds, -k), np.ldexp(es, -k)     # the entries the oracle sees, at order one
    ref = np.linalg.svd(oracle.dense(du, eu), compute_uv=False)
    s, U, VT = oracle.bdsqr(ds, es)
    su = np.ldexp(s, -k)
    tol = 4 * n * EPS + 2.0 ** (-1074 - k) / ref[0]
    assert check.sigma_rel_err(su, ref) <= tol
    assert oracle.residual(du, eu, su, U, VT) <= tol
    assert check.orth_err(U) <= 4 * n * EPS and check.orth_err(VT.T) <= 4 * n * EPS


def test_entries_across_the_exponent_range_against_lapack():
    """Entries of 1e150 beside entries of 1e-170 (below the normal range once
    divided by the largest): norm-wise against LAPACK."""
    n = 80
    d, e = inputs.uniform(n, 32)
    d, e = d * 1e150, e * 1e150
    d[::7] = 1e-170
    e[3::11] = -1e-170
    ref = np.linalg.svd(oracle.dense(d, e), compute_uv=False)
    s, U, VT = oracle.bdsqr(d, e)
    assert check.sigma_rel_err(s, ref) <= 4 * n * EPS
    assert oracle.residual(d, e, s, U, VT) <= 4 * n * EPS
    assert check.orth_err(U) <= 4 * n * EPS and check.orth_err(VT.T) <= 4 * n * EPS


def test_invariants_graded():
    n = 256
    d, e = inputs.graded(n, 1)
    s = oracle.sigma_only(d, e)
    fro2 = np.sum(d * d) + np.sum(e * e)
    assert abs(np.sum(s * s) - fro2) <= 4 * n * EPS * fro2
    # prod s_i = prod |d_i| (det B), compared in logs: 8 decades of grading
    assert abs(np.sum(np.log(s)) - np.sum(np.log(np.abs(d)))) <= 1e-9


def test_sturm_matches_qr_tiny():
    for n in range(1, 33, 5):
        d, e = inputs.uniform(n, 11 + n)
        st = oracle.sturm_sigma(d, e)
        s = oracle.sigma_only(d, e)
        assert np.max(np.abs(st - s)) <= 8 * n * EPS * s[0]


def test_zero_diagonal_entry():
    d, e = inputs.uniform(50, 3)
    d = d.copy()
    d[17] = 0.0
    s, U, VT = oracle.bdsqr(d, e)
    assert s[-1] <= 8 * 50 * EPS
    assert oracle.residual(d, e, s, U, VT) <= 8 * 50 * EPS
    d2 = d.copy()
    d2[17] = 1.0
    d2[-1] = 0.0
    s, U, VT = oracle.bdsqr(d2, e)
    assert s[-1] <= 8 * 50 * EPS
    assert oracle.residual(d2, e, s, U, VT) <= 8 * 50 * EPS


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_exact_charpoly(seed):
    """Tiny integer bidiagonals: sigma^2 = roots of det(B^T B - x I), exact in sympy."""
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(100 + seed)
    n = 3 + seed  # 3, 4, 5
    d = rng.integers(1, 6, n).astype(float)
    e = rng.integers(1, 6, n - 1).astype(float)
    B = sympy.zeros(n, n)
    for i in range(n):
        B[i, i] = int(d[i])
        if i + 1 < n:
            B[i, i + 1] = int(e[i])
    x = sympy.symbols("x")
    p = (B.T * B - x * sympy.eye(n)).det()
    roots = sorted([float(sympy.re(r)) for r in sympy.Poly(p, x).nroots(n=40)], reverse=True)
    ex = np.sqrt(np.array(roots))
    s = oracle.sigma_only(d, e)
    assert np.max(np.abs(s - ex)) <= 8 * n * EPS * ex[0]


def test_residual_detects_wrong_vectors():
    # the residual checker is not vacuous: a swapped pair of columns fails it
    d, e = inputs.uniform(20, 4)
    s, U, VT = oracle.bdsqr(d, e)
    U2 = U.copy()
    U2[:, [0, 1]] = U2[:, [1, 0]]
    assert oracle.residual(d, e, s, U2, VT) > 0.1
    assert oracle.residual(d, e, s, U, VT) < 1e-13
