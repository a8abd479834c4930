"""Pins of the dense oracle (oracle/dense.py): Householder reflectors, the
bidiagonalization of Sec. 4.1, the QR factorization of Sec. 4.3 and the
whole SVD pipeline, checked against identities and LAPACK (numpy) on the CPU.
Each pin fails for a plausible slip (a sign, a transposed application, a
dropped scale): the mutation tests at the end plant such slips in the
oracle and check that the pins catch them."""
import numpy as np
import pytest

import oracle
from oracle import dense_svd as dense

EPS = np.finfo(np.float64).eps


def _rand(m, n, seed):
    return np.random.default_rng(seed).standard_normal((m, n))


@pytest.mark.parametrize("x", [[3.0, 4.0], [-3.0, 4.0, 0.0, 12.0], [2.0, 0.0, 0.0], [0.0, 1e-300, 1e-300],
                               [-1e200, 1e200]])
def test_householder_maps_to_beta_e1(x):
    x = np.asarray(x)
    y, tau, beta = dense.householder(x)
    H = np.eye(len(x)) - tau * np.outer(y, y)
    s = np.max(np.abs(x))
    nx = s * np.linalg.norm(x / s)                 # ||x|| without overflow or underflow
    hx = s * (H @ (x / s))
    assert y[0] == 1.0
    assert abs(hx[0] - beta) <= 4 * EPS * nx
    assert np.all(np.abs(hx[1:]) <= 4 * EPS * nx)
    assert np.linalg.norm(H @ H.T - np.eye(len(x))) <= 8 * EPS
    assert abs(abs(beta) - nx) <= 4 * EPS * nx
    if np.all(x[1:] == 0):
        assert tau == 0.0 and beta == x[0]
    else:
        assert 1.0 <= tau <= 2.0 and np.sign(beta) == -np.sign(x[0] if x[0] != 0 else 1.0)


@pytest.mark.parametrize("m,n", [(1, 1), (2, 2), (7, 3), (40, 30), (50, 50), (65, 17)])
def test_gebrd_reduces_to_bidiagonal(m, n):
    A = _rand(m, n, m * 100 + n)
    Ar, d, e, tq, tp = dense.gebrd(A)
    Q = dense.form_q(Ar, tq)
    P = dense.form_p(Ar, tp)
    B = dense.bidiagonal(d, e)
    nA = np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ A @ P - B) <= 20 * n * EPS * nA
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 20 * n * EPS
    assert np.linalg.norm(P.T @ P - np.eye(n)) <= 20 * n * EPS
    # the reflectors sit below the diagonal / right of the superdiagonal of Ar
    assert np.allclose(np.diag(Ar), d, rtol=0, atol=0)
    if n > 1:
        assert np.allclose(np.diag(Ar, 1), e, rtol=0, atol=0)
    # the singular values of B are A's (LAPACK, numpy)
    s = oracle.sigma_only(d, e)
    s_ref = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(s - s_ref)) <= 20 * n * EPS * s_ref[0]


def test_gebrd_of_a_bidiagonal_is_itself():
    """A positive upper bidiagonal needs no reflector: every tau is 0 and
    (d, e) come back exactly."""
    rng = np.random.default_rng(3)
    d0, e0 = rng.uniform(0.5, 1.5, 20), rng.uniform(0.5, 1.5, 19)
    Ar, d, e, tq, tp = dense.gebrd(dense.bidiagonal(d0, e0))
    assert np.array_equal(d, d0) and np.array_equal(e, e0)
    assert not np.any(tq) and not np.any(tp)


def test_gebrd_of_orthonormal_columns_has_unit_singular_values():
    Q, _ = np.linalg.qr(_rand(60, 25, 4))
    _, d, e, _, _ = dense.gebrd(Q)
    assert np.max(np.abs(oracle.sigma_only(d, e) - 1.0)) <= 100 * EPS


@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (60, 60), (200, 31), (100, 100)])
def test_geqrf_matches_lapack_and_reconstructs(m, n):
    A = _rand(m, n, m + 7 * n)
    Ar, tau = dense.geqrf(A)
    R = np.triu(Ar[:n, :n])
    R_lapack = np.linalg.qr(A, mode="r")       # LAPACK dgeqrf: the same reflector convention
    assert np.max(np.abs(R - R_lapack)) <= 20 * n * EPS * np.linalg.norm(A)
    Q = dense.orgqr(Ar, tau)
    assert np.linalg.norm(Q @ R - A) <= 20 * n * EPS * np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 20 * n * EPS


@pytest.mark.parametrize("m,n,qr", [(30, 30, False), (80, 30, False), (80, 30, True), (200, 40, None)])
def test_gesvd_pipeline(m, n, qr):
    A = _rand(m, n, m * 3 + n)
    s, U, VT = dense.gesvd(A, qr_first=qr)
    s_ref = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(s - s_ref)) <= 40 * n * EPS * s_ref[0]
    assert np.linalg.norm(U * s[None, :] @ VT - A) <= 40 * n * EPS * np.linalg.norm(A)
    assert np.linalg.norm(U.T @ U - np.eye(n)) <= 40 * n * EPS
    assert np.linalg.norm(VT @ VT.T - np.eye(n)) <= 40 * n * EPS


# ------------------------------------------------------- planted mistakes
def test_pins_catch_a_wrong_reflector_sign(monkeypatch):
    real = dense.householder

    def flipped(x):
        y, tau, beta = real(x)
        return y, tau, -beta                       # the reflector's image with the wrong sign
    monkeypatch.setattr(dense, "householder", flipped)
    A = _rand(30, 20, 9)
    Ar, d, e, tq, tp = dense.gebrd(A)
    Q, P = dense.form_q(Ar, tq), dense.form_p(Ar, tp)
    assert np.linalg.norm(Q.T @ A @ P - dense.bidiagonal(d, e)) > 1e-3


def test_pins_catch_a_dropped_tau(monkeypatch):
    real = dense.householder

    def lazy(x):
        y, tau, beta = real(x)
        return y, 1.0 if tau else 0.0, beta        # tau replaced by 1
    monkeypatch.setattr(dense, "householder", lazy)
    A = _rand(40, 10, 10)
    Ar, tau = dense.geqrf(A)
    assert np.max(np.abs(np.triu(Ar[:10, :10]) - np.linalg.qr(A, mode="r"))) > 1e-3
