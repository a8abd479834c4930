"""FP64 CPU oracle for the dense front and back end of the SVD (test
infrastructure only; see the package docstring for who may import it).

The paper's SVD of a dense A (Sec. 4) is: an optional QR factorization for
tall-and-skinny A (Sec. 4.3), the reduction A = Q1 B P1^T to upper bidiagonal
form by Householder reflectors (Sec. 4.1), the bidiagonal SVD B = U2 S V2^T
(Sec. 4.2), and the back-transformation U = Q1 U2, V^T = V2^T P1^T
(Sec. 4.3).  This module restates each step unblocked, one reflector at a
time, in the order the paper defines it (Sec. 4.1, Eqs. gebrd-house and
tail-nonblock; Sec. 4.3, Eq. orgqr-q):

* ``householder``  the reflector H = I - tau y y^T with H x = beta e_1,
  beta = -sign(x_1) ||x||_2, y = (1, x_2 / (x_1 - beta), ...), tau =
  (beta - x_1) / beta (the same sign convention as LAPACK's larfg; tau = 0
  when x_2..x_n are already zero).
* ``gebrd``  column reflector H_i then row reflector G_i for i = 1..n,
  each applied to the whole trailing matrix at once (no blocking), with the
  reflectors stored LAPACK style: y_i below the diagonal of column i, u_i to
  the right of the superdiagonal of row i.
* ``form_q`` / ``form_p``  Q1 = H_1 ... H_n and P1 = G_1 ... G_{n-1} as
  explicit matrices (Eq. gebrd-house).
* ``geqrf`` / ``orgqr``  Householder QR and its explicit Q (Eq. orgqr-q).
* ``gesvd``  the whole SVD: [geqrf, orgqr] -> gebrd -> oracle.bdsqr -> back
  transformation.

Everything is FP64 numpy on the host; a matrix product of numpy is the only
library primitive used (the unblocked updates are rank-one outer products).
"""
from __future__ import annotations

import numpy as np


def householder(x):
    """(y, tau, beta) with (I - tau y y^T) x = beta e_1, y[0] = 1."""
    x = np.asarray(x, dtype=np.float64)
    alpha = float(x[0])
    rest = x[1:]
    y = np.zeros_like(x)
    y[0] = 1.0
    if not np.any(rest):
        return y, 0.0, alpha                      # already a multiple of e_1: H = I
    # ||x|| as s ||x / s||, s = max |x_j|: no overflow or underflow of the squares
    s = float(np.max(np.abs(x)))
    xs = x / s
    norm = s * float(np.sqrt(np.dot(xs, xs)))
    beta = -norm if alpha >= 0.0 else norm
    y[1:] = rest / (alpha - beta)
    tau = (beta - alpha) / beta
    return y, tau, beta


def gebrd(A):
    """Bidiagonalize A (m x n, m >= n): returns (Ar, d, e, tauq, taup) where
    Q1^T A P1 is upper bidiagonal with diagonal d[n] and superdiagonal
    e[n-1], and Ar holds the reflectors (column i below the diagonal: y_i
    with y_i[i] = 1 implicit; row i right of the superdiagonal: u_i with
    u_i[i+1] = 1 implicit)."""
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    m, n = A.shape
    if m < n:
        raise ValueError("gebrd oracle: m >= n")
    d = np.zeros(n)
    e = np.zeros(max(n - 1, 0))
    tauq = np.zeros(n)
    taup = np.zeros(n)
    for i in range(n):
        # H_i annihilates A[i+1:, i]; applied to the trailing columns
        y, t, beta = householder(A[i:, i])
        d[i] = beta
        tauq[i] = t
        if i + 1 < n and t != 0.0:
            w = y @ A[i:, i + 1:]
            A[i:, i + 1:] -= t * np.outer(y, w)
        A[i, i] = beta
        A[i + 1:, i] = y[1:]
        if i + 1 < n:
            # G_i annihilates A[i, i+2:]; applied to the trailing rows
            u, p, beta = householder(A[i, i + 1:])
            e[i] = beta
            taup[i] = p
            if i + 1 < m and p != 0.0:
                w = A[i + 1:, i + 1:] @ u
                A[i + 1:, i + 1:] -= p * np.outer(w, u)
            A[i, i + 1] = beta
            A[i, i + 2:] = u[1:]
    return A, d, e, tauq, taup


def _col_reflector(Ar, i):
    m = Ar.shape[0]
    y = np.zeros(m)
    y[i] = 1.0
    y[i + 1:] = Ar[i + 1:, i]
    return y


def _row_reflector(Ar, i):
    n = Ar.shape[1]
    u = np.zeros(n)
    u[i + 1] = 1.0
    u[i + 2:] = Ar[i, i + 2:]
    return u


def form_q(Ar, tauq, ncols=None):
    """Q1 = H_1 H_2 ... H_n, its first ncols columns (default n)."""
    m, n = Ar.shape
    k = n if ncols is None else ncols
    Q = np.eye(m, k)
    for i in range(n - 1, -1, -1):               # H_1 (H_2 (... (H_n I)))
        y = _col_reflector(Ar, i)
        Q -= tauq[i] * np.outer(y, y @ Q)
    return Q


def form_p(Ar, taup):
    """P1 = G_1 G_2 ... G_{n-1} (n x n)."""
    n = Ar.shape[1]
    P = np.eye(n)
    for i in range(n - 2, -1, -1):
        u = _row_reflector(Ar, i)
        P -= taup[i] * np.outer(u, u @ P)
    return P


def geqrf(A):
    """Householder QR: (Ar, tau) with R in the upper triangle of Ar and the
    reflectors y_i (y_i[i] = 1 implicit) below the diagonal."""
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    m, n = A.shape
    tau = np.zeros(min(m, n))
    for i in range(min(m, n)):
        y, t, beta = householder(A[i:, i])
        tau[i] = t
        if i + 1 < n and t != 0.0:
            w = y @ A[i:, i + 1:]
            A[i:, i + 1:] -= t * np.outer(y, w)
        A[i, i] = beta
        A[i + 1:, i] = y[1:]
    return A, tau


def orgqr(Ar, tau, ncols=None):
    """The first ncols (default n) columns of Q = H_1 ... H_k (Eq. orgqr-q)."""
    m, n = Ar.shape
    k = n if ncols is None else ncols
    Q = np.eye(m, k)
    for i in range(len(tau) - 1, -1, -1):
        y = _col_reflector(Ar, i)
        Q -= tau[i] * np.outer(y, y @ Q)
    return Q


def bidiagonal(d, e):
    n = len(d)
    B = np.diag(np.asarray(d, dtype=np.float64))
    if n > 1:
        B += np.diag(np.asarray(e, dtype=np.float64), 1)
    return B


def gesvd(A, qr_first=None):
    """A = U diag(s) V^T (m >= n), s descending: the paper's pipeline with
    the oracle's own steps (QR first when m >= 1.6 n unless told)."""
    import oracle
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if qr_first is None:
        qr_first = m >= 1.6 * n
    if qr_first:
        Ar, tau = geqrf(A)
        Q = orgqr(Ar, tau)
        R = np.triu(Ar[:n, :n])
        s, Ur, VT = gesvd(R, qr_first=False)
        return s, Q @ Ur, VT
    Ar, d, e, tq, tp = gebrd(A)
    s, U2, VT2 = oracle.bdsqr(d, e)
    U = form_q(Ar, tq) @ U2
    VT = VT2 @ form_p(Ar, tp).T
    return s, U, VT
