"""Seeded synthetic bidiagonals (shared by the GPU path's tests and the oracle).

This module holds only random-number generation and the input recipes; it
contains none of the SVD method's arithmetic and imports nothing else from
the package.

Generator: splitmix64 (Steele, Lea, Flood 2014) used counter-based: value i
of stream s under seed k is mix(k * G + s * H + (i + 1) * G) with
G = 0x9E3779B97F4A7C15, H = 0x632BE59BD9B4E019, and
mix(x) = x ^ (x >> 30) * 0xBF58476D1CE4E5B9 ; x ^ (x >> 27) * 0x94D049BB133111EB ;
x ^ (x >> 31).  Uniforms on [0, 1) are (x >> 11) * 2^-53; Gaussians use
Box-Muller on two uniform streams.

Recipes (n x n upper bidiagonal, diagonal d[n], superdiagonal e[n-1]):
  uniform   d, e ~ U(0.5, 1.5)
  graded    d_i = 10^(-8 i / n) * U(0.5, 1.5), e_i = 0.5 d_i   (i = 0..n-1)
  clustered d = e = 1 + 1e-10 * N(0, 1)
  ones      d = e = 1  (sigma_k = 2 cos(k pi / (2n + 1)))
  batch     n_k = floor(exp(U(ln 32, ln 1024))), each matrix 'uniform'

Dense test matrices (m x n, m >= n) with prescribed singular values, after
the SVD_arith / SVD_geo / SVD_logrand kinds of the paper's test set with
condition number kappa: sigma_i = 1 - (i / (n-1)) (1 - 1/kappa) (arith),
kappa^(-i/(n-1)) (geo), exp(U(ln(1/kappa), 0)) sorted descending
(logrand).  A = Qm[:, :n] diag(sigma) Qn^T with orthogonal factors
Q = D1 P1 C P2 D2 built in closed form: C the orthonormal DCT-II matrix
C[k, j] = c_k cos(pi (2 j + 1) k / (2 N)), P random permutations, D random
signs (no factorization is used to make them).
"""
from __future__ import annotations

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_H = np.uint64(0x632BE59BD9B4E019)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(x: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        x = (x ^ (x >> np.uint64(30))) * _M1
        x = (x ^ (x >> np.uint64(27))) * _M2
        return x ^ (x >> np.uint64(31))


def uniform01(seed: int, stream: int, count: int) -> np.ndarray:
    """count uniforms on [0, 1) from (seed, stream), counter-based."""
    i = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _G + np.uint64(stream) * _H
        x = _mix(base + i * _G)
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """count standard normals by Box-Muller on streams (2s, 2s+1) + 1000."""
    u1 = 1.0 - uniform01(seed, 1000 + 2 * stream, count)     # (0, 1]
    u2 = uniform01(seed, 1001 + 2 * stream, count)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def uniform(n: int, seed: int = 0):
    d = 0.5 + uniform01(seed, 0, n)
    e = 0.5 + uniform01(seed, 1, max(n - 1, 0))
    return d, e


def graded(n: int, seed: int = 1):
    i = np.arange(n, dtype=np.float64)
    d = 10.0 ** (-8.0 * i / max(n, 1)) * (0.5 + uniform01(seed, 0, n))
    e = 0.5 * d[: max(n - 1, 0)]
    return d, e


def clustered(n: int, seed: int = 2):
    d = 1.0 + 1e-10 * normal(seed, 0, n)
    e = 1.0 + 1e-10 * normal(seed, 1, max(n - 1, 0))
    return d, e


def ones(n: int):
    return np.ones(n), np.ones(max(n - 1, 0))


KINDS = {"uniform": uniform, "graded": graded, "clustered": clustered}


def make(kind: str, n: int, seed: int):
    if kind == "ones":
        return ones(n)
    return KINDS[kind](n, seed)


def batch_sizes(count: int = 2048, seed: int = 3, lo: int = 32, hi: int = 1024) -> np.ndarray:
    """n_k = floor(exp(U(ln lo, ln hi))) for k < count (log-uniform sizes)."""
    u = uniform01(seed, 7, count)
    n = np.floor(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)
    return np.clip(n, lo, hi)


def batch(count: int = 2048, seed: int = 3, lo: int = 32, hi: int = 1024):
    """List of (d, e) uniform bidiagonals with log-uniform sizes."""
    sizes = batch_sizes(count, seed, lo, hi)
    out = []
    for k, n in enumerate(sizes):
        d = 0.5 + uniform01(seed, 100 + 2 * k, int(n))
        e = 0.5 + uniform01(seed, 101 + 2 * k, int(n) - 1)
        out.append((d, e))
    return out


def dct_orthogonal(N: int, seed: int, stream: int, cols: int = None) -> np.ndarray:
    """The first `cols` columns (default N) of a randomized N x N orthogonal
    matrix D1 P1 C P2 D2 (C the orthonormal DCT-II matrix)."""
    cols = N if cols is None else cols
    p1 = np.argsort(uniform01(seed, stream, N))
    p2 = np.argsort(uniform01(seed, stream + 1, N))[:cols]
    s1 = np.where(uniform01(seed, stream + 2, N) < 0.5, -1.0, 1.0)
    s2 = np.where(uniform01(seed, stream + 3, cols) < 0.5, -1.0, 1.0)
    k = p1[:, None].astype(np.int64)                  # rows of C, permuted
    j = p2[None, :].astype(np.int64)                  # columns of C, permuted
    # the angle pi (2j+1) k / (2N) reduced exactly modulo 2 pi on the integers
    r = ((2 * j + 1) * k) % (4 * N)
    C = np.cos(np.pi * r.astype(np.float64) / (2.0 * N)) * np.sqrt(2.0 / N)
    C[p1 == 0, :] *= np.sqrt(0.5)
    return s1[:, None] * C * s2[None, :]


def dense_sigma(kind: str, n: int, kappa: float, seed: int) -> np.ndarray:
    i = np.arange(n, dtype=np.float64)
    t = i / max(n - 1, 1)
    if kind == "arith":
        return 1.0 - t * (1.0 - 1.0 / kappa)
    if kind == "geo":
        return kappa ** (-t)
    if kind == "logrand":
        return np.sort(np.exp(np.log(1.0 / kappa) * uniform01(seed, 40, n)))[::-1].copy()
    raise ValueError(kind)


def dense(kind: str, m: int, n: int, kappa: float = 1e4, seed: int = 0):
    """(Qm_cols (m x n), sigma (n), Qn (n x n)): A = Qm_cols diag(sigma) Qn^T."""
    return dct_orthogonal(m, seed, 50, n), dense_sigma(kind, n, kappa, seed), dct_orthogonal(n, seed, 60)
