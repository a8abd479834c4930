"""Accuracy metrics for a computed bidiagonal SVD (test infrastructure only).

* ``sigma_rel_err``  -- max_i |s_i - s^_i| / s^_max
* ``orth_err``       -- ||X^T X - I||_F (one library matmul; never the GEMM
  of the GPU path)
* ``residual``       -- ||B V - U S||_F / ||B||_F, O(n^2) (see oracle.residual)
* ``e_sigma``        -- the paper's E_sigma = ||S_1 - S_2||_F / n (Sec. 5.1)
* ``e_svd``          -- the paper's E_svd = ||A - U S V^T||_F / ||A||_F
  (Sec. 5.1), with A = B dense
"""
from __future__ import annotations

import numpy as np

from . import dense, residual


def sigma_rel_err(s, s_ref) -> float:
    s = np.asarray(s, dtype=np.float64)
    s_ref = np.asarray(s_ref, dtype=np.float64)
    if s_ref.size == 0:
        return 0.0
    scale = float(np.max(np.abs(s_ref)))
    if scale == 0.0:
        return float(np.max(np.abs(s)))
    return float(np.max(np.abs(s - s_ref)) / scale)


def orth_err(X) -> float:
    X = np.asarray(X, dtype=np.float64)
    G = X.T @ X
    G[np.diag_indices_from(G)] -= 1.0
    return float(np.linalg.norm(G))


def e_sigma(s, s_ref) -> float:
    s = np.asarray(s, dtype=np.float64)
    return float(np.linalg.norm(s - np.asarray(s_ref)) / max(s.size, 1))


def e_svd(d, e, s, U, VT) -> float:
    B = dense(d, e)
    R = B - (np.asarray(U) * np.asarray(s)[None, :]) @ np.asarray(VT)
    nb = np.linalg.norm(B)
    return float(np.linalg.norm(R) / nb) if nb > 0 else float(np.linalg.norm(R))


__all__ = ["sigma_rel_err", "orth_err", "residual", "e_sigma", "e_svd"]
