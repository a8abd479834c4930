"""FP64 CPU oracle for the bidiagonal SVD (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package.  The product path
(``paper_2508_11467_gb300``) never imports it, and it never imports the
product: the two share no code.

Contents
--------
* ``bdsqr`` / ``sigma_only`` -- Golub-Kahan implicit-shift QR (plain C, FP64),
  the classical bidiagonal SVD the paper contrasts with divide-and-conquer
  (Sec. 2).  It computes the plain definition B = U diag(s) V^T that the
  divide-and-conquer of Sec. 4.2 reaches up to rounding.
* ``sturm_sigma`` -- singular values by bisection on Sturm counts of the
  2n x 2n Golub-Kahan tridiagonal; independent of the QR code.
* ``residual`` -- ||B V - U S||_F / ||B||_F in O(n^2).
* ``merge`` -- the merge-step quantities of Sec. 4.2 (secular roots, Eq. for
  z-tilde, singular vectors of M, deflation) written from their definitions
  in numpy FP64.
* ``check`` -- accuracy metrics (relative sigma error, orthogonality, the
  paper's E_sigma and E_svd of Sec. 5.1).
* ``dense_svd`` -- the dense front and back end of Sec. 4.1 and 4.3 written
  unblocked: Householder reflectors, bidiagonalization, QR, the explicit
  Q1, P1, Q and the whole SVD pipeline (numpy FP64).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle/bdsqr.c with gcc into oracle/_build/liboracle.so."""
    src = os.path.join(_HERE, "bdsqr.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    # -ffp-contract=off: no fused multiply-adds, plain IEEE double arithmetic
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_bdsqr.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.c_int,
                                         dp, ctypes.c_int, ctypes.c_int]
            lib.oracle_bdsqr.restype = ctypes.c_int
            lib.oracle_sturm_count.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double]
            lib.oracle_sturm_count.restype = ctypes.c_long
            lib.oracle_sturm_sigma.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int]
            lib.oracle_sturm_sigma.restype = ctypes.c_double
            lib.oracle_residual.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.c_int,
                                            dp, ctypes.c_int]
            lib.oracle_residual.restype = ctypes.c_double
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _de(d, e):
    d = np.ascontiguousarray(d, dtype=np.float64)
    n = d.shape[0]
    e = np.ascontiguousarray(e if e is not None else np.zeros(max(n - 1, 0)), dtype=np.float64)
    if e.shape[0] < max(n - 1, 0):
        raise ValueError("e must have n-1 entries")
    if e.shape[0] == 0:
        e = np.zeros(1)
    return d, e, n


def bdsqr(d, e, max_sweeps: int = 30):
    """Full SVD of the upper bidiagonal (d, e): returns (s, U, VT), s descending."""
    lib = _load()
    d, e, n = _de(d, e)
    s = np.zeros(max(n, 1))
    U = np.zeros((n, n), order="F")
    VT = np.zeros((n, n), order="F")
    if n == 0:
        return s[:0], U, VT
    info = lib.oracle_bdsqr(n, _ptr(d), _ptr(e), _ptr(s), _ptr(U), n, _ptr(VT), n, max_sweeps)
    if info != 0:
        raise RuntimeError(f"oracle_bdsqr failed, info={info}")
    return s[:n], U, VT


def sigma_only(d, e, max_sweeps: int = 30):
    """Singular values only (same sweeps, no vector accumulation), descending."""
    lib = _load()
    d, e, n = _de(d, e)
    s = np.zeros(max(n, 1))
    if n == 0:
        return s[:0]
    info = lib.oracle_bdsqr(n, _ptr(d), _ptr(e), _ptr(s), None, n, None, n, max_sweeps)
    if info != 0:
        raise RuntimeError(f"oracle_bdsqr failed, info={info}")
    return s[:n]


def _sigma_job(de):
    return sigma_only(*de)


def sigma_only_many(mats, workers=None):
    """sigma_only of every (d, e) in `mats`, in order, over a pool of
    spawned worker processes (the matrices are independent; each one is
    solved by the same single-threaded QR)."""
    import multiprocessing as mp
    build()
    mats = [(np.asarray(d, dtype=np.float64), np.asarray(e, dtype=np.float64)) for d, e in mats]
    workers = workers or max(1, min(len(mats), len(os.sched_getaffinity(0))))
    if workers <= 1 or len(mats) <= 1:
        return [sigma_only(d, e) for d, e in mats]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_sigma_job, mats, chunksize=max(1, len(mats) // (4 * workers)))


def sturm_count(d, e, x: float) -> int:
    """Eigenvalues below x of the Golub-Kahan tridiagonal of (d, e)."""
    lib = _load()
    d, e, n = _de(d, e)
    return int(lib.oracle_sturm_count(n, _ptr(d), _ptr(e), float(x)))


def sturm_sigma(d, e, k=None):
    """k-th largest singular value(s) by Sturm bisection (all if k is None)."""
    lib = _load()
    d, e, n = _de(d, e)
    ks = range(n) if k is None else np.atleast_1d(k)
    out = np.array([lib.oracle_sturm_sigma(n, _ptr(d), _ptr(e), int(i)) for i in ks])
    return out


def residual(d, e, s, U, VT) -> float:
    """||B V - U diag(s)||_F / ||B||_F (U columns, VT rows are the vectors)."""
    lib = _load()
    d, e, n = _de(d, e)
    s = np.ascontiguousarray(s, dtype=np.float64)
    U = np.asfortranarray(U, dtype=np.float64)
    VT = np.asfortranarray(VT, dtype=np.float64)
    return float(lib.oracle_residual(n, _ptr(d), _ptr(e), _ptr(s), _ptr(U), U.shape[0],
                                     _ptr(VT), VT.shape[0]))


def dense(d, e) -> np.ndarray:
    """The n x n upper bidiagonal as a dense array."""
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    B = np.diag(d)
    if n > 1:
        B += np.diag(np.asarray(e, dtype=np.float64)[: n - 1], 1)
    return B
