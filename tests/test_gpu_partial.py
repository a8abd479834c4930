"""Partial-vector solves (the "next" row of the solve with vectors for one
side only, Sec. 4.2; the paper's accuracy study distinguishes solves with and
without vectors, Sec. 5.1).

* vectors="v" skips the U side of every merge.  The V side runs the same
  arithmetic as the full solve, so S and V^T must equal the full solve's bit
  for bit.
* vectors="u" solves J B^T J (J the reversal: an upper bidiagonal with d and
  e reversed) and writes its right vectors, rows reversed, as U.

Both are also checked against the FP64 oracle: singular values (relative
error <= 1e-13 n), orthogonality (cuBLAS, <= 1e-13 n) and the one-sided
residual of the side formed, ||B^T B V - V S^2||_F / ||B||_F^2 or
||B B^T U - U S^2||_F / ||B||_F^2 (<= 1e-13 n).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import check
from paper_2508_11467_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bdc():
    from paper_2508_11467_gb300 import bdc as b
    from paper_2508_11467_gb300 import build
    build.build()
    b.lib()
    return b


def _orth(X):
    G = X.t() @ X
    G.diagonal().sub_(1.0)
    return float(torch.linalg.norm(G))


def _bmul(d, e, X):
    """B X for the upper bidiagonal (d, e) (rows of X)."""
    Y = d[:, None] * X
    Y[:-1] += e[:, None] * X[1:]
    return Y


def _btmul(d, e, X):
    """B^T X."""
    Y = d[:, None] * X
    Y[1:] += e[:, None] * X[:-1]
    return Y


def _one_sided(d, e, S, X, side):
    d = torch.as_tensor(d, device="cuda")
    e = torch.as_tensor(e, device="cuda")
    nb2 = float((d * d).sum() + (e * e).sum())
    if side == "v":    # B^T B V - V S^2
        R = _btmul(d, e, _bmul(d, e, X)) - X * (S * S)[None, :]
    else:              # B B^T U - U S^2
        R = _bmul(d, e, _btmul(d, e, X)) - X * (S * S)[None, :]
    return float(torch.linalg.norm(R)) / max(nb2, 1e-300)


CASES = [(n, kind) for n in (1, 2, 5, 33, 300, 1000) for kind in ("uniform", "graded", "clustered")] + \
        [(4096, "uniform"), (4096, "graded"), (4096, "clustered")]


@pytest.mark.parametrize("n,kind", CASES)
@pytest.mark.parametrize("vectors", ["v", "u"])
def test_partial_vectors_match_oracle(bdc, n, kind, vectors):
    d, e = inputs.make(kind, n, 50 + n)
    dc, ec = torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda()
    prec = "exact" if n >= 1000 else "fp64"
    S, U, VT, info = bdc.svd(dc, ec, prec=prec, vectors=vectors)
    torch.cuda.synchronize()
    assert info == 0
    tol = 1e-13 * n
    s = S.cpu().numpy()
    assert np.all(np.diff(s) <= 0) and np.all(s >= 0)
    assert check.sigma_rel_err(s, oracle.sigma_only(d, e)) <= tol
    X = VT.t() if vectors == "v" else U
    assert (U is None) == (vectors == "v") and (VT is None) == (vectors == "u")
    assert _orth(X) <= tol
    assert _one_sided(d, e, S, X, vectors) <= tol
    if vectors == "v":
        # the V side is the full solve's, bit for bit
        S2, U2, VT2, _ = bdc.svd(dc, ec, prec=prec)
        assert torch.equal(S, S2) and torch.equal(VT, VT2)


@pytest.mark.parametrize("vectors", ["v", "u"])
def test_partial_vectors_n16384(bdc, vectors):
    """The headline size, split-BF16 products, one side."""
    n = 16384
    d, e = inputs.uniform(n, 0)
    S, U, VT, info = bdc.svd(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda(), prec="exact",
                             vectors=vectors)
    torch.cuda.synchronize()
    assert info == 0
    X = VT.t() if vectors == "v" else U
    tol = 1e-13 * n
    assert _orth(X) <= tol
    assert _one_sided(d, e, S, X, vectors) <= tol


def test_partial_vectors_null_outputs_and_args(bdc):
    import ctypes
    L = bdc.lib()
    n = 64
    d, e = inputs.uniform(n, 1)
    dc, ec = torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda()
    S = torch.empty(n, dtype=torch.float64, device="cuda")
    M = torch.empty((n, n), dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    for vec, u, vt, ldu, ldvt in (("v", None, M, 0, n), ("u", M, None, n, 0)):
        o = bdc.make_opts("fp64", vectors=vec)
        lw = bdc.workspace_bytes(n, o)
        work = torch.empty(lw + 256, dtype=torch.uint8, device="cuda")
        rc = L.bdc_svd_ex(n, bdc._ptr(dc), bdc._ptr(ec), bdc._ptr(u), bdc._ptr(S), bdc._ptr(vt), ldu, ldvt,
                          ctypes.byref(o), bdc._ptr(work), work.numel(), bdc._ptr(info), None)
        assert rc == 0
        torch.cuda.synchronize()
        assert int(info.item()) == 0
    # the formed side still needs its pointer and leading dimension
    o = bdc.make_opts("fp64", vectors="v")
    assert L.bdc_svd_ex(n, bdc._ptr(dc), bdc._ptr(ec), None, bdc._ptr(S), None, 0, n, ctypes.byref(o), None, 0,
                        bdc._ptr(info), None) == -6
    o.vectors = 3
    assert L.bdc_svd_ex(n, bdc._ptr(dc), bdc._ptr(ec), bdc._ptr(M), bdc._ptr(S), bdc._ptr(M), n, n,
                        ctypes.byref(o), None, 0, bdc._ptr(info), None) == -9
