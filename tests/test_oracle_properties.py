"""Property-based pins of the FP64 oracles over random small bidiagonals
whose entries mix zeros, values of order one, and tiny and huge magnitudes
(1e-150 to 1e150, either sign): the inputs on which the QR's zero-diagonal
chases, splits and scaling, and the merge model's deflation cases, are taken.

* the QR oracle against LAPACK (numpy's SVD of the dense bidiagonal);
* the numpy model of Algorithm 2 (merge.bdc_svd, leaves of 4 and 8) against
  the QR oracle;
* the dense oracle (dense_svd.gesvd, with and without the QR first) against
  LAPACK on small m x n matrices: Gaussian, with zero columns, with columns
  graded down to 1e-12, of rank one, and scaled by 1e-150 or 1e150.

Bar: singular values norm-wise within 8 n eps, residual and orthogonality of
the vectors within 8 n eps.
"""
import numpy as np
import pytest

import oracle
from oracle import check, dense_svd, merge

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

EPS = np.finfo(np.float64).eps

_entry = st.one_of(
    st.just(0.0),
    st.floats(min_value=0.5, max_value=1.5),
    st.floats(min_value=-1.5, max_value=-0.5),
    st.sampled_from([1e-150, -1e-150, 1e-20, 3e-8, 1e8, 1e150, -1e150]),
)


@st.composite
def bidiagonals(draw):
    n = draw(st.integers(min_value=1, max_value=24))
    d = np.array(draw(st.lists(_entry, min_size=n, max_size=n)), dtype=np.float64)
    e = np.array(draw(st.lists(_entry, min_size=n - 1, max_size=n - 1)), dtype=np.float64)
    scale = draw(st.sampled_from([1.0, 1e-100, 1e100]))
    return d * scale, e * scale


@settings(max_examples=300, deadline=None)
@given(bidiagonals())
def test_oracle_against_lapack_on_mixed_magnitudes(de):
    d, e = de
    n = d.shape[0]
    B = oracle.dense(d, e)
    ref = np.linalg.svd(B, compute_uv=False)
    s, U, VT = oracle.bdsqr(d, e)
    assert np.all(np.diff(s) <= 0) and np.all(s >= 0)
    if ref[0] == 0.0:
        assert np.all(s == 0.0)
        return
    assert np.max(np.abs(s - ref)) <= 8 * n * EPS * ref[0]
    assert np.array_equal(oracle.sigma_only(d, e), s)
    assert oracle.residual(d, e, s, U, VT) <= 8 * n * EPS
    assert check.orth_err(U) <= 8 * n * EPS and check.orth_err(VT.T) <= 8 * n * EPS


@settings(max_examples=150, deadline=None)
@given(bidiagonals(), st.sampled_from([4, 8]))
def test_merge_model_against_qr_on_mixed_magnitudes(de, leaf):
    d, e = de
    n = d.shape[0]
    ref = oracle.sigma_only(d, e)
    with np.errstate(all="ignore"):
        s, U, VT = merge.bdc_svd(d, e, leaf=leaf)
    s = np.asarray(s)
    assert np.all(np.isfinite(s)) and np.all(s >= 0)
    if ref[0] == 0.0:
        assert np.all(s == 0.0)
        return
    assert np.max(np.abs(np.sort(s)[::-1] - ref)) <= 8 * n * EPS * ref[0]
    assert oracle.residual(d, e, s, U, VT) <= 8 * n * EPS
    assert check.orth_err(U) <= 8 * n * EPS and check.orth_err(VT.T) <= 8 * n * EPS


@st.composite
def dense_matrices(draw):
    n = draw(st.integers(min_value=1, max_value=12))
    m = draw(st.integers(min_value=n, max_value=20))
    rng = np.random.default_rng(draw(st.integers(min_value=0, max_value=10 ** 6)))
    A = rng.standard_normal((m, n))
    kind = draw(st.sampled_from(["gauss", "zero_cols", "graded_cols", "rank1", "scaled"]))
    if kind == "zero_cols":
        A[:, rng.integers(0, n, max(1, n // 3))] = 0.0
    elif kind == "graded_cols":
        A = A * np.logspace(0, -12, n)[None, :]
    elif kind == "rank1":
        A = np.outer(rng.standard_normal(m), rng.standard_normal(n))
    elif kind == "scaled":
        A = A * draw(st.sampled_from([1e-150, 1e150]))
    return A


@settings(max_examples=200, deadline=None)
@given(dense_matrices(), st.booleans())
def test_dense_oracle_against_lapack(A, qr_first):
    m, n = A.shape
    ref = np.linalg.svd(A, compute_uv=False)
    S, U, VT = dense_svd.gesvd(A, qr_first=qr_first)
    S = np.asarray(S)
    tol = 8 * max(m, n) * EPS
    assert np.all(np.isfinite(S)) and np.all(np.diff(S) <= 0)
    if ref[0] == 0.0:
        assert np.all(S == 0.0)
        return
    assert np.max(np.abs(S - ref)) <= tol * ref[0]
    U = U[:, :n]
    assert np.linalg.norm(A - (U * S[None, :]) @ VT) <= tol * np.linalg.norm(A)
    assert check.orth_err(U) <= tol and check.orth_err(VT.T) <= tol
