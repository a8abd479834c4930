"""End-to-end parity of the GPU divide-and-conquer SVD with the FP64 oracle.

Tolerances (FP64 path): relative singular-value error, ||B V - U S||_F/||B||_F
and ||U^T U - I||_F, ||V^T V - I||_F each <= 1e-13 * n.  Vectors are compared
by residual and orthogonality (signs and bases in clusters are not unique).
Orthogonality is measured with cuBLAS (torch.matmul), never the library's own
GEMM.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import check
from paper_2508_11467_gb300 import inputs

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def bdc():
    from paper_2508_11467_gb300 import bdc as b
    from paper_2508_11467_gb300 import build
    build.build()
    b.lib()
    return b


def _orth_gpu(X):
    G = X.t() @ X
    G.diagonal().sub_(1.0)
    return float(torch.linalg.norm(G))


def _run(bdc, d, e, **kw):
    S, U, VT, info = bdc.svd(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda(), **kw)
    torch.cuda.synchronize()
    return S, U, VT, info


def _check_full(bdc, d, e, tol_scale=1e-13, ref=None, **kw):
    n = d.shape[0]
    S, U, VT, info = _run(bdc, d, e, **kw)
    assert info == 0
    s = S.cpu().numpy()
    if ref is None:
        ref = oracle.sigma_only(d, e)
    tol = tol_scale * max(n, 1)
    err = check.sigma_rel_err(s, ref)
    res = oracle.residual(d, e, s, U.cpu().numpy(), VT.cpu().numpy())
    ou, ov = _orth_gpu(U), _orth_gpu(VT.t())
    assert np.all(np.diff(s) <= 0) and np.all(s >= 0)
    assert err <= tol, ("sigma", err, tol)
    assert res <= tol, ("residual", res, tol)
    assert ou <= tol and ov <= tol, ("orth", ou, ov, tol)
    return err, res, ou, ov


@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 31, 32])
def test_single_leaf(bdc, n):
    d, e = inputs.uniform(n, 20 + n)
    _check_full(bdc, d, e, leaf=32)


@pytest.mark.parametrize("n,leaf", [(17, 16), (33, 16), (64, 16), (100, 8), (129, 32), (257, 4)])
def test_small_trees(bdc, n, leaf):
    d, e = inputs.uniform(n, n)
    _check_full(bdc, d, e, leaf=leaf)


def test_config1_uniform_n256_leaf16(bdc):
    """n = 256, d, e ~ U(0.5, 1.5) seed 0, leaf 16: full oracle with vectors."""
    d, e = inputs.uniform(256, 0)
    s_ref, U_ref, VT_ref = oracle.bdsqr(d, e)
    assert oracle.residual(d, e, s_ref, U_ref, VT_ref) < 1e-13
    _check_full(bdc, d, e, ref=s_ref, leaf=16)


@pytest.mark.parametrize("n", [256, 4096])
def test_closed_form_ones(bdc, n):
    d, e = inputs.ones(n)
    k = np.arange(1, n + 1)
    exact = 2.0 * np.cos(k * np.pi / (2 * n + 1))
    _check_full(bdc, d, e, ref=exact, leaf=16 if n == 256 else 32)


@pytest.mark.parametrize("kind,seed", [("uniform", 0), ("graded", 1), ("clustered", 2)])
def test_config2_n4096(bdc, kind, seed):
    d, e = inputs.make(kind, 4096, seed)
    _check_full(bdc, d, e, leaf=32)


@pytest.mark.parametrize("kind", ["graded", "clustered"])
def test_ragged_sizes(bdc, kind):
    for n, leaf in [(1000, 32), (777, 16)]:
        d, e = inputs.make(kind, n, 5)
        _check_full(bdc, d, e, leaf=leaf)


def test_full_deflation_diagonal(bdc):
    d, _ = inputs.uniform(300, 6)
    e = np.zeros(299)
    S, U, VT, info = _run(bdc, d, e, leaf=16)
    assert info == 0
    assert np.max(np.abs(S.cpu().numpy() - np.sort(d)[::-1])) <= 4 * EPS
    assert oracle.residual(d, e, S.cpu().numpy(), U.cpu().numpy(), VT.cpu().numpy()) <= 4 * EPS


def test_zero_diagonal_entries(bdc):
    d, e = inputs.uniform(200, 7)
    d = d.copy()
    d[[0, 57, 99, 199]] = 0.0
    _check_full(bdc, d, e, leaf=16)


def test_all_zero_matrix(bdc):
    n = 100
    S, U, VT, info = _run(bdc, np.zeros(n), np.zeros(n - 1), leaf=16)
    assert info == 0
    assert float(S.abs().max()) == 0.0
    assert _orth_gpu(U) <= 1e-13 * n and _orth_gpu(VT.t()) <= 1e-13 * n


def test_nonfinite_input_reports_error(bdc):
    d, e = inputs.uniform(50, 8)
    d = d.copy()
    d[10] = np.nan
    S, U, VT, info = _run(bdc, d, e, leaf=16, check=False)
    assert info == bdc.BDC_ERR_NONFINITE


def test_sync_entry_point_matches_async(bdc):
    # bdc_svd uses the library defaults; bdc_svd_ex with default options must match bitwise
    d, e = inputs.uniform(300, 9)
    S1, U1, VT1, info = _run(bdc, d, e)
    S2, U2, VT2, rc = bdc.svd_sync(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda())
    assert rc == 0 and info == 0
    assert torch.equal(S1, S2) and torch.equal(U1, U2) and torch.equal(VT1, VT2)


def test_deterministic(bdc):
    d, e = inputs.graded(1000, 1)
    a = _run(bdc, d, e)
    b = _run(bdc, d, e)
    for x, y in zip(a[:3], b[:3]):
        assert torch.equal(x, y)


def test_negative_and_scaled_entries(bdc):
    d, e = inputs.uniform(300, 10)
    sgn = np.where(np.arange(300) % 3 == 0, -1.0, 1.0)
    d = d * sgn * 1e150
    e = e * sgn[:299] * 1e150
    _check_full(bdc, d, e, leaf=16)


def test_scaling_subnormal_maximum(bdc):
    """Largest entry subnormal: the scale's exponent comes from ilogb (not
    the exponent field) and every entry is scaled up by scalbn.  B and S are
    checked after multiplying both by 2^k (exact at these magnitudes), so
    that the checks themselves do not underflow; S keeps the spacing of the
    subnormal range, 2^-1074, which is 2^-41 of its largest value here."""
    n, k = 200, 1033
    d, e = inputs.uniform(n, 11)
    ds, es = np.ldexp(d, -k), np.ldexp(e, -k)
    assert np.max(np.abs(np.concatenate([ds, es]))) < np.finfo(np.float64).tiny
    S, U, VT, info = _run(bdc, ds, es, leaf=16)
    assert info == 0
    s = np.ldexp(S.cpu().numpy(), k)
    du, eu = np.ldexp(ds, k), np.ldexp(es, k)      # the same (rounded) entries, scaled up exactly
    tol = 1e-13 * n
    assert np.all(np.diff(s) <= 0) and np.all(s >= 0)
    assert check.sigma_rel_err(s, oracle.sigma_only(du, eu)) <= tol
    assert oracle.residual(du, eu, s, U.cpu().numpy(), VT.cpu().numpy()) <= tol
    assert _orth_gpu(U) <= tol and _orth_gpu(VT.t()) <= tol


def test_scaling_entries_below_normal_range(bdc):
    """Entries that leave the normal range once scaled (largest ~1e150, some
    of 1e-170: ~1e-320 after scaling), which take scalbn instead of the
    exponent arithmetic; norm-wise against the oracle on the same input."""
    d, e = inputs.uniform(300, 12)
    d, e = d * 1e150, e * 1e150
    d[::7] = 1e-170
    e[3::11] = -1e-170
    _check_full(bdc, d, e, leaf=16)


# ---------------------------------------------------------------- mixed precision
@pytest.mark.parametrize("kind,seed", [("uniform", 0), ("graded", 1), ("clustered", 2)])
def test_mixed_exact_n4096(bdc, kind, seed):
    """Split-BF16 merge products (6 slices): same FP64 tolerances as the
    FP64 path, residual well inside 1e-12."""
    d, e = inputs.make(kind, 4096, seed)
    err, res, ou, ov = _check_full(bdc, d, e, leaf=32, prec="exact", slices=6)
    assert res <= 1e-12 and ou <= 1e-12 * 4096 and ov <= 1e-12 * 4096


@pytest.mark.parametrize("kind,seed", [("uniform", 3), ("clustered", 4)])
def test_mixed_exact_auto_slices_fp64_bar(bdc, kind, seed):
    """Automatic slice count (7): the split-BF16 products meet the FP64 bar
    itself (sigma, residual and orthogonality <= 1e-13 n)."""
    d, e = inputs.make(kind, 4096, seed)
    _check_full(bdc, d, e, prec="exact")


@pytest.mark.parametrize("n,leaf", [(33, 16), (300, 16), (1000, 32)])
def test_mixed_exact_small(bdc, n, leaf):
    d, e = inputs.uniform(n, 40 + n)
    _check_full(bdc, d, e, leaf=leaf, prec="exact", slices=6)


def test_mixed_exact_closed_form(bdc):
    n = 2048
    d, e = inputs.ones(n)
    k = np.arange(1, n + 1)
    _check_full(bdc, d, e, ref=2.0 * np.cos(k * np.pi / (2 * n + 1)), leaf=32, prec="exact", slices=6)


def test_bf16x3_literal_split_error_is_reported(bdc):
    # the literal 3-term BF16 split with FP32 accumulation is ~1e-5 accurate:
    # it runs end to end and its (larger) error is what bench/DESIGN report
    d, e = inputs.make("clustered", 1024, 2)
    S, U, VT, info = _run(bdc, d, e, leaf=32, prec="bf16x3")
    s = S.cpu().numpy()
    res = oracle.residual(d, e, s, U.cpu().numpy(), VT.cpu().numpy())
    assert info == 0 and np.all(np.isfinite(s))
    assert 1e-9 < res < 1e-2


@pytest.mark.parametrize("kind,seed", [("uniform", 0), ("graded", 1), ("clustered", 2)])
def test_fp32_start_parity_and_fp64_iterations(bdc, kind, seed):
    """FP32 pre-iterations of the secular roots: the FP64 finish keeps the
    FP64 bar, and the FP64 root-finder steps drop on deflating inputs."""
    n = 4096
    d, e = inputs.make(kind, n, seed)
    its = {}
    for pre in (False, True):
        bdc.profile_begin()
        _check_full(bdc, d, e, fp32_start=pre)
        prof = bdc.profile_end()
        its[pre] = prof["secular"]["iters"] / max(prof["secular"]["roots"], 1)
    print(f"{kind}: FP64 steps per root without / with FP32 start {its[False]:.3f} / {its[True]:.3f}")
    if kind != "clustered":
        assert its[True] <= 0.7 * its[False], its


@pytest.mark.parametrize("entries", [0, 40, 1300])
@pytest.mark.parametrize("kind", ["uniform", "graded"])
def test_leaf_log_overflow_fallback(bdc, monkeypatch, entries, kind):
    """Leaves whose rotation log would overflow are iterated by the vectors
    kernel itself: with the log capacity lowered (all leaves overflow at 0
    and 40 entries, some at 1300) the SVD still meets the FP64 bar and agrees
    with the logged path."""
    d, e = inputs.make(kind, 700, 21)
    S0, _, _, _ = _run(bdc, d, e, leaf=16)
    monkeypatch.setenv("BDC_LEAF_LOG_ENTRIES", str(entries))
    _check_full(bdc, d, e, leaf=16)
    S1, _, _, _ = _run(bdc, d, e, leaf=16)
    assert float((S1 - S0).abs().max()) <= 1e-13 * 700 * float(S0[0])


@pytest.mark.parametrize("leaf", [4, 7, 33, 64])
def test_leaf_sizes_wide_range(bdc, leaf):
    """Leaf sizes across the allowed range (log capacity and lane layout scale with L)."""
    for kind, seed in (("uniform", 3), ("graded", 4)):
        d, e = inputs.make(kind, 1000, seed)
        _check_full(bdc, d, e, leaf=leaf)
