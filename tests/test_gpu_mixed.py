"""Split-BF16 tensor-core merge products (tcgen05) against FP64.

BDC_MIXED_EXACT with S slices represents each row of A and column of B to
2^-(8S-1) of its largest entry and accumulates the leading slice products
exactly, so |C - AB| <= c * 2^-(8S-1) * sum_k |A_rk| |B_kc| max-scaled;
the test bound is 2^-(8S-6) * (|A| |B|)_rc with |A|, |B| replaced by the row /
column maxima (a deliberately loose constant).  BDC_MIXED_BF16X3 is a 16-bit
split with FP32 accumulation: bound 2^-14 (|A| |B|).
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bdc():
    from paper_2508_11467_gb300 import bdc as b
    from paper_2508_11467_gb300 import build
    build.build()
    b.lib()
    return b


def _check(bdc, M, N, K, prec, slices, seed, scale_rows=False):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    if scale_rows:
        A *= np.exp(rng.uniform(-20, 20, (M, 1)))
        B *= np.exp(rng.uniform(-20, 20, (1, N)))
    C = bdc.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), prec, slices).cpu().numpy()
    ref = A @ B
    ra = np.max(np.abs(A), axis=1, keepdims=True)
    cb = np.max(np.abs(B), axis=0, keepdims=True)
    bound_scale = (ra * cb) * K
    if prec == "exact":
        tol = 2.0 ** (-(8 * slices - 6))
    else:
        tol = 2.0 ** -14
    err = np.max(np.abs(C - ref) / bound_scale)
    assert np.all(np.isfinite(C))
    assert err <= tol, (M, N, K, prec, slices, err, tol)
    return err


def test_mixed_single_tile(bdc):
    _check(bdc, 128, 128, 64, "exact", 6, 0)


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (100, 37, 5), (129, 130, 65), (300, 257, 190), (700, 300, 2000)])
def test_mixed_exact_shapes(bdc, M, N, K):
    _check(bdc, M, N, K, "exact", 6, M + N + K)


@pytest.mark.parametrize("slices", [4, 5, 7])
def test_mixed_exact_slices(bdc, slices):
    _check(bdc, 256, 200, 300, "exact", slices, slices)


def test_mixed_exact_wide_range(bdc):
    _check(bdc, 200, 150, 400, "exact", 6, 9, scale_rows=True)


def test_mixed_bf16x3(bdc):
    _check(bdc, 300, 200, 500, "bf16x3", 2, 3)


def test_mixed_long_k_accumulates_exactly(bdc):
    # K = 16384: 256 exact chunks; FP32 accumulation of the leading groups
    # over the whole K would lose ~2^-24 relative, far above the bound
    err = _check(bdc, 128, 128, 16384, "exact", 6, 11)
    assert err < 2.0 ** -40
