"""bdc_deflate_noalloc: the allocation-free deflation entry point.

It exists for callers that cannot allocate device memory while they call
(another component owns the allocator, or all memory is reserved up front):
its scratch is a fixed array in the library's device memory instead of a
cudaMallocAsync allocation.  These tests call it through the C ABI and check
that it returns exactly what the allocating bdc_deflate returns, on two calls
in a row (the second call reuses the array the first one left behind), and
that sizes above its limit are refused.  The file sorts last so that a run
stopping at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import merge

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def bdc():
    from paper_2508_11467_gb300 import bdc as b
    from paper_2508_11467_gb300 import build
    build.build()
    b.lib()
    return b


def _case(m, seed):
    rng = np.random.default_rng(seed)
    d = np.concatenate(([0.0], np.sort(rng.uniform(0, 1, m - 1))))
    z = rng.uniform(-0.5, 0.5, m)
    z[rng.choice(np.arange(1, m), max(m // 8, 1), replace=False)] = 1e-19   # small z
    d[1:3] = [1e-18, 2e-18]                                               # close to d_0 = 0
    for j in range(5, m - 2, 29):                                          # close pairs / chains
        d[j + 1] = d[j] + 1e-17
    return np.maximum.accumulate(d), z


def test_noalloc_matches_allocating_entry_point_twice(bdc):
    for m, seed in [(4000, 1), (777, 2)]:          # two calls in a row, second one smaller
        d, z = _case(m, seed)
        tol = merge.deflation_tol(d, 0.5, 0.5)
        dc, zc = torch.from_numpy(d).cuda(), torch.from_numpy(z).cuda()
        k1, z1, v1 = bdc.deflate(dc, zc, tol)
        k2, z2, v2 = bdc.deflate_noalloc(dc, zc, tol)
        torch.cuda.synchronize()
        assert torch.equal(k1, k2)                  # survivor decisions: exact
        kept = k1.bool()
        assert torch.allclose(z1[kept], z2[kept], rtol=4 * EPS, atol=0)
        gone = ~kept
        assert torch.allclose(v1[gone], v2[gone], rtol=4 * EPS, atol=0)


def test_noalloc_at_its_size_limit(bdc):
    """m = BDC_DEFLATE_NOALLOC_MAX uses the whole fixed array."""
    m = bdc.NOALLOC_MAX
    d, z = _case(m, 3)
    tol = merge.deflation_tol(d, 0.5, 0.5)
    dc, zc = torch.from_numpy(d).cuda(), torch.from_numpy(z).cuda()
    k1, z1, v1 = bdc.deflate(dc, zc, tol)
    k2, z2, v2 = bdc.deflate_noalloc(dc, zc, tol)
    torch.cuda.synchronize()
    assert torch.equal(k1, k2)
    kept = k1.bool()
    assert torch.allclose(z1[kept], z2[kept], rtol=4 * EPS, atol=0)
    assert torch.allclose(v1[~kept], v2[~kept], rtol=4 * EPS, atol=0)


def test_noalloc_rejects_sizes_above_its_limit(bdc):
    L = bdc.lib()
    p = ctypes.c_void_p(256)          # never dereferenced: the size check comes first
    assert L.bdc_deflate_noalloc(bdc.NOALLOC_MAX + 1, p, p, 1e-15, p, p, p, None) == -1
    assert L.bdc_deflate_noalloc(-3, p, p, 1e-15, p, p, p, None) == -1
