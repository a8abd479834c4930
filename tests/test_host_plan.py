"""Host logic of the C ABI that runs without a GPU: the workspace sizing of
the entry points (the plan layout is built on the host) and its error
returns for shapes an entry point rejects.

* the full solve keeps n x n column slots for U and V and the merge
  operands: its workspace grows as n^2; the values-only solve keeps two rows
  of V per node: it grows as n;
* the split-BF16 products add slice buffers to the FP64 layout;
* a batch of one matrix is laid out like the single solve;
* shapes an entry point rejects give a workspace of 0.
"""
import ctypes

import pytest

from oracle import mlp as M


@pytest.fixture(scope="module")
def lib():
    from paper_2508_11467_gb300 import bdc as b
    from paper_2508_11467_gb300 import build
    build.build()
    L = b.lib()
    for name in ("bdc_svd_values_workspace", "bdc_svd_batched_workspace", "bdc_gebrd_workspace",
                 "bdc_geqrf_workspace", "bdc_gesvd_workspace", "bdc_gemm_workspace"):
        getattr(L, name).restype = ctypes.c_size_t
    return b, L


def test_full_workspace_grows_as_n_squared(lib):
    b, _ = lib
    o = b.make_opts("fp64", 0)
    w = {n: b.workspace_bytes(n, o) for n in (4096, 8192, 16384)}
    assert 3.9 <= w[8192] / w[4096] <= 4.1 and 3.9 <= w[16384] / w[8192] <= 4.1
    assert w[16384] >= 2 * 8 * 16384 ** 2          # the U and V column slots at least


def test_values_workspace_grows_as_n(lib):
    b, L = lib
    o = b.make_opts("fp64", 0)
    w = {n: L.bdc_svd_values_workspace(n, ctypes.byref(o)) for n in (4096, 8192, 16384)}
    assert 1.9 <= w[8192] / w[4096] <= 2.1 and 1.9 <= w[16384] / w[8192] <= 2.1
    assert w[16384] <= 1024 * 16384
    assert w[16384] * 100 < b.workspace_bytes(16384, o)


@pytest.mark.parametrize("n", [1, 16, 17, 1000, 4096])
def test_split_products_need_at_least_the_fp64_layout(lib, n):
    b, _ = lib
    assert b.workspace_bytes(n, b.make_opts("exact", 0)) >= b.workspace_bytes(n, b.make_opts("fp64", 0))


def test_batch_of_one_is_the_single_layout(lib):
    b, L = lib
    o = b.make_opts("fp64", 0)
    for n in (1, 33, 1000, 2048):
        arr = (ctypes.c_int * 1)(n)
        assert L.bdc_svd_batched_workspace(1, arr, ctypes.byref(o)) == b.workspace_bytes(n, o)


def test_rejected_shapes_give_no_workspace(lib):
    b, L = lib
    o = b.make_opts("fp64", 0)
    assert b.workspace_bytes(-1, o) == 0
    assert L.bdc_svd_batched_workspace(2, (ctypes.c_int * 2)(1000, 3000), ctypes.byref(o)) == 0   # n > 2048
    assert L.bdc_svd_batched_workspace(2, (ctypes.c_int * 2)(1000, 0), ctypes.byref(o)) == 0
    assert L.bdc_svd_batched_workspace(0, None, ctypes.byref(o)) == 0
    assert L.bdc_gebrd_workspace(100, 200) == 0                                                  # m < n
    assert L.bdc_gesvd_workspace(100, 200, ctypes.byref(o)) == 0
    assert L.bdc_gemm_workspace(-1, 1, 1, 0, 0) == 0
    assert L.bdc_gebrd_workspace(4096, 4096) > 0 and L.bdc_geqrf_workspace(100, 200) > 0


def test_gemm_workspace_split_over_fp64(lib):
    _, L = lib
    assert L.bdc_gemm_workspace(1024, 1024, 1024, 0, 0) < L.bdc_gemm_workspace(1024, 1024, 1024, 2, 0)


def test_mlp_layout_matches_the_oracle(lib):
    b, _ = lib
    assert b.mlp_param_count() == M.N_PARAMS
    assert b.mlp_feature_count() == M.N_IN
