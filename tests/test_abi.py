"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/bdc.h (no compute calls)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bdc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bdc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2508_11467_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("bdc_svd", "bdc_svd_ex", "bdc_svd_batched", "bdc_secular_solve", "bdc_lowner_z",
                 "bdc_m_vectors", "bdc_deflate", "bdc_gemm", "bdc_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(bdc_[a-z0-9_]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_matches(libpath):
    from paper_2508_11467_gb300 import bdc
    L = bdc.lib()
    for name in _declared():
        assert hasattr(L, name)
    assert set(bdc.exported_symbols()) == set(_declared())
    # host-only calls: no GPU needed
    assert bdc.status_string(0) == "success"
    assert "NaN" in bdc.status_string(bdc.BDC_ERR_NONFINITE)
    o = bdc.make_opts("exact", leaf=16)
    assert o.prec == 2 and o.leaf == 16
    assert bdc.workspace_bytes(4096, o) > 4 * 4096 * 4096 * 8


def test_argument_errors_without_gpu(libpath):
    import ctypes
    from paper_2508_11467_gb300 import bdc
    L = bdc.lib()
    # argument checks run before any CUDA call
    assert L.bdc_svd(-1, None, None, None, None, None, 1, 1, None) == -1
    assert L.bdc_svd(4, None, None, None, None, None, 4, 4, None) == -2
    fake = ctypes.c_void_p(16)
    assert L.bdc_svd(4, fake, fake, fake, fake, fake, 3, 4, None) == -7
    assert L.bdc_svd(4, fake, fake, fake, fake, fake, 4, 2, None) == -8
    assert L.bdc_svd(0, None, None, None, None, None, 1, 1, None) == 0


def test_cuda_failure_returns_error_code_without_gpu(libpath):
    """With no CUDA device the first CUDA call fails: the entry point returns
    BDC_ERR_CUDA and records the message (no crash, no retry loop)."""
    import ctypes
    import torch
    if torch.cuda.is_available() or os.path.exists("/dev/nvidia0"):
        pytest.skip("needs a machine without a CUDA device")
    from paper_2508_11467_gb300 import bdc
    L = bdc.lib()
    fake = ctypes.c_void_p(16)       # never dereferenced: the workspace allocation fails first
    assert L.bdc_svd_values(4, fake, fake, fake, None) == bdc.BDC_ERR_CUDA
