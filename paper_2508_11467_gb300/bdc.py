"""Thin ctypes binding of libbdc.so (include/bdc.h).

Argument marshalling only: tensors are passed as raw device pointers, the
current PyTorch stream as the CUDA stream.  Every step of the SVD runs in the
library's CUDA kernels; there is no CPU path.  The library is loaded on first
use and a missing build raises immediately.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

LIB_PATH = _build.LIB

BDC_FP64, BDC_MIXED_BF16X3, BDC_MIXED_EXACT = 0, 1, 2
BDC_SEED_PLAIN, BDC_SEED_MLP, BDC_SEED_ANALYTIC = 0, 1, 2
SEED = {"plain": BDC_SEED_PLAIN, "mlp": BDC_SEED_MLP, "analytic": BDC_SEED_ANALYTIC}
BDC_ERR_CUDA, BDC_ERR_TIMEOUT, BDC_ERR_NONFINITE, BDC_ERR_INTERNAL, BDC_ERR_CHECK = -1000, -1001, -1002, -1003, -1004
PREC = {"fp64": BDC_FP64, "bf16x3": BDC_MIXED_BF16X3, "exact": BDC_MIXED_EXACT, "mixed": BDC_MIXED_EXACT}


class Opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("seed", ctypes.c_int), ("leaf", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("slices", ctypes.c_int), ("checked", ctypes.c_int),
                ("mlp", ctypes.c_void_p), ("mixed_min", ctypes.c_int), ("fp32_start", ctypes.c_int),
                ("vectors", ctypes.c_int)]


_lock = threading.Lock()
_lib = None

_VP, _I, _SZ, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_double
_SIGS = {
    "bdc_opts_default": (None, [_VP]),
    "bdc_svd": (_I, [_I, _VP, _VP, _VP, _VP, _VP, _I, _I, _VP]),
    "bdc_svd_workspace": (_SZ, [_I, _VP]),
    "bdc_svd_ex": (_I, [_I, _VP, _VP, _VP, _VP, _VP, _I, _I, _VP, _VP, _SZ, _VP, _VP]),
    "bdc_svd_batched_workspace": (_SZ, [_I, _VP, _VP]),
    "bdc_svd_values_workspace": (_SZ, [_I, _VP]),
    "bdc_svd_values_ex": (_I, [_I, _VP, _VP, _VP, _VP, _VP, _SZ, _VP, _VP]),
    "bdc_svd_values": (_I, [_I, _VP, _VP, _VP, _VP]),
    "bdc_svd_batched": (_I, [_I, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP, _VP]),
    "bdc_secular_solve": (_I, [_I, _VP, _VP, _VP, _VP, _VP, _I, _VP, _VP]),
    "bdc_lowner_z": (_I, [_I, _VP, _VP, _VP, _VP, _VP, _VP]),
    "bdc_m_vectors": (_I, [_I, _VP, _VP, _VP, _VP, _VP, _I, _VP, _I, _VP]),
    "bdc_deflate": (_I, [_I, _VP, _VP, _D, _VP, _VP, _VP, _VP]),
    "bdc_deflate_noalloc": (_I, [_I, _VP, _VP, _D, _VP, _VP, _VP, _VP]),
    "bdc_gemm_workspace": (_SZ, [_I, _I, _I, _I, _I]),
    "bdc_gemm": (_I, [_I, _I, _I, _VP, _I, _VP, _I, _VP, _I, _I, _I, _VP, _SZ, _VP]),
    "bdc_mlp_param_count": (_I, []),
    "bdc_mlp_feature_count": (_I, []),
    "bdc_mlp_features": (_I, [_I, _VP, _VP, _VP, _VP, _VP]),
    "bdc_secular_solve_ex": (_I, [_I, _VP, _VP, _I, _VP, _VP, _VP, _VP, _VP, _I, _VP, _VP]),
    "bdc_svd_harvest": (_I, [_I, _VP, _VP, _VP, _VP, _VP, _I, _I, _VP, _VP, _SZ, _VP, _VP, _VP, _I, _VP,
                             _VP]),
    "bdc_mlp_init": (_I, [_VP, _VP, _VP, _I, ctypes.c_ulonglong, _VP]),
    "bdc_mlp_grad_workspace": (_SZ, [_I]),
    "bdc_mlp_grad": (_I, [_VP, _VP, _VP, _I, ctypes.c_float, _VP, _VP, _VP, _SZ, _VP]),
    "bdc_mlp_adam": (_I, [_VP, _VP, _VP, _VP, _I, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                          ctypes.c_float, _VP]),
    "bdc_mlp_predict": (_I, [_VP, _VP, _I, _VP, _VP]),
    "bdc_mlp_fit": (_I, [_VP, _VP, _VP, _I, _I, ctypes.c_float, ctypes.c_float, ctypes.c_ulonglong, _VP, _VP]),
    "bdc_mlp_train": (_I, [_VP, _VP, _VP, _VP, _VP, ctypes.c_char_p, _VP]),
    "bdc_plan_create": (_I, [_VP, _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "bdc_plan_launch": (_I, [_VP, _VP]),
    "bdc_plan_destroy": (None, [_VP]),
    "bdc_autotune": (_I, [_I, _VP, _VP, _I, _VP, _VP]),
    "bdc_svd_batched_workspace_f32": (_SZ, [_I, _VP, _VP]),
    "bdc_autotune_f32": (_I, [_I, _VP, _VP, _I, _VP, _VP]),
    "bdc_svd_batched_f32": (_I, [_I, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP, _VP]),
    "bdc_plan_create_f32": (_I, [_VP, _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "bdc_status_string": (ctypes.c_char_p, [_I]),
    "bdc_gebrd_workspace": (_SZ, [_I, _I]),
    "bdc_gebrd": (_I, [_I, _I, _VP, _I, _VP, _VP, _VP, _VP, _VP, _SZ, _VP, _VP]),
    "bdc_ormbr_workspace": (_SZ, [_I, _I, _I]),
    "bdc_ormbr": (_I, [_I, _I, _I, _VP, _I, _VP, _VP, _I, _I, _VP, _SZ, _VP]),
    "bdc_geqrf_workspace": (_SZ, [_I, _I]),
    "bdc_geqrf": (_I, [_I, _I, _VP, _I, _VP, _VP, _SZ, _VP, _VP]),
    "bdc_orgqr": (_I, [_I, _I, _VP, _I, _VP, _VP, _SZ, _VP]),
    "bdc_gesvd_workspace": (_SZ, [_I, _I, _VP]),
    "bdc_gesvd": (_I, [_I, _I, _VP, _I, _VP, _VP, _I, _VP, _I, _VP, _VP, _SZ, _VP, _VP]),
    "bdc_profile_begin": (_I, [_I]),
    "bdc_profile_end": (_I, [_VP, _VP, _VP]),
    "bdc_profile_secular": (_I, [_VP, _VP]),
    "bdc_profile_fp64": (_I, [_VP]),
    "bdc_profile_levels": (_I, [_I, _I, _VP, _VP]),
    "bdc_last_error_string": (ctypes.c_char_p, []),
}

STAGES = ["scale", "leaf", "prep", "gather", "secular", "vectors", "gemm", "finish", "final", "slice", "lowner"]


def profile_begin():
    _check("bdc_profile_begin", lib().bdc_profile_begin(1))


def profile_end():
    """Per-stage device ms, launch counts, algorithmic work (tensor flops for
    "gemm", HBM bytes for the others) and FP64 operations since
    profile_begin()."""
    import numpy as np
    k = len(STAGES)
    ms = np.zeros(k)
    ln = np.zeros(k, dtype=np.int64)
    wk = np.zeros(k)
    f64 = np.zeros(k)
    _check("bdc_profile_end", lib().bdc_profile_end(ms.ctypes.data_as(ctypes.c_void_p),
                                                     ln.ctypes.data_as(ctypes.c_void_p),
                                                     wk.ctypes.data_as(ctypes.c_void_p)))
    lib().bdc_profile_fp64(f64.ctypes.data_as(ctypes.c_void_p))
    out = {s: {"ms": float(ms[i]), "launches": int(ln[i]), "work": float(wk[i]), "fp64": float(f64[i])}
           for i, s in enumerate(STAGES)}
    for i, st_name in enumerate(STAGES):
        lm = np.zeros(32)
        lw = np.zeros(32)
        lib().bdc_profile_levels(i, 32, lm.ctypes.data_as(ctypes.c_void_p), lw.ctypes.data_as(ctypes.c_void_p))
        nz = int(np.max(np.nonzero(lm)[0]) + 1) if np.any(lm) else 0
        if nz:
            out[st_name]["level_ms"] = [float(x) for x in lm[:nz]]
            out[st_name]["level_work"] = [float(x) for x in lw[:nz]]
    r, it = ctypes.c_longlong(0), ctypes.c_longlong(0)
    lib().bdc_profile_secular(ctypes.byref(r), ctypes.byref(it))
    out["secular"]["roots"] = int(r.value)
    out["secular"]["iters"] = int(it.value)
    return out


def exported_symbols():
    """Names the binding expects the library to export."""
    return sorted(_SIGS)


def lib():
    """Load libbdc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "paper_2508_11467_gb300.build.build() (nvcc, sm_103a)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().bdc_status_string(int(code)).decode()


class BDCError(RuntimeError):
    def __init__(self, where: str, code: int):
        detail = lib().bdc_last_error_string().decode() if code == BDC_ERR_CUDA else ""
        super().__init__(f"{where}: {code} ({status_string(code)}{': ' + detail if detail else ''})")
        self.code = code


def _check(where, code):
    if code != 0:
        raise BDCError(where, code)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype=torch.float64):
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(t)
    if t.device.type != "cuda":
        raise ValueError("bdc expects CUDA tensors (device memory)")
    return t.to(dtype).contiguous()


VECTORS = {"both": 0, "v": 1, "u": 2}


def make_opts(prec="fp64", leaf=0, max_iter=64, slices=0, seed="plain", mlp=None, mixed_min=0,
              fp32_start=True, vectors="both", checked=False) -> Opts:
    o = Opts()
    lib().bdc_opts_default(ctypes.byref(o))
    o.checked = 1 if checked else 0
    o.fp32_start = 1 if fp32_start else 0
    o.vectors = VECTORS[vectors] if isinstance(vectors, str) else int(vectors)
    o.mixed_min = int(mixed_min)
    o.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    o.leaf = int(leaf)
    o.max_iter = int(max_iter)
    o.slices = int(slices)
    o.seed = SEED[seed] if isinstance(seed, str) else int(seed)
    o.mlp = ctypes.c_void_p(mlp.data_ptr()) if mlp is not None else None
    return o


def workspace_bytes(n: int, opts: Opts) -> int:
    return int(lib().bdc_svd_workspace(int(n), ctypes.byref(opts)))


def svd(d, e, *, prec="fp64", leaf=0, max_iter=64, slices=0, seed="plain", mlp=None,
        stream=None, work=None, check=True, mixed_min=0, fp32_start=True, vectors="both", checked=False):
    """SVD of the upper bidiagonal (d, e) on the GPU.

    Returns (S, U, VT) as CUDA float64 tensors (U column-major: U[:, i] is a
    left vector; VT[i, :] a right vector) and the status code.  vectors="v"
    forms V^T only (U is None), vectors="u" U only (VT is None).
    """
    d = _dev(d)
    n = d.shape[0]
    e = _dev(e) if n > 1 else torch.zeros(1, dtype=torch.float64, device=d.device)
    o = make_opts(prec, leaf, max_iter, slices, seed, mlp, mixed_min, fp32_start, vectors, checked)
    # column-major outputs: allocate the transpose and view it back
    Ut = torch.empty((n, n), dtype=torch.float64, device=d.device) if vectors != "v" else None
    VTt = torch.empty((n, n), dtype=torch.float64, device=d.device) if vectors != "u" else None
    S = torch.empty(max(n, 1), dtype=torch.float64, device=d.device)
    info = torch.zeros(1, dtype=torch.int32, device=d.device)
    lw = workspace_bytes(n, o)
    if work is None or work.numel() < lw + 256:
        work = torch.empty(lw + 256, dtype=torch.uint8, device=d.device)
    rc = lib().bdc_svd_ex(n, _ptr(d), _ptr(e), _ptr(Ut), _ptr(S), _ptr(VTt), max(n, 1), max(n, 1),
                          ctypes.byref(o), _ptr(work), work.numel(), _ptr(info), _stream(stream))
    _check("bdc_svd_ex", rc)
    code = int(info.item())
    if check and code != 0:
        raise BDCError("bdc_svd_ex (device status)", code)
    return S[:n], (Ut.t() if Ut is not None else None), (VTt.t() if VTt is not None else None), code


def svd_values(d, e, *, leaf=0, max_iter=64, seed="plain", mlp=None, stream=None, check=True, fp32_start=True):
    """Singular values only (descending), CUDA float64; and the status code."""
    d = _dev(d)
    n = d.shape[0]
    e = _dev(e) if n > 1 else torch.zeros(1, dtype=torch.float64, device=d.device)
    o = make_opts("fp64", leaf, max_iter, 0, seed, mlp, 0, fp32_start)
    S = torch.empty(max(n, 1), dtype=torch.float64, device=d.device)
    info = torch.zeros(1, dtype=torch.int32, device=d.device)
    lw = int(lib().bdc_svd_values_workspace(n, ctypes.byref(o)))
    work = torch.empty(lw + 256, dtype=torch.uint8, device=d.device)
    _check("bdc_svd_values_ex", lib().bdc_svd_values_ex(n, _ptr(d), _ptr(e), _ptr(S), ctypes.byref(o), _ptr(work),
                                                         work.numel(), _ptr(info), _stream(stream)))
    code = int(info.item())
    if check and code != 0:
        raise BDCError("bdc_svd_values_ex (device status)", code)
    return S[:n], code


def svd_sync(d, e, stream=None):
    """bdc_svd: defaults, library-managed workspace, synchronous status."""
    d = _dev(d)
    n = d.shape[0]
    e = _dev(e) if n > 1 else torch.zeros(1, dtype=torch.float64, device=d.device)
    Ut = torch.empty((n, n), dtype=torch.float64, device=d.device)
    VTt = torch.empty((n, n), dtype=torch.float64, device=d.device)
    S = torch.empty(max(n, 1), dtype=torch.float64, device=d.device)
    rc = lib().bdc_svd(n, _ptr(d), _ptr(e), _ptr(Ut), _ptr(S), _ptr(VTt), max(n, 1), max(n, 1),
                       _stream(stream))
    return S[:n], Ut.t(), VTt.t(), rc


def svd_batched(ds, es, *, prec="fp64", leaf=0, max_iter=64, slices=0, stream=None, work=None):
    """Batched SVD of bidiagonals of uneven sizes (lists of CUDA tensors)."""
    import numpy as np
    B = len(ds)
    ns = np.array([int(x.shape[0]) for x in ds], dtype=np.int32)
    o = make_opts(prec, leaf, max_iter, slices)
    dev = ds[0].device
    ds = [_dev(x) for x in ds]
    es = [_dev(x) if x.numel() > 0 else torch.zeros(1, dtype=torch.float64, device=dev) for x in es]
    Us = [torch.empty((n, n), dtype=torch.float64, device=dev) for n in ns]
    Ss = [torch.empty(int(n), dtype=torch.float64, device=dev) for n in ns]
    VTs = [torch.empty((n, n), dtype=torch.float64, device=dev) for n in ns]
    arr = lambda ts: (ctypes.c_void_p * B)(*[t.data_ptr() for t in ts])
    lw = int(lib().bdc_svd_batched_workspace(B, ns.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o)))
    if work is None or work.numel() < lw + 256:
        work = torch.empty(lw + 256, dtype=torch.uint8, device=dev)
    info = torch.zeros(B, dtype=torch.int32, device=dev)
    lds = ns.copy()
    rc = lib().bdc_svd_batched(B, ns.ctypes.data_as(ctypes.c_void_p), arr(ds), arr(es), arr(Us), arr(Ss),
                               arr(VTs), lds.ctypes.data_as(ctypes.c_void_p), lds.ctypes.data_as(ctypes.c_void_p),
                               ctypes.byref(o), _ptr(work), work.numel(), _ptr(info), _stream(stream))
    _check("bdc_svd_batched", rc)
    return Ss, [u.t() for u in Us], [v.t() for v in VTs], info


def secular_solve(d, z, max_iter=64, stream=None):
    d, z = _dev(d), _dev(z)
    N = d.shape[0]
    org = torch.empty(N, dtype=torch.int32, device=d.device)
    tau = torch.empty(N, dtype=torch.float64, device=d.device)
    om = torch.empty(N, dtype=torch.float64, device=d.device)
    info = torch.zeros(1, dtype=torch.int32, device=d.device)
    _check("bdc_secular_solve", lib().bdc_secular_solve(N, _ptr(d), _ptr(z), _ptr(org), _ptr(tau), _ptr(om),
                                                         int(max_iter), _ptr(info), _stream(stream)))
    return org, tau, om, info


def lowner_z(d, z, org, tau, stream=None):
    d, z, tau = _dev(d), _dev(z), _dev(tau)
    org = _dev(org, torch.int32)
    zt = torch.empty_like(d)
    _check("bdc_lowner_z", lib().bdc_lowner_z(d.shape[0], _ptr(d), _ptr(z), _ptr(org), _ptr(tau), _ptr(zt),
                                               _stream(stream)))
    return zt


def m_vectors(d, zt, org, tau, stream=None):
    d, zt, tau = _dev(d), _dev(zt), _dev(tau)
    org = _dev(org, torch.int32)
    N = d.shape[0]
    UMt = torch.empty((N, N), dtype=torch.float64, device=d.device)
    VMt = torch.empty((N, N), dtype=torch.float64, device=d.device)
    _check("bdc_m_vectors", lib().bdc_m_vectors(N, _ptr(d), _ptr(zt), _ptr(org), _ptr(tau), _ptr(UMt), N,
                                                 _ptr(VMt), N, _stream(stream)))
    return UMt.t(), VMt.t()


def deflate(d, z, tol, stream=None):
    d, z = _dev(d), _dev(z)
    m = d.shape[0]
    keep = torch.empty(m, dtype=torch.int32, device=d.device)
    zout = torch.empty(m, dtype=torch.float64, device=d.device)
    dval = torch.empty(m, dtype=torch.float64, device=d.device)
    _check("bdc_deflate", lib().bdc_deflate(m, _ptr(d), _ptr(z), float(tol), _ptr(keep), _ptr(zout), _ptr(dval),
                                             _stream(stream)))
    return keep, zout, dval


NOALLOC_MAX = 65536


def deflate_noalloc(d, z, tol, stream=None):
    """bdc_deflate_noalloc: deflation with the library's fixed device scratch.

    For callers that cannot allocate device memory during the call; m is at
    most NOALLOC_MAX and calls that overlap on the GPU must be ordered.
    """
    d, z = _dev(d), _dev(z)
    m = d.shape[0]
    keep = torch.empty(m, dtype=torch.int32, device=d.device)
    zout = torch.empty(m, dtype=torch.float64, device=d.device)
    dval = torch.empty(m, dtype=torch.float64, device=d.device)
    _check("bdc_deflate_noalloc", lib().bdc_deflate_noalloc(m, _ptr(d), _ptr(z), float(tol), _ptr(keep), _ptr(zout),
                                                             _ptr(dval), _stream(stream)))
    return keep, zout, dval


def gemm(A, B, prec="fp64", slices=6, stream=None, work=None):
    """C = A @ B for column-major views (A: M x K, B: K x N) through bdc_gemm."""
    A = _dev(A).t().contiguous().t()   # column-major storage
    B = _dev(B).t().contiguous().t()
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    Ct = torch.empty((N, M), dtype=torch.float64, device=A.device)
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    lw = int(lib().bdc_gemm_workspace(M, N, K, p, slices))
    if work is None or work.numel() < lw + 256:
        work = torch.empty(lw + 256, dtype=torch.uint8, device=A.device)
    _check("bdc_gemm", lib().bdc_gemm(M, N, K, _ptr(A), max(M, 1), _ptr(B), max(K, 1), _ptr(Ct), max(M, 1), p,
                                       int(slices), _ptr(work), work.numel(), _stream(stream)))
    return Ct.t()


# ---------------------------------------------------------------- MLP start points
def mlp_param_count() -> int:
    return int(lib().bdc_mlp_param_count())


def mlp_feature_count() -> int:
    return int(lib().bdc_mlp_feature_count())


def mlp_features(d, z, stream=None):
    """Features ((N-1) x 11 float32) and analytic estimates y_q ((N-1)
    float64) of roots 0..N-2 of one sorted secular problem."""
    d, z = _dev(d), _dev(z)
    N = d.shape[0]
    f = torch.empty((max(N - 1, 0), mlp_feature_count()), dtype=torch.float32, device=d.device)
    yq = torch.empty(max(N - 1, 0), dtype=torch.float64, device=d.device)
    _check("bdc_mlp_features", lib().bdc_mlp_features(N, _ptr(d), _ptr(z), _ptr(f), _ptr(yq), _stream(stream)))
    return f, yq


def secular_solve_ex(d, z, seed="plain", mlp=None, max_iter=64, stream=None):
    """Secular roots with a chosen start rule; also the iterations per root."""
    d, z = _dev(d), _dev(z)
    N = d.shape[0]
    org = torch.empty(N, dtype=torch.int32, device=d.device)
    tau = torch.empty(N, dtype=torch.float64, device=d.device)
    om = torch.empty(N, dtype=torch.float64, device=d.device)
    it = torch.empty(N, dtype=torch.int32, device=d.device)
    info = torch.zeros(1, dtype=torch.int32, device=d.device)
    _check("bdc_secular_solve_ex",
           lib().bdc_secular_solve_ex(N, _ptr(d), _ptr(z), SEED[seed] if isinstance(seed, str) else int(seed),
                                      _ptr(mlp), _ptr(org), _ptr(tau), _ptr(om), _ptr(it), int(max_iter),
                                      _ptr(info), _stream(stream)))
    return org, tau, om, it, info


class Harvest:
    """Device buffers that collect (features, target) pairs from SVD runs."""

    def __init__(self, cap: int, device="cuda"):
        self.cap = int(cap)
        self.feat = torch.empty((self.cap, mlp_feature_count()), dtype=torch.float32, device=device)
        self.targ = torch.empty(self.cap, dtype=torch.float32, device=device)
        self.count = torch.zeros(1, dtype=torch.int32, device=device)

    def size(self) -> int:
        return min(int(self.count.item()), self.cap)

    def data(self):
        k = self.size()
        return self.feat[:k], self.targ[:k]


def svd_harvest(d, e, harvest: Harvest, *, prec="fp64", leaf=0, max_iter=64, slices=0, stream=None,
                check=True, mixed_min=0):
    """svd() that appends every merge root's (features, target) to `harvest`."""
    d = _dev(d)
    n = d.shape[0]
    e = _dev(e) if n > 1 else torch.zeros(1, dtype=torch.float64, device=d.device)
    o = make_opts(prec, leaf, max_iter, slices, "plain", None, mixed_min)
    Ut = torch.empty((n, n), dtype=torch.float64, device=d.device)
    VTt = torch.empty((n, n), dtype=torch.float64, device=d.device)
    S = torch.empty(max(n, 1), dtype=torch.float64, device=d.device)
    info = torch.zeros(1, dtype=torch.int32, device=d.device)
    lw = workspace_bytes(n, o)
    work = torch.empty(lw + 256, dtype=torch.uint8, device=d.device)
    rc = lib().bdc_svd_harvest(n, _ptr(d), _ptr(e), _ptr(Ut), _ptr(S), _ptr(VTt), max(n, 1), max(n, 1),
                               ctypes.byref(o), _ptr(work), work.numel(), _ptr(info), _ptr(harvest.feat),
                               _ptr(harvest.targ), harvest.cap, _ptr(harvest.count), _stream(stream))
    _check("bdc_svd_harvest", rc)
    code = int(info.item())
    if check and code != 0:
        raise BDCError("bdc_svd_harvest (device status)", code)
    return S[:n], Ut.t(), VTt.t(), code


def mlp_init(feat, targ=None, seed=0, stream=None):
    """Fresh parameters (normalisation from the data, Glorot hidden weights,
    zero output layer)."""
    P = torch.empty(mlp_param_count(), dtype=torch.float32, device=feat.device)
    _check("bdc_mlp_init", lib().bdc_mlp_init(_ptr(P), _ptr(feat), _ptr(targ), int(feat.shape[0]),
                                               int(seed), _stream(stream)))
    return P


def mlp_grad(P, feat, targ, huber=0.25, stream=None, work=None):
    """(gradient, loss) of the mean Huber loss (threshold `huber`; <= 0:
    squares), both on the device."""
    count = int(feat.shape[0])
    g = torch.empty_like(P)
    loss = torch.empty(1, dtype=torch.float32, device=P.device)
    lw = int(lib().bdc_mlp_grad_workspace(count))
    if work is None or work.numel() < lw:
        work = torch.empty(max(lw, 1), dtype=torch.uint8, device=P.device)
    _check("bdc_mlp_grad", lib().bdc_mlp_grad(_ptr(P), _ptr(feat), _ptr(targ), count, float(huber), _ptr(g),
                                               _ptr(loss), _ptr(work), work.numel(), _stream(stream)))
    return g, loss


def mlp_adam(P, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check("bdc_mlp_adam", lib().bdc_mlp_adam(_ptr(P), _ptr(g), _ptr(m), _ptr(v), int(step), float(lr),
                                               float(beta1), float(beta2), float(eps), _stream(stream)))


def mlp_predict(P, feat, stream=None):
    out = torch.empty(int(feat.shape[0]), dtype=torch.float32, device=P.device)
    _check("bdc_mlp_predict", lib().bdc_mlp_predict(_ptr(P), _ptr(feat), int(feat.shape[0]), _ptr(out),
                                                     _stream(stream)))
    return out


def mlp_train(feat, targ, steps=1500, lr=3e-3, seed=0, huber=0.25, stream=None):
    """bdc_mlp_fit: initialisation and full-batch Adam on the harvested pairs
    (Huber loss, threshold `huber`; learning rate decaying linearly to
    lr/10).  Returns (params, losses), both on the device."""
    P = torch.empty(mlp_param_count(), dtype=torch.float32, device=feat.device)
    losses = torch.empty(max(int(steps), 1), dtype=torch.float32, device=feat.device)
    _check("bdc_mlp_fit", lib().bdc_mlp_fit(_ptr(P), _ptr(feat), _ptr(targ), int(feat.shape[0]), int(steps),
                                             float(lr), float(huber), int(seed), _ptr(losses), _stream(stream)))
    return P, losses[:int(steps)]


class MlpTrainOpts(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("steps", ctypes.c_int), ("lr", ctypes.c_float), ("huber", ctypes.c_float),
                ("seed", ctypes.c_ulonglong)]


def mlp_train_harvest(n=8192, steps=1500, lr=3e-3, huber=0.25, seed=0, leaf=0, out_path=None, device="cuda",
                      stream=None):
    """bdc_mlp_train: harvest roots from FP64 solves of an n x n uniform and
    an n x n graded bidiagonal generated on the device, then fit the network.
    Returns (params, losses, samples)."""
    P = torch.empty(mlp_param_count(), dtype=torch.float32, device=device)
    losses = torch.empty(max(int(steps), 1), dtype=torch.float32, device=device)
    t = MlpTrainOpts(int(n), int(steps), float(lr), float(huber), int(seed))
    o = make_opts("fp64", leaf)
    cnt = ctypes.c_int(0)
    _check("bdc_mlp_train", lib().bdc_mlp_train(ctypes.byref(o), ctypes.byref(t), _ptr(P), _ptr(losses),
                                                 ctypes.byref(cnt), out_path.encode() if out_path else None,
                                                 _stream(stream)))
    return P, losses[:int(steps)], int(cnt.value)


def mlp_save(P, path):
    """Write the parameters as raw little-endian float32."""
    import numpy as np
    np.asarray(P.detach().cpu().numpy(), dtype="<f4").tofile(path)


def mlp_load(path, device="cuda"):
    import numpy as np
    a = np.fromfile(path, dtype="<f4")
    if a.size != mlp_param_count():
        raise ValueError(f"{path}: {a.size} floats, expected {mlp_param_count()}")
    return torch.from_numpy(a).to(device)


# ---------------------------------------------------------------- batched plans
class BatchPlan:
    """A fixed batch of bidiagonals solved by one CUDA-graph launch.

    d_flat, e_flat: CUDA float64 tensors holding the matrices back to back
    (matrix b at offset sum(ns[:b]); e has n-1 entries there).  Outputs live in
    flat buffers: S at the same offsets, U and V^T (column-major, n x n) at
    offsets sum(ns[:b]**2).  Built by bdc_plan_create; launch() enqueues the
    whole solve on the stream."""

    def __init__(self, d_flat, e_flat, ns, *, prec="fp64", leaf=0, max_iter=64, slices=0, seed="plain",
                 mlp=None, mixed_min=0, dtype=torch.float64):
        import numpy as np
        self.ns = np.asarray(ns, dtype=np.int32)
        B = len(self.ns)
        dev = d_flat.device
        self.dtype = dtype
        f32 = dtype == torch.float32
        esz = 4 if f32 else 8
        self.d, self.e = _dev(d_flat, dtype), _dev(e_flat, dtype)
        self.off = np.concatenate([[0], np.cumsum(self.ns, dtype=np.int64)])
        self.off2 = np.concatenate([[0], np.cumsum(self.ns.astype(np.int64) ** 2)])
        self.S = torch.empty(int(self.off[-1]), dtype=dtype, device=dev)
        self.U = torch.empty(int(self.off2[-1]), dtype=dtype, device=dev)
        self.VT = torch.empty(int(self.off2[-1]), dtype=dtype, device=dev)
        self.info = torch.zeros(B, dtype=torch.int32, device=dev)
        self.opts = make_opts(prec, leaf, max_iter, slices, seed, mlp, mixed_min)
        self._mlp = mlp
        wsfn = lib().bdc_svd_batched_workspace_f32 if f32 else lib().bdc_svd_batched_workspace
        lw = int(wsfn(B, self.ns.ctypes.data_as(ctypes.c_void_p), ctypes.byref(self.opts)))
        if lw == 0:
            raise BDCError("bdc_svd_batched_workspace", -2)
        self.work = torch.empty(lw + 256, dtype=torch.uint8, device=dev)
        ptrs = lambda base, offs: (ctypes.c_void_p * B)(*[base.data_ptr() + int(o) * esz for o in offs[:B]])
        self._pd = ptrs(self.d, self.off)
        self._pe = ptrs(self.e, self.off)
        self._pu = ptrs(self.U, self.off2)
        self._ps = ptrs(self.S, self.off)
        self._pv = ptrs(self.VT, self.off2)
        self._ld = self.ns.copy()
        self._plan = ctypes.c_void_p()
        create = lib().bdc_plan_create_f32 if f32 else lib().bdc_plan_create
        _check("bdc_plan_create", create(
            ctypes.byref(self._plan), B, self.ns.ctypes.data_as(ctypes.c_void_p), self._pd, self._pe, self._pu,
            self._ps, self._pv, self._ld.ctypes.data_as(ctypes.c_void_p), self._ld.ctypes.data_as(ctypes.c_void_p),
            ctypes.byref(self.opts), _ptr(self.work), self.work.numel(), _ptr(self.info)))

    def launch(self, stream=None):
        _check("bdc_plan_launch", lib().bdc_plan_launch(self._plan, _stream(stream)))

    def result(self, b):
        """(S, U, VT) of matrix b as CUDA views (U[:, i] left vectors)."""
        n = int(self.ns[b])
        o, o2 = int(self.off[b]), int(self.off2[b])
        U = self.U[o2:o2 + n * n].view(n, n).t()
        VT = self.VT[o2:o2 + n * n].view(n, n).t()
        return self.S[o:o + n], U, VT

    def close(self):
        if getattr(self, "_plan", None) is not None and self._plan.value:
            lib().bdc_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(ns, prec="fp64", seed="plain", slices=0, reps=3, stream=None, dtype=torch.float64):
    """bdc_autotune (bdc_autotune_f32 for dtype=torch.float32): (leaf,
    mixed_min, ms per batch) for a batch of orders ns."""
    import numpy as np
    ns = np.asarray(ns, dtype=np.int32)
    o = make_opts(prec, 16, 64, slices, seed)
    ms = ctypes.c_double(0.0)
    fn = lib().bdc_autotune_f32 if dtype == torch.float32 else lib().bdc_autotune
    _check("bdc_autotune", fn(len(ns), ns.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o),
                              int(reps), ctypes.byref(ms), _stream(stream)))
    return int(o.leaf), int(o.mixed_min), float(ms.value)


# ---------------------------------------------------------------- dense front and back end
def _colmajor(A):
    """A (rows x cols) as a CUDA float64 column-major copy (returned as the
    transpose-view of a contiguous tensor)."""
    A = _dev(A)
    return A.t().contiguous().t()


def gebrd(A, stream=None):
    """bdc_gebrd: (Ar, d, e, tauq, taup, info); Ar is A overwritten by the
    reflectors (column-major view), B = diag(d) + superdiag(e)."""
    A = _colmajor(A)
    m, n = A.shape
    dev = A.device
    d = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
    e = torch.empty(max(n - 1, 1), dtype=torch.float64, device=dev)
    tq = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
    tp = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    lw = int(lib().bdc_gebrd_workspace(m, n))
    work = torch.empty(max(lw, 1), dtype=torch.uint8, device=dev)
    _check("bdc_gebrd", lib().bdc_gebrd(m, n, _ptr(A), max(m, 1), _ptr(d), _ptr(e), _ptr(tq), _ptr(tp), _ptr(work),
                                         work.numel(), _ptr(info), _stream(stream)))
    return A, d[:n], e[:max(n - 1, 0)], tq[:n], tp[:n], int(info.item())


def ormbr(vect, Ar, tau, C, stream=None):
    """bdc_ormbr: vect 0: Q1 C (C m x k); vect 1: C P1^T (C k x n).  C is
    updated in place (it must be a column-major CUDA float64 tensor)."""
    m, n = Ar.shape
    rows, cols = C.shape
    assert C.stride(0) == 1, "C must be column-major"
    cdim = cols if vect == 0 else rows
    lw = int(lib().bdc_ormbr_workspace(m, n, cdim))
    work = torch.empty(max(lw, 1), dtype=torch.uint8, device=Ar.device)
    _check("bdc_ormbr", lib().bdc_ormbr(int(vect), m, n, _ptr(Ar), max(Ar.stride(1), 1), _ptr(tau), _ptr(C),
                                         max(C.stride(1), 1), cdim, _ptr(work), work.numel(), _stream(stream)))
    return C


def geqrf(A, stream=None):
    """bdc_geqrf: (Ar, tau, info)."""
    A = _colmajor(A)
    m, n = A.shape
    tau = torch.empty(max(min(m, n), 1), dtype=torch.float64, device=A.device)
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    lw = int(lib().bdc_geqrf_workspace(m, n))
    work = torch.empty(max(lw, 1), dtype=torch.uint8, device=A.device)
    _check("bdc_geqrf", lib().bdc_geqrf(m, n, _ptr(A), max(m, 1), _ptr(tau), _ptr(work), work.numel(), _ptr(info),
                                         _stream(stream)))
    return A, tau[:min(m, n)], int(info.item())


def orgqr(Ar, tau, stream=None):
    """bdc_orgqr: the explicit m x n Q in place of Ar's reflectors."""
    m, n = Ar.shape
    lw = int(lib().bdc_geqrf_workspace(m, n))
    work = torch.empty(max(lw, 1), dtype=torch.uint8, device=Ar.device)
    _check("bdc_orgqr", lib().bdc_orgqr(m, n, _ptr(Ar), max(Ar.stride(1), 1), _ptr(tau), _ptr(work), work.numel(),
                                         _stream(stream)))
    return Ar


def gesvd(A, *, prec="fp64", leaf=0, slices=0, seed="plain", mlp=None, stream=None, check=True, work=None):
    """bdc_gesvd: dense SVD A = U diag(S) V^T (m >= n); returns (S, U, VT, info)."""
    A = _colmajor(A)
    m, n = A.shape
    dev = A.device
    o = make_opts(prec, leaf, 64, slices, seed, mlp)
    S = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
    Ut = torch.empty((n, m), dtype=torch.float64, device=dev)      # column-major m x n
    VTt = torch.empty((n, n), dtype=torch.float64, device=dev)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    lw = int(lib().bdc_gesvd_workspace(m, n, ctypes.byref(o)))
    if work is None or work.numel() < lw:
        work = torch.empty(max(lw, 1), dtype=torch.uint8, device=dev)
    _check("bdc_gesvd", lib().bdc_gesvd(m, n, _ptr(A), max(m, 1), _ptr(S), _ptr(Ut), max(m, 1), _ptr(VTt), max(n, 1),
                                         ctypes.byref(o), _ptr(work), work.numel(), _ptr(info), _stream(stream)))
    code = int(info.item())
    if check and code != 0:
        raise BDCError("bdc_gesvd (device status)", code)
    return S[:n], Ut.t(), VTt.t(), code
