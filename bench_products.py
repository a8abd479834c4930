"""The split-BF16 merge product alone (bdc_gemm, 7 slices) at the shapes of
the top merges of an n = 16384 solve: M x K times K x N for (M, N, K) =
(8193, 420, 420), (8193, 1024, 1024), (4097, 2048, 2048), Gaussian operands
with unit column norms.  Prints per call the time, the slicing and MMA
kernels' times (stage profiler) and the executed slice-pair rate.

  python bench_products.py [calls per shape]
"""
import sys, os, time
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import torch
from paper_2508_11467_gb300 import bdc, build
build.build(); bdc.lib()
torch.manual_seed(0)
shapes = [(8193, 420, 420), (8193, 1024, 1024), (4097, 2048, 2048)]
reps = int(sys.argv[1]) if len(sys.argv) > 1 else 5
for (M, N, K) in shapes:
    A = torch.randn(M, K, dtype=torch.float64, device="cuda") / M**0.5
    B = torch.randn(K, N, dtype=torch.float64, device="cuda") / K**0.5
    C = bdc.gemm(A, B, prec="exact", slices=7)
    ref = A @ B
    err = float((C - ref).abs().max())
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    lw = int(bdc.lib().bdc_gemm_workspace(M, N, K, 2, 7))
    work = torch.empty(lw + 256, dtype=torch.uint8, device="cuda")
    for _ in range(2): bdc.gemm(A, B, prec="exact", slices=7, work=work)
    torch.cuda.synchronize()
    bdc.profile_begin()
    e0.record()
    for _ in range(reps): bdc.gemm(A, B, prec="exact", slices=7, work=work)
    e1.record(); torch.cuda.synchronize()
    pr = bdc.profile_end()
    ms = e0.elapsed_time(e1) / reps
    fl = 2.0 * M * N * K * 28
    print(f"M={M} N={N} K={K}: {ms*1e3:.1f} us/call, slice {pr['slice']['ms']/reps*1e3:.1f} us, mma {pr['gemm']['ms']/reps*1e3:.1f} us, "
          f"executed {fl/ (pr['gemm']['ms']/reps*1e-3)/1e12:.0f} TFLOP/s in the MMA kernels, max err {err:.2e}")
