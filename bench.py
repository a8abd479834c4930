#!/usr/bin/env python
"""Benchmark of the GB300 bidiagonal divide-and-conquer SVD.

Workload: one n x n upper bidiagonal (default n = 16384, d, e ~ U(0.5, 1.5),
seed 0), singular values and both vector sets, through the C ABI
(bdc_svd_ex).  A step is one whole SVD (all stages of Algorithm 2).
The metric is time per SVD (lower is better).  The same invocation times the
three forms the metric compares, with the same warm-up and step counts:
split-BF16 merge products (the timed value), FP64 merge products, and split
BF16 with the MLP-seeded secular roots.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec exact|fp64|bf16x3]
                  [--start mlp|analytic|plain]
  python bench.py --impl reference ...   # the FP64 CPU oracle on host cores
  python bench.py --batched [--dtype fp32] # the 2048-matrix batch on its own line

Multi-GPU runs (torchrun) are independent replicas (weak scaling): every rank
solves its own matrix; value = max-over-ranks step time / N.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "n=16384 bidiagonal SVD (σ+U,V) time, mixed vs FP64 at ≤1e-12 residual; %roofline"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
# FP64 rates of this part measured by throughput probes (per SM per clock):
# mma.sync.m8n8k4.f64 6.66 MAC; DFMA 1.99 lane operations (independent chains
# on every SM: 626.7 G DFMA/s = 1.253 TFLOP/s at 2070 MHz; bench_fp64_peak.cu)
FP64_DMMA_MAC_PER_CLK_SM = 6.66
FP64_ALU_OPS_PER_CLK_SM = 1.99
SMS = 152
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_bdc_exact_uniform_n16384.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2508_11467_gb300", "csrc", f) for f in
                  ("bdc_gemm_mixed.cu", "bdc_secular.cu", "bdc_merge.cu", "bdc_driver.cu", "bdc_leaf.cu",
                   "bdc_gemm64.cu", "bdc_internal.cuh")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default=os.environ.get("BDC_BENCH_PREC", "exact"),
                    choices=["fp64", "exact", "bf16x3"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--kind", default="uniform", choices=["uniform", "graded", "clustered", "ones"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--leaf", type=int, default=8)
    ap.add_argument("--slices", type=int, default=0, help="0 = automatic (7)")
    ap.add_argument("--mixed-min", type=int, default=0, help="smallest merge order using split BF16 (0 = auto)")
    ap.add_argument("--batched", action="store_true",
                    help="only the 2048-matrix batch (n log-uniform in [32, 1024]), one CUDA-graph launch per batch")
    ap.add_argument("--dtype", default="fp64", choices=["fp64", "fp32"], help="batched mode working precision")
    ap.add_argument("--start", default="plain", choices=["plain", "analytic", "mlp"],
                    help="secular root start of the timed form: interval midpoint (FP32 pre-iterations), "
                         "analytic estimate, or analytic + trained MLP")
    ap.add_argument("--no-mlp", action="store_true", help="skip training the root-start MLP (and its timing)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-product comparison")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched keys of the headline line")
    ap.add_argument("--no-dense", action="store_true", help="skip the dense-SVD keys of the headline line")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--oracle-timing", action="store_true",
                    help="only the host oracle: QR with U,V at n = 256 and 4096 (configs 1 and 2, their three "
                         "seeded inputs), one core each and all three on three cores; one JSON line, no GPU")
    return ap.parse_args()


def load_peaks():
    try:
        with open(PEAKS_FILE) as fh:
            p = json.load(fh)
        return p, "measured"
    except Exception:
        return dict(FALLBACK), "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="bdc_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


def workload_name(kind, n, seed):
    rec = {"uniform": "d,e~U(0.5,1.5)", "graded": "d_i=10^(-8i/n)U(0.5,1.5), e=0.5d",
           "clustered": "d=e=1+1e-10 N(0,1)", "ones": "d=e=1"}[kind]
    return f"upper bidiagonal n={n} {rec} seed {seed}, sigma+U+V"


def host_cores():
    try:
        aff = sorted(os.sched_getaffinity(0))
    except AttributeError:
        aff = list(range(os.cpu_count() or 1))
    return aff


# ------------------------------------------------------------- CPU oracle runs
def _oracle_sigma_job(args):
    """One sigma-only QR of the (kind, n, seed) bidiagonal; seconds."""
    kind, n, seed = args
    import oracle
    from paper_2508_11467_gb300 import inputs
    d, e = inputs.make(kind, n, seed)
    t0 = time.perf_counter()
    oracle.sigma_only(d, e)
    return time.perf_counter() - t0


def _oracle_full_job(args):
    """One QR with U and V of the (kind, n, seed) bidiagonal; seconds."""
    kind, n, seed = args
    import oracle
    from paper_2508_11467_gb300 import inputs
    d, e = inputs.make(kind, n, seed)
    t0 = time.perf_counter()
    oracle.bdsqr(d, e)
    return time.perf_counter() - t0


def oracle_parallel(job, args_list, workers):
    """Run oracle jobs in a pool of `workers` spawned processes (spawn: the
    parent may hold a CUDA context); returns (wall seconds, per-job seconds)."""
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        pool.map(_noop, range(workers))          # start-up (interpreter, imports) outside the timing
        t0 = time.perf_counter()
        per = pool.map(job, args_list, chunksize=1)
        wall = time.perf_counter() - t0
    return wall, per


def _noop(_):
    import oracle  # noqa: F401
    from paper_2508_11467_gb300 import inputs  # noqa: F401
    return 0


def cpu_baseline_measured(kind, n, seed, d, e, sigma_seconds):
    """The FP64 QR oracle measured on this host: the sigma-only QR of the
    bench matrix itself (timed by the caller, sigma_seconds, 1 core), and the
    QR with vectors at n=1024 on 1 core and on all cores of the affinity set
    (independent matrices, one per core).  The n^3 scaling to n is a separate,
    labelled field."""
    aff = host_cores()
    cores = len(aff)
    nv = 1024
    t1 = _oracle_full_job((kind, nv, seed))
    wall, per = oracle_parallel(_oracle_full_job, [(kind, nv, seed + k) for k in range(cores)], cores)
    return {"value": sigma_seconds, "unit": "s", "cores": 1, "kind": "oracle",
            "sample": f"sigma-only Golub-Kahan QR of this n={n} {kind} seed {seed} matrix (the sigma reference "
                      f"of accuracy), 1 host core",
            "nproc": os.cpu_count(), "affinity": f"{len(aff)} cores ({aff[0]}..{aff[-1]})",
            "with_vectors": {"n": nv, "s_1core": t1, "s_per_svd_all_cores": wall / cores, "cores": cores,
                             "per_job_s_median": statistics.median(per),
                             "sample": f"Golub-Kahan QR with U,V at n={nv} ({kind}), 1 core; and {cores} "
                                       f"matrices (seeds {seed}..{seed + cores - 1}) on {cores} cores"},
            "with_vectors_n3_extrapolated_to_n_s_1core": {"value": t1 * (n / nv) ** 3, "model": "s_1core x (n/1024)^3",
                                                           "measured": False}}


def run_oracle_timing():
    """The FP64 QR oracle with vectors at the sizes of configs 1 and 2 (n = 256
    and 4096: uniform seed 0, graded seed 1, clustered seed 2), each matrix on
    one core, and the three of a size on three cores at once (one matrix per
    core).  Measured once, separately from the default bench line (the three
    n = 4096 solves take minutes)."""
    aff = host_cores()
    out = {"impl": "oracle-timing", "nproc": os.cpu_count(), "affinity": f"{len(aff)} cores ({aff[0]}..{aff[-1]})",
           "kind": "oracle", "unit": "s", "sizes": {}}
    cases = [("uniform", 0), ("graded", 1), ("clustered", 2)]
    for n in (256, 4096):
        one = {f"{kind} seed {seed}": _oracle_full_job((kind, n, seed)) for kind, seed in cases}
        wall, per = oracle_parallel(_oracle_full_job, [(kind, n, seed) for kind, seed in cases], len(cases))
        out["sizes"][str(n)] = {"s_1core": one, "s_3_matrices_on_3_cores": wall, "per_job_s": per}
    print(json.dumps(out), flush=True)


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over the ranks: N replicas finish a step when the slowest
    one does, so a step's time is the maximum of the ranks' times."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seconds_per_svd(ms_max: float, world: int) -> float:
    """Whole-job seconds per SVD: N replicas each solve one SVD per step of
    ms_max milliseconds (the slowest rank's), N SVDs per step."""
    return ms_max / 1e3 / world


def run_reference(a, rank, world):
    """The FP64 CPU oracle as the reference arm: each step is the sigma-only
    Golub-Kahan QR of the workload matrix (the QR with vectors at n=16384
    runs for hours); the steps run concurrently, one per host core of the
    affinity set, and the value is the wall time of the timed steps / steps."""
    if rank != 0:
        return
    aff = host_cores()
    workers = max(1, min(len(aff), max(a.steps, a.warmup)))
    args = (a.kind, a.n, a.seed)
    wwall, _ = oracle_parallel(_oracle_sigma_job, [args] * a.warmup, workers) if a.warmup > 0 else (0.0, [])
    wall, per = oracle_parallel(_oracle_sigma_job, [args] * a.steps, workers)
    v = wall / a.steps
    line = {
        "metric": METRIC, "value": v, "unit": "s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": workload_name(a.kind, a.n, a.seed), "n": a.n,
                   "impl": "FP64 CPU oracle (Golub-Kahan QR), singular values only"},
        "cpu_baseline": {"value": v, "unit": "s", "cores": workers, "kind": "oracle",
                         "sample": f"sigma-only QR of the n={a.n} {a.kind} seed {a.seed} matrix, {a.steps} steps "
                                   f"run concurrently on {workers} host cores ({wall:.1f} s wall; one step alone "
                                   f"{statistics.median(per):.1f} s median); no vectors",
                         "nproc": os.cpu_count(), "affinity_cores": len(aff)},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ batched
def batched_run(a, dtype_name, steps, warmup, with_oracle=False):
    """The 2048-matrix batch (n log-uniform in [32, 1024], seed 3): autotuned
    plan replayed as one CUDA graph per batch; returns a dict of results."""
    import torch

    from paper_2508_11467_gb300 import bdc, inputs

    dev = torch.device("cuda", 0)
    count = 2048
    mats = inputs.batch(count, seed=3)
    ns = np.array([len(d) for d, _ in mats], dtype=np.int32)
    off = np.concatenate([[0], np.cumsum(ns)])
    Dh = np.zeros(int(off[-1]))
    Eh = np.zeros(int(off[-1]))
    for b, (d, e) in enumerate(mats):
        Dh[off[b]:off[b] + len(d)] = d
        Eh[off[b]:off[b] + len(e)] = e
    dt = torch.float32 if dtype_name == "fp32" else torch.float64
    D_pin = torch.from_numpy(Dh).to(dt).pin_memory()
    E_pin = torch.from_numpy(Eh).to(dt).pin_memory()
    prec = "fp64" if dtype_name == "fp32" else a.prec
    t0 = time.perf_counter()
    leaf, mm, _ = bdc.autotune(ns, prec, slices=a.slices, reps=2, dtype=dt)
    tune_s = time.perf_counter() - t0
    plan = bdc.BatchPlan(D_pin.to(dev), E_pin.to(dev), ns, prec=prec, leaf=leaf, mixed_min=mm, slices=a.slices,
                         dtype=dt)
    st = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.launch()
    torch.cuda.synchronize()
    if int(plan.info.abs().max()) != 0:
        raise RuntimeError("device status " + str(int(plan.info.abs().max())))
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(st)
    for _ in range(steps):
        plan.launch()
    ev1.record(st)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    # end to end: H2D of every d, e; the graph; D2H of every S, U, V^T
    esz = 4 if dtype_name == "fp32" else 8
    # page-locked at allocation (torch.empty(pin_memory=True)); a pageable
    # tensor pinned afterwards measured up to 2x slower in the copies
    S_h = torch.empty(plan.S.shape, dtype=plan.S.dtype, pin_memory=True)
    U_h = torch.empty(plan.U.shape, dtype=plan.U.dtype, pin_memory=True)
    VT_h = torch.empty(plan.VT.shape, dtype=plan.VT.dtype, pin_memory=True)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    k2 = max(1, min(steps, 3))
    w2 = max(1, min(warmup, 2))                 # untimed passes first (first use of the host buffers)
    for it in range(w2 + k2):
        if it == w2:
            f0.record(st)
        plan.d.copy_(D_pin, non_blocking=True)
        plan.e.copy_(E_pin, non_blocking=True)
        plan.launch()
        S_h.copy_(plan.S, non_blocking=True)
        U_h.copy_(plan.U, non_blocking=True)
        VT_h.copy_(plan.VT, non_blocking=True)
    f1.record(st)
    torch.cuda.synchronize()
    ems = f0.elapsed_time(f1) / k2
    # accuracy of a spread of matrices (torch/cuBLAS checkers in FP64)
    order = np.argsort(ns)
    worst = {"residual": 0.0, "orth": 0.0, "checked": 16}
    for b in order[np.linspace(0, count - 1, 16).astype(int)]:
        S, U, VT = plan.result(int(b))
        d = torch.from_numpy(mats[b][0]).to(dev).to(dt).double()
        e = torch.from_numpy(mats[b][1]).to(dev).to(dt).double()
        U, VT, S = U.double(), VT.double(), S.double()
        V = VT.t()
        BV = d[:, None] * V
        BV[:-1] += e[:, None] * V[1:]
        res = float(torch.linalg.norm(BV - U * S[None, :]) / torch.sqrt((d * d).sum() + (e * e).sum()))
        G = U.t() @ U
        G.diagonal().sub_(1.0)
        worst["residual"] = max(worst["residual"], res)
        worst["orth"] = max(worst["orth"], float(torch.linalg.norm(G)))
    out = {"matrices_per_s": count / (ms * 1e-3), "ms_per_batch": ms, "leaf": leaf,
           "mixed_min": mm if prec != "fp64" else None, "prec": prec, "autotune_s": tune_s,
           "e2e_matrices_per_s": count / (ems * 1e-3), "accuracy": worst,
           "h2d_bytes": int(2 * esz * off[-1]), "d2h_bytes": int(esz * (off[-1] + 2 * plan.U.numel())),
           "gflops_model_8n3_3": float(np.sum((8.0 / 3.0) * ns.astype(np.float64) ** 3)) / (ms * 1e-3) / 1e9}
    if with_oracle:
        # the FP64 QR oracle with vectors, every matrix of a spread of 64, on all cores
        sample = [int(b) for b in order[np.linspace(0, count - 1, 64).astype(int)]]
        cores = len(host_cores())
        wall, _ = oracle_parallel(_oracle_batch_job, [(3, b) for b in sample], cores)
        n3 = float(np.sum(ns.astype(np.float64) ** 3))
        s3 = float(np.sum(ns[sample].astype(np.float64) ** 3))
        out["cpu_baseline"] = {"value": count / (wall * n3 / s3), "unit": "matrices/s", "cores": cores,
                               "kind": "oracle",
                               "sample": f"Golub-Kahan QR with U,V on 64 of the 2048 matrices (spread over the "
                                         f"sizes) in {wall:.2f} s on {cores} cores, scaled by sum n^3 to the batch"}
    plan.close()
    del plan
    torch.cuda.empty_cache()
    return out


def _oracle_batch_job(args):
    seed, b = args
    import oracle
    from paper_2508_11467_gb300 import inputs
    d, e = inputs.batch(2048, seed=seed)[b]
    oracle.bdsqr(d, e)
    return 0


def dense_run(steps, warmup):
    """The dense front and back end (Sec. 4.1, 4.3): bidiagonalization of a
    square n = 4096 matrix, and the whole SVD of it and of the paper's
    tall-and-skinny shape m = 20000, n = 1000 (SVD_geo, kappa = 1e4), each
    timed with CUDA events over `steps` calls after `warmup`.  Roofline of the
    reduction: (8/3) n^3 flops, half in products with the trailing matrix
    (the BLAS2 part, FP64 ALU-bound on this part) and half in the merged
    rank-(2b) updates (FP64 tensor cores)."""
    import torch

    from paper_2508_11467_gb300 import bdc, inputs

    out = {}
    clk = 2070e6
    alu = FP64_ALU_OPS_PER_CLK_SM * SMS * clk * 2 / 1e12          # TFLOP/s (FMA = 2)
    dmma = 2 * FP64_DMMA_MAC_PER_CLK_SM * SMS * clk / 1e12
    for name, (m, n, kind) in {"square_n4096": (4096, 4096, "gauss"), "ts_m20000_n1000": (20000, 1000, "geo")}.items():
        if kind == "gauss":
            A0 = torch.randn(m, n, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(7))
        else:
            Q, sg, V = inputs.dense(kind, m, n, 1e4, 0)
            A0 = (torch.from_numpy(Q).cuda() * torch.from_numpy(sg).cuda()[None, :]) @ torch.from_numpy(V).cuda().t()
        A0 = A0.t().contiguous().t()
        res = {}
        # bidiagonalization alone
        lw = int(bdc.lib().bdc_gebrd_workspace(m, n))
        wk = torch.empty(lw, dtype=torch.uint8, device="cuda")
        A = torch.empty_like(A0)
        d = torch.empty(n, dtype=torch.float64, device="cuda")
        e = torch.empty(n, dtype=torch.float64, device="cuda")
        tq = torch.empty(n, dtype=torch.float64, device="cuda")
        tp = torch.empty(n, dtype=torch.float64, device="cuda")
        info = torch.zeros(1, dtype=torch.int32, device="cuda")
        st = torch.cuda.current_stream()

        def gebrd():
            A.copy_(A0)
            rc = bdc.lib().bdc_gebrd(m, n, bdc._ptr(A), m, bdc._ptr(d), bdc._ptr(e), bdc._ptr(tq), bdc._ptr(tp),
                                     bdc._ptr(wk), wk.numel(), bdc._ptr(info), bdc._stream())
            if rc != 0:
                raise RuntimeError(f"bdc_gebrd {rc}")

        def timeit(fn):
            for _ in range(warmup):
                fn()
            torch.cuda.synchronize()
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record(st)
            for _ in range(steps):
                fn()
            c1.record(st)
            torch.cuda.synchronize()
            return c0.elapsed_time(c1) / steps

        ms_copy = timeit(lambda: A.copy_(A0))
        ms_brd = timeit(gebrd) - ms_copy
        flops = 4.0 * m * n * n - 4.0 * n ** 3 / 3.0
        t_min = (flops / 2) / (alu * 1e12) + (flops / 2) / (dmma * 1e12)
        res["gebrd_ms"] = ms_brd
        res["gebrd_gflops"] = flops / (ms_brd * 1e-3) / 1e9
        res["gebrd_roofline_frac"] = t_min / (ms_brd * 1e-3)
        res["gebrd_status"] = int(info.item())
        if m == n:
            del wk
            # the whole dense SVD (split-BF16 merge products in the bidiagonal solve)
            o = bdc.make_opts("exact")
            lw2 = int(bdc.lib().bdc_gesvd_workspace(m, n, __import__("ctypes").byref(o)))
            wk2 = torch.empty(lw2, dtype=torch.uint8, device="cuda")
            S, U, VT = (torch.empty(n, dtype=torch.float64, device="cuda"),
                        torch.empty((n, m), dtype=torch.float64, device="cuda"),
                        torch.empty((n, n), dtype=torch.float64, device="cuda"))
        else:
            o = bdc.make_opts("exact")
            lw2 = int(bdc.lib().bdc_gesvd_workspace(m, n, __import__("ctypes").byref(o)))
            wk2 = torch.empty(lw2, dtype=torch.uint8, device="cuda")
            S, U, VT = (torch.empty(n, dtype=torch.float64, device="cuda"),
                        torch.empty((n, m), dtype=torch.float64, device="cuda"),
                        torch.empty((n, n), dtype=torch.float64, device="cuda"))
        import ctypes as _ct

        def gesvd():
            A.copy_(A0)
            rc = bdc.lib().bdc_gesvd(m, n, bdc._ptr(A), m, bdc._ptr(S), bdc._ptr(U), m, bdc._ptr(VT), n,
                                     _ct.byref(o), bdc._ptr(wk2), wk2.numel(), bdc._ptr(info), bdc._stream())
            if rc != 0:
                raise RuntimeError(f"bdc_gesvd {rc}")

        ms_svd = timeit(gesvd) - ms_copy
        Uc, VTc = U.t(), VT.t()
        rel = float(torch.linalg.norm(Uc * S[None, :] @ VTc - A0) / torch.linalg.norm(A0))
        res.update({"gesvd_ms": ms_svd, "gesvd_status": int(info.item()), "gesvd_residual": rel,
                    "shape": [m, n], "matrix": kind, "bdc_products": "split BF16 (7 slices)",
                    "qr_first": m >= 1.6 * n})
        out[name] = res
        del A, A0, U, VT, wk2
        torch.cuda.empty_cache()
    out["roofline_note"] = (f"bidiagonalization lower bound: half its (4 m n^2 - 4 n^3 / 3) flops at the FP64 ALU "
                            f"peak {alu:.3f} TFLOP/s, half at the FP64 mma.sync peak {dmma:.2f} TFLOP/s")
    return out


def run_batched(a):
    """--batched: the batch on its own JSON line (matrices/s)."""
    import torch

    from paper_2508_11467_gb300 import bdc, build

    torch.cuda.set_device(0)
    build.build()
    bdc.lib()
    clocks = ClockSampler(0)
    clocks.start()
    r = batched_run(a, a.dtype, a.steps, a.warmup, with_oracle=not a.no_cpu_baseline)
    clk = clocks.stop()
    line = {
        "metric": "2048 bidiagonals (n log-uniform in [32,1024]) SVD (sigma+U,V) throughput",
        "value": r["matrices_per_s"], "unit": "matrices/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": r["ms_per_batch"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if a.dtype == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": "2048 upper bidiagonals, n = floor(exp(U(ln 32, ln 1024))) seed 3, d,e~U(0.5,1.5)",
                   "prec": r["prec"], "leaf": r["leaf"], "mixed_min": r["mixed_min"], "autotune_s": r["autotune_s"],
                   "launch": "one CUDA graph per batch (bdc_plan_launch)",
                   "l2": "U, V and workspace of the batch (> 5 GB) exceed L2"},
        "gflops_model_8n3_3": r["gflops_model_8n3_3"],
        "accuracy": r["accuracy"], "roofline": None, "gpu_launches": None,
        "e2e": {"value": r["e2e_matrices_per_s"], "unit": "matrices/s", "h2d_bytes_per_step": r["h2d_bytes"],
                "d2h_bytes_per_step": r["d2h_bytes"]},
        "cpu_baseline": r.get("cpu_baseline"), "clocks": clk,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ rooflines
def kernel_sources_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None when there is none or the kernel sources changed since it was taken
    (the summary records the hash of the kernel sources it measured)."""
    try:
        txt = open(TRAFFIC_FILE).read()
    except OSError:
        return None
    m = re.search(r"^sources:\s*([0-9a-f]{16})", txt, re.M)
    if not m or m.group(1) != kernel_sources_hash():
        return None
    m = re.search(rf"^traffic_per_launch\s+{re.escape(kernel)}\s+([0-9.eE+]+)", txt, re.M)
    return float(m.group(1)) if m else None


STAGE_KERNELS = {"scale": "k_scale", "leaf": "k_leaf_rotations + k_leaf_vectors", "prep": "k_merge_prep",
                 "gather": "k_merge_gather", "secular": "k_secular (+ k_root_start)", "lowner": "k_lowner",
                 "vectors": "k_vectors_warp", "slice": "k_slice_a + k_slice_b",
                 "gemm": "k_mma (tcgen05) / k_gemm64 (DMMA f64)", "finish": "k_merge_finish", "final": "k_final"}


def stage_table(prof, steps, peaks, clock_mhz, fp64_products):
    """Per stage: time, launches, algorithmic bytes and FP64 operations, the
    achieved rates and their fractions of the measured HBM copy bandwidth, the
    FP64 ALU rate and the tensor peak; `bound` names the roofline that binds."""
    hbm = float(peaks.get("hbm_gbs", FALLBACK["hbm_gbs"]))
    clk = (clock_mhz or 2070.0) * 1e6
    fp64_alu = FP64_ALU_OPS_PER_CLK_SM * SMS * clk / 1e9          # G FP64 ops / s
    fp64_dmma = 2 * FP64_DMMA_MAC_PER_CLK_SM * SMS * clk / 1e12   # TFLOP/s
    bf16 = float(peaks.get("bf16_tflops", FALLBACK["bf16_tflops"]))
    out = {}
    for k, v in prof.items():
        if v["ms"] <= 0:
            continue
        t = v["ms"] * 1e-3
        row = {"kernel": STAGE_KERNELS.get(k, k), "ms_per_step": v["ms"] / steps,
               "launches_per_step": v["launches"] / steps}
        if k == "gemm":
            tf = v["work"] / t / 1e12
            peak = fp64_dmma if fp64_products else bf16
            row.update({"tflops_executed": tf, "tensor_peak_tflops": peak, "tensor_frac": tf / peak,
                        "bound": "tensor", "work_per_step": v["work"] / steps})
        else:
            gbs = v["work"] / t / 1e9
            fg = v["fp64"] / t / 1e9
            row.update({"bytes_per_step": v["work"] / steps, "GBps": gbs, "hbm_frac": gbs / hbm,
                        "fp64_ops_per_step": v["fp64"] / steps, "fp64_gops": fg, "fp64_frac": fg / fp64_alu})
            row["bound"] = "fp64" if row["fp64_frac"] > row["hbm_frac"] else "hbm"
            if max(row["fp64_frac"], row["hbm_frac"]) < 0.05:
                row["bound"] += " (latency: below 5% of both)"
        if v.get("level_ms"):
            # per merge height (0 = right above the leaves): ms and the fraction of
            # the stage's peak (FP64 ALU for the FP64 stages, tensor for products)
            row["level_ms"] = [x / steps for x in v["level_ms"]]
            if k in ("secular", "lowner", "vectors"):
                row["level_fp64_frac"] = [(w / (t * 1e-3)) / (fp64_alu * 1e9) if t > 0 else 0.0
                                          for w, t in zip(v["level_work"], v["level_ms"])]
            elif k == "gemm":
                row["level_tensor_frac"] = [(w / (t * 1e-3)) / ((fp64_dmma if fp64_products else bf16) * 1e12)
                                            if t > 0 else 0.0 for w, t in zip(v["level_work"], v["level_ms"])]
        out[k] = row
    if prof["secular"].get("roots"):
        out.setdefault("secular", {})["roots_per_step"] = prof["secular"]["roots"] / steps
        out["secular"]["iters_per_root"] = prof["secular"]["iters"] / prof["secular"]["roots"]
    return out, {"hbm_gbs": hbm, "fp64_alu_gops": fp64_alu, "fp64_dmma_tflops": fp64_dmma, "bf16_tflops": bf16}


def main():
    a = parse()
    if a.oracle_timing:
        run_oracle_timing()
        return
    if a.batched and a.impl != "reference":
        if int(os.environ.get("WORLD_SIZE", "1")) > 1:
            raise SystemExit("--batched measures one GPU; run it without torchrun")
        run_batched(a)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return

    import ctypes

    import torch
    import torch.distributed as dist

    from paper_2508_11467_gb300 import bdc, build, inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    build.build()
    L = bdc.lib()

    n = a.n
    d_h, e_h = inputs.make(a.kind, n, a.seed + rank)
    d_pin = torch.from_numpy(d_h).pin_memory()
    e_pin = torch.from_numpy(e_h).pin_memory()
    d = d_pin.to(dev)
    e = e_pin.to(dev)
    # root starts: the MLP is trained here, before any timing, by the
    # library (bdc_mlp_train: roots harvested from FP64 solves of an n = 8192
    # uniform and an n = 8192 graded bidiagonal generated on the device)
    P = None
    train_info = None
    if a.start == "mlp" or not a.no_mlp:
        t0 = time.perf_counter()
        P, losses, samples = bdc.mlp_train_harvest(n=8192, steps=1500, lr=3e-3, huber=0.25, seed=1)
        torch.cuda.synchronize()
        train_info = {"samples": samples, "steps": 1500, "loss": [float(losses[0]), float(losses[-1])],
                      "seconds": time.perf_counter() - t0,
                      "data": "bdc_mlp_train: n=8192 uniform + graded bidiagonals generated on the device (seed 1)"}

    forms = {"mixed": bdc.make_opts(a.prec, a.leaf, 64, a.slices, seed=a.start, mlp=P, mixed_min=a.mixed_min)}
    if not a.no_fp64 and a.prec != "fp64":
        forms["fp64"] = bdc.make_opts("fp64", a.leaf, 64, 0, seed="plain")
    if P is not None and a.start != "mlp" and a.prec != "fp64":
        forms["mixed_mlp"] = bdc.make_opts(a.prec, a.leaf, 64, a.slices, seed="mlp", mlp=P, mixed_min=a.mixed_min)
    lw = max(bdc.workspace_bytes(n, o) for o in forms.values())
    work = torch.empty(lw + 256, dtype=torch.uint8, device=dev)
    Ut = torch.empty((n, n), dtype=torch.float64, device=dev)
    VTt = torch.empty((n, n), dtype=torch.float64, device=dev)
    S = torch.empty(n, dtype=torch.float64, device=dev)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    st = torch.cuda.current_stream()

    def step(o, dd, ee, U_=Ut, S_=S, VT_=VTt, stream=st):
        rc = L.bdc_svd_ex(n, bdc._ptr(dd), bdc._ptr(ee), bdc._ptr(U_), bdc._ptr(S_), bdc._ptr(VT_), n, n,
                          ctypes.byref(o), bdc._ptr(work), work.numel(), bdc._ptr(info),
                          ctypes.c_void_p(stream.cuda_stream))
        if rc != 0:
            raise RuntimeError(f"bdc_svd_ex failed: {rc} {bdc.status_string(rc)}")

    # sigma reference: the oracle's sigma-only QR of this matrix (also the CPU baseline)
    sigma_ref = sigma_s = None
    if rank == 0 and not (a.no_check and a.no_cpu_baseline):
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        sigma_ref = oracle.sigma_only(d_h, e_h)
        sigma_s = time.perf_counter() - t0

    def accuracy():
        U = Ut.t()
        VT = VTt.t()
        V = VT.t()
        BV = d[:, None] * V
        BV[:-1] += e[:, None] * V[1:]
        R = BV - U * S[None, :]
        bn = torch.sqrt((d * d).sum() + (e * e).sum())
        res = float(torch.linalg.norm(R) / bn)
        g = torch.Generator(device="cpu").manual_seed(1)
        cols = torch.randperm(n, generator=g)[:256].to(dev)
        Gu = U[:, cols].t() @ U
        Gv = VT[cols, :] @ VT.t()
        idx = torch.arange(256, device=dev)
        Gu[idx, cols] -= 1.0
        Gv[idx, cols] -= 1.0
        acc = {"residual": res, "orth_u_sample": float(torch.linalg.norm(Gu)),
               "orth_v_sample": float(torch.linalg.norm(Gv)),
               "orth_sample": "256 random columns against all n, Frobenius"}
        if sigma_ref is not None:
            s = S.cpu().numpy()
            acc["sigma_rel_err"] = float(np.max(np.abs(s - sigma_ref)) / sigma_ref[0])
            acc["sigma_ref"] = "oracle sigma-only QR (FP64, host)"
        return acc

    clocks = ClockSampler(local)
    clocks.start()
    timed = {}
    accs = {}
    for name, o in forms.items():
        for _ in range(a.warmup):
            step(o, d, e)
        torch.cuda.synchronize()
        if int(info.item()) != 0:
            raise RuntimeError(f"{name}: device status {int(info.item())}: {bdc.status_string(int(info.item()))}")
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(st)
        for _ in range(a.steps):
            step(o, d, e)
        ev1.record(st)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        timed[name] = max_over_ranks(ev0.elapsed_time(ev1) / a.steps, world, dev)
        if int(info.item()) != 0:
            raise RuntimeError(f"{name}: device status {int(info.item())}")
        if not a.no_check and rank == 0:
            accs[name] = accuracy()
    clk = clocks.stop()
    ms = timed["mixed"]
    status = int(info.item())

    # stage split: one profiled (untimed) SVD of each form after the timed ones
    profs = {}
    for name, o in forms.items():
        bdc.profile_begin()
        step(o, d, e)
        torch.cuda.synchronize()
        profs[name] = bdc.profile_end()

    # end to end through the C ABI from pinned host buffers: H2D of d, e, the
    # SVD, D2H of S, U, V^T every step.  Two schedules, both timed: serial
    # (one stream) and double-buffered (the device-to-host copy of step k on
    # a copy stream overlaps the SVD of step k+1); the faster is the value.
    e2e = None
    if not a.no_e2e:
        o = forms["mixed"]
        cs = torch.cuda.Stream(device=dev)
        outs = [(Ut, S, VTt)] + [(torch.empty_like(Ut), torch.empty_like(S), torch.empty_like(VTt))]
        hosts = []
        for _ in range(2):
            hU = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
            hS = torch.empty(n, dtype=torch.float64, pin_memory=True)
            hVT = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
            hosts.append((hU, hS, hVT))
        d2 = torch.empty_like(d)
        e2 = torch.empty_like(e)
        svd_done = [torch.cuda.Event() for _ in range(2)]
        copy_done = [torch.cuda.Event() for _ in range(2)]
        k2 = max(2, a.steps)

        def e2e_serial(k_steps):
            hU, hS, hVT = hosts[0]
            for _ in range(k_steps):
                d2.copy_(d_pin, non_blocking=True)
                e2.copy_(e_pin, non_blocking=True)
                step(o, d2, e2)
                hS.copy_(S, non_blocking=True)
                hU.copy_(Ut, non_blocking=True)
                hVT.copy_(VTt, non_blocking=True)

        def e2e_pipelined(k_steps):
            for k in range(k_steps):
                b = k % 2
                if k >= 2:
                    st.wait_event(copy_done[b])          # host buffer b and outputs b are free again
                d2.copy_(d_pin, non_blocking=True)
                e2.copy_(e_pin, non_blocking=True)
                U_, S_, VT_ = outs[b]
                step(o, d2, e2, U_, S_, VT_)
                svd_done[b].record(st)
                cs.wait_event(svd_done[b])
                hU, hS, hVT = hosts[b]
                with torch.cuda.stream(cs):
                    hS.copy_(S_, non_blocking=True)
                    hU.copy_(U_, non_blocking=True)
                    hVT.copy_(VT_, non_blocking=True)
                copy_done[b].record(cs)
            for b in range(2):
                st.wait_event(copy_done[b])

        def time_e2e(fn):
            fn(2)                                        # warm-up (page-in of the pinned buffers)
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(st)
            fn(k2)
            f1.record(st)
            torch.cuda.synchronize()
            return max_over_ranks(f0.elapsed_time(f1) / k2, world, dev)

        ms_serial = time_e2e(e2e_serial)
        ms_pipe = time_e2e(e2e_pipelined)
        ok = bool(torch.equal(hosts[(k2 - 1) % 2][1], S.cpu()))
        best = min(ms_serial, ms_pipe)
        e2e = {"value": replica_seconds_per_svd(best, world), "unit": "s", "h2d_bytes_per_step": int(8 * (2 * n - 1)),
               "d2h_bytes_per_step": int(8 * (n + 2 * n * n)), "steps": k2,
               "serial_ms": ms_serial, "pipelined_ms": ms_pipe,
               "schedule": "pipelined" if ms_pipe <= ms_serial else "serial",
               "pipelined": "outputs double-buffered: D2H of step k on a copy stream overlaps the SVD of step k+1",
               "result_matches_device_run": ok}
        del outs, hosts

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peaks, peak_src = load_peaks()
    sm_mhz = (clk or {}).get("sm_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
    stages = {}
    pk = None
    for name, pr in profs.items():
        stages[name], pk = stage_table(pr, 1, peaks, sm_mhz, fp64_products=(name == "fp64"))
    main_stages = stages["mixed"]
    dominant = max(main_stages, key=lambda k: main_stages[k].get("ms_per_step", 0.0))
    dom = main_stages[dominant]
    if dom["bound"] == "tensor":
        roofline = {"bound": "tensor", "achieved": dom["tflops_executed"], "peak": dom["tensor_peak_tflops"],
                    "unit": "TFLOP/s", "frac": dom["tensor_frac"]}
        roofline["peak_source"] = (f"bf16_tflops burst ({peak_src}; an ms-scale kernel timed alone)"
                                   if a.prec != "fp64" else "FP64 mma.sync probe rate x clock")
    elif dom["bound"].startswith("fp64"):
        roofline = {"bound": "alu", "achieved": dom["fp64_gops"], "peak": pk["fp64_alu_gops"], "unit": "GFLOP/s",
                    "frac": dom["fp64_frac"],
                    "peak_source": f"FP64 lane operations: {FP64_ALU_OPS_PER_CLK_SM}/clk/SM (DFMA probe) x {SMS} SMs "
                                   f"x {sm_mhz:.0f} MHz (median SM clock of the timed region)"}
    else:
        roofline = {"bound": "hbm", "achieved": dom["GBps"], "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": dom["hbm_frac"], "peak_source": f"hbm_gbs ({peak_src})"}
    roofline["kernel"] = dom["kernel"]
    roofline["stage"] = dominant
    roofline["stage_ms_per_step"] = dom["ms_per_step"]
    roofline["traffic"] = read_traffic(dominant)
    roofline["traffic_note"] = ("dram__bytes_read.sum + dram__bytes_write.sum per launch, " + os.path.relpath(
        TRAFFIC_FILE, ROOT)) if roofline["traffic"] is not None else "no ncu capture of the current kernel sources"
    launches = int(sum(v["launches"] for v in profs["mixed"].values()))

    root_start = {"mode": a.start, "iters_per_root": main_stages.get("secular", {}).get("iters_per_root"),
                  "mlp_training": train_info}
    if "mixed_mlp" in stages:
        root_start["mlp"] = {"iters_per_root": stages["mixed_mlp"].get("secular", {}).get("iters_per_root"),
                             "svd_ms": timed["mixed_mlp"],
                             "secular_ms": stages["mixed_mlp"].get("secular", {}).get("ms_per_step")}

    comparison = {"mixed_ms": timed["mixed"]}
    if "fp64" in timed:
        comparison.update({"fp64_ms": timed["fp64"], "fp64_over_mixed": timed["fp64"] / timed["mixed"]})
    if "mixed_mlp" in timed:
        comparison.update({"mixed_mlp_ms": timed["mixed_mlp"], "fp64_over_mixed_mlp":
                           (timed["fp64"] / timed["mixed_mlp"]) if "fp64" in timed else None,
                           "mixed_mlp_over_mixed": timed["mixed_mlp"] / timed["mixed"]})

    batch = None
    if not a.no_batch and world == 1:
        del work, Ut, VTt
        torch.cuda.empty_cache()
        batch = {}
        for dt in ("fp64", "fp32"):
            r = batched_run(a, dt, a.steps, a.warmup)
            batch[dt] = {k: r[k] for k in ("matrices_per_s", "ms_per_batch", "e2e_matrices_per_s", "leaf",
                                           "mixed_min", "prec", "accuracy")}
        batch["workload"] = "2048 bidiagonals, n = floor(exp(U(ln 32, ln 1024))) seed 3, d,e~U(0.5,1.5); one graph"

    dense = None
    if not a.no_dense and world == 1:
        if "work" in dir():
            pass
        torch.cuda.empty_cache()
        dense = dense_run(max(1, min(a.steps, 3)), 1)

    cpu = None
    if not a.no_cpu_baseline and world == 1 and sigma_s is not None:
        cpu = cpu_baseline_measured(a.kind, n, a.seed, d_h, e_h, sigma_s)

    line = {
        "metric": METRIC,
        "value": replica_seconds_per_svd(ms, world),
        "unit": "s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": ms,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if a.prec == "fp64" else "f64 (merge products: bf16 slices, exact int accumulation)",
        "data": "synthetic",
        "config": {"workload": workload_name(a.kind, n, a.seed), "n": n, "prec": a.prec, "leaf": a.leaf,
                   "slices": (a.slices or 7) if a.prec == "exact" else None,
                   "l2": "inputs larger than L2 (U, V and workspace > 10 GB per step)",
                   "start": a.start, "fp32_root_start": True, "parallelism": f"replicas x{world}"},
        "comparison": comparison,
        "status": status,
        "accuracy": accs.get("mixed"),
        "accuracy_fp64": accs.get("fp64"),
        "accuracy_mixed_mlp": accs.get("mixed_mlp"),
        "roofline": roofline,
        "peaks": pk,
        "stages": main_stages,
        "stages_fp64": stages.get("fp64"),
        "root_start": root_start,
        "batched": batch,
        "dense": dense,
        "gpu_launches": launches * a.steps,
        "gflops_model_8n3_3": 8.0 / 3.0 * n ** 3 / (ms * 1e-3) / 1e9,
        "gflops_model_note": "the paper's (8/3) n^3 flop model / time; deflation removes most of that work here",
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
