#!/usr/bin/env python
"""Benchmark of the GB300 bidiagonal divide-and-conquer SVD.

Workload: one n x n upper bidiagonal (default n = 16384, d, e ~ U(0.5, 1.5),
seed 0), singular values and both vector sets, through the C ABI
(bdc_svd_ex).  A step is one whole SVD (all stages of Algorithm 2).
The metric is time per SVD (lower is better).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec exact|fp64|bf16x3]
                  [--start mlp|analytic|plain]
  python bench.py --impl reference ...   # the FP64 CPU oracle on host cores

Multi-GPU runs (torchrun) are independent replicas (weak scaling): every rank
solves its own matrix; value = max-over-ranks step time / N.
"""
from __future__ import annotations

import argparse
import json
import os
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
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# FP64 tensor-core (mma.sync f64) rate measured on this part by a throughput
# probe: 6.66 MAC/clk/SM x 152 SMs x 2.07 GHz x 2 = 4.19 TFLOP/s
FP64_DMMA_TFLOPS = 4.19


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
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
                    help="2048 bidiagonals, n log-uniform in [32, 1024], one CUDA-graph launch per batch")
    ap.add_argument("--dtype", default="fp64", choices=["fp64", "fp32"], help="batched mode working precision")
    ap.add_argument("--start", default="plain", choices=["plain", "analytic", "mlp"],
                    help="timed secular root start: interval midpoint (FP32 pre-iterations), analytic estimate, "
                         "or analytic + trained MLP; the other two are reported from untimed runs")
    ap.add_argument("--no-mlp", action="store_true", help="skip training the root-start MLP (and its comparison)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-check", action="store_true")
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
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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


def workload_name(a):
    rec = {"uniform": "d,e~U(0.5,1.5)", "graded": "d_i=10^(-8i/n)U(0.5,1.5), e=0.5d",
           "clustered": "d=e=1+1e-10 N(0,1)", "ones": "d=e=1"}[a.kind]
    return f"upper bidiagonal n={a.n} {rec} seed {a.seed}, sigma+U+V"


def cpu_baseline_oracle(n_target: int, kind: str, seed: int, n_sample: int = 1024, reps: int = 2):
    """Time the FP64 QR oracle (with vectors) on a bounded sample and scale by n^3."""
    import oracle
    from paper_2508_11467_gb300 import inputs
    oracle.build()
    d, e = inputs.make(kind, n_sample, seed)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.bdsqr(d, e)
        times.append(time.perf_counter() - t0)
    t = min(times)
    scale = (n_target / n_sample) ** 3
    return {"value": t * scale, "unit": "s", "cores": 1, "kind": "oracle",
            "sample": f"Golub-Kahan QR with U,V at n={n_sample} ({kind}, seed {seed}), best of {reps} "
                      f"= {t:.3f} s on 1 host core, scaled by (n/{n_sample})^3 to n={n_target}"}


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
    if rank != 0:
        return
    for _ in range(a.warmup):
        cpu_baseline_oracle(a.n, a.kind, a.seed, reps=1)
    vals = []
    t0 = time.perf_counter()
    for _ in range(a.steps):
        vals.append(cpu_baseline_oracle(a.n, a.kind, a.seed, reps=1)["value"])
    wall = time.perf_counter() - t0
    cb = cpu_baseline_oracle.__defaults__
    v = float(np.median(vals))
    line = {
        "metric": METRIC, "value": v, "unit": "s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": workload_name(a), "n": a.n, "impl": "FP64 CPU oracle (Golub-Kahan QR)"},
        "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": f"Golub-Kahan QR with U,V at n={cb[0]}, scaled by n^3; "
                                   f"{a.steps} steps in {wall:.1f} s"},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batched(a):
    """The 2048-matrix batch (n log-uniform in [32, 1024]): the whole batch per step, replayed as one CUDA graph."""
    import torch

    from paper_2508_11467_gb300 import bdc, build, inputs

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    build.build()
    bdc.lib()
    count = 2048
    mats = inputs.batch(count, seed=3)
    ns = np.array([len(d) for d, _ in mats], dtype=np.int32)
    off = np.concatenate([[0], np.cumsum(ns)])
    Dh = np.zeros(int(off[-1]))
    Eh = np.zeros(int(off[-1]))
    for b, (d, e) in enumerate(mats):
        Dh[off[b]:off[b] + len(d)] = d
        Eh[off[b]:off[b] + len(e)] = e
    dt = torch.float32 if a.dtype == "fp32" else torch.float64
    D_pin = torch.from_numpy(Dh).to(dt).pin_memory()
    E_pin = torch.from_numpy(Eh).to(dt).pin_memory()
    # FP64 batches take the split-BF16 products (FP64-accurate, autotuned
    # mixed_min) unless --prec fp64 asks for FP64 tensor-core products
    prec = "fp64" if a.dtype == "fp32" else a.prec
    t0 = time.perf_counter()
    leaf, mm, tune_ms = bdc.autotune(ns, prec, slices=a.slices, reps=2, dtype=dt)
    tune_s = time.perf_counter() - t0
    plan = bdc.BatchPlan(D_pin.to(dev), E_pin.to(dev), ns, prec=prec, leaf=leaf, mixed_min=mm, slices=a.slices,
                         dtype=dt)
    st = torch.cuda.current_stream()
    for _ in range(a.warmup):
        plan.launch()
    torch.cuda.synchronize()
    if int(plan.info.abs().max()) != 0:
        raise RuntimeError("device status " + str(int(plan.info.abs().max())))
    clocks = ClockSampler(0)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(st)
    for _ in range(a.steps):
        plan.launch()
    ev1.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / a.steps
    # end to end: H2D of every d, e; the graph; D2H of every S, U, V^T
    esz = 4 if a.dtype == "fp32" else 8
    S_h = torch.empty_like(plan.S, device="cpu").pin_memory()
    U_h = torch.empty_like(plan.U, device="cpu").pin_memory()
    VT_h = torch.empty_like(plan.VT, device="cpu").pin_memory()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    k2 = max(1, min(a.steps, 3))
    f0.record(st)
    for _ in range(k2):
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
    worst = {"residual": 0.0, "orth": 0.0}
    for b in order[np.linspace(0, count - 1, 12).astype(int)]:
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
    # the FP64 QR oracle on host cores, per matrix, on a bounded sample
    cpu = None
    if not a.no_cpu_baseline:
        import oracle
        oracle.build()
        sample = [int(b) for b in order[np.linspace(0, count - 1, 24).astype(int)]]
        t0 = time.perf_counter()
        for b in sample:
            oracle.bdsqr(*mats[b])
        t = time.perf_counter() - t0
        n3 = float(np.sum(ns.astype(np.float64) ** 3))
        s3 = float(np.sum(ns[sample].astype(np.float64) ** 3))
        cpu_s = t * n3 / s3
        cpu = {"value": count / cpu_s, "unit": "matrices/s", "cores": 1, "kind": "oracle",
               "sample": f"Golub-Kahan QR with U,V on 24 of the 2048 matrices (spread over the sizes) = {t:.2f} s "
                         f"on 1 host core, scaled by sum n^3 to the batch"}
    flops = float(np.sum((8.0 / 3.0) * ns.astype(np.float64) ** 3))
    line = {
        "metric": "2048 bidiagonals (n log-uniform in [32,1024]) SVD (sigma+U,V) throughput",
        "value": count / (ms * 1e-3), "unit": "matrices/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if a.dtype == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": "2048 upper bidiagonals, n = floor(exp(U(ln 32, ln 1024))) seed 3, d,e~U(0.5,1.5)",
                   "prec": prec, "slices": a.slices if a.slices else 7,
                   "leaf": leaf, "mixed_min": mm if prec != "fp64" else None, "autotune_s": tune_s, "launch": "one CUDA graph per batch (bdc_plan_launch)",
                   "l2": "U, V and workspace of the batch (> 5 GB) exceed L2"},
        "gflops_paper_model": flops / (ms * 1e-3) / 1e9,
        "accuracy": worst,
        "roofline": None,
        "gpu_launches": None,
        "e2e": {"value": count / (ems * 1e-3), "unit": "matrices/s", "h2d_bytes_per_step": int(2 * esz * off[-1]),
                "d2h_bytes_per_step": int(esz * (off[-1] + 2 * plan.U.numel()))},
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    plan.close()
    print(json.dumps(line), flush=True)


def main():
    a = parse()
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
    # root starts: the MLP is trained here, before any timing, with the
    # library's own kernels on roots harvested from FP64 runs of n = 8192
    # uniform (seed 4) and graded (seed 5) bidiagonals
    P = None
    train_info = None
    if a.start == "mlp" or not a.no_mlp:
        t0 = time.perf_counter()
        H = bdc.Harvest(1 << 21, device=dev)
        for kind, sd in (("uniform", 4), ("graded", 5)):
            dh, eh = inputs.make(kind, 8192, sd)
            bdc.svd_harvest(torch.from_numpy(dh).to(dev), torch.from_numpy(eh).to(dev), H)
        F, R = H.data()
        P, losses = bdc.mlp_train(F, R, steps=1500, lr=3e-3, seed=0, huber=0.25)
        torch.cuda.synchronize()
        g = bdc.mlp_predict(P, F)
        train_info = {"samples": int(F.shape[0]), "steps": 1500, "loss": [float(losses[0]), float(losses[-1])],
                      "median_abs_err_analytic": float(R.abs().median()),
                      "median_abs_err_mlp": float((g - R).abs().median()),
                      "seconds": time.perf_counter() - t0,
                      "data": "harvest of n=8192 uniform seed 4 + graded seed 5 (FP64 runs)"}
        del H
    o = bdc.make_opts(a.prec, a.leaf, 64, a.slices, seed=a.start, mlp=P, mixed_min=a.mixed_min)
    lw = bdc.workspace_bytes(n, o)
    work = torch.empty(lw + 256, dtype=torch.uint8, device=dev)
    Ut = torch.empty((n, n), dtype=torch.float64, device=dev)
    VTt = torch.empty((n, n), dtype=torch.float64, device=dev)
    S = torch.empty(n, dtype=torch.float64, device=dev)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    st = torch.cuda.current_stream()

    import ctypes

    def step(dd, ee):
        rc = L.bdc_svd_ex(n, bdc._ptr(dd), bdc._ptr(ee), bdc._ptr(Ut), bdc._ptr(S), bdc._ptr(VTt), n, n,
                          ctypes.byref(o), bdc._ptr(work), work.numel(), bdc._ptr(info),
                          ctypes.c_void_p(st.cuda_stream))
        if rc != 0:
            raise RuntimeError(f"bdc_svd_ex failed: {rc} {bdc.status_string(rc)}")

    for _ in range(a.warmup):
        step(d, e)
    torch.cuda.synchronize()
    if int(info.item()) != 0:
        raise RuntimeError(f"device status {int(info.item())}: {bdc.status_string(int(info.item()))}")

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    bdc.profile_begin()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(st)
    for _ in range(a.steps):
        step(d, e)
    ev1.record(st)
    torch.cuda.synchronize()
    prof = bdc.profile_end()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / a.steps, world, dev)
    status = int(info.item())

    # end to end through the C ABI from pinned host buffers: H2D inputs, SVD, D2H S, U, V^T
    e2e = None
    if not a.no_e2e:
        S_h = torch.empty(n, dtype=torch.float64).pin_memory()
        U_h = torch.empty((n, n), dtype=torch.float64).pin_memory()
        VT_h = torch.empty((n, n), dtype=torch.float64).pin_memory()
        d2 = torch.empty_like(d)
        e2 = torch.empty_like(e)
        k2 = max(1, min(a.steps, 3))
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(st)
        for _ in range(k2):
            d2.copy_(d_pin, non_blocking=True)
            e2.copy_(e_pin, non_blocking=True)
            step(d2, e2)
            S_h.copy_(S, non_blocking=True)
            U_h.copy_(Ut, non_blocking=True)
            VT_h.copy_(VTt, non_blocking=True)
        f1.record(st)
        torch.cuda.synchronize()
        ems = max_over_ranks(f0.elapsed_time(f1) / k2, world, dev)
        e2e = {"value": replica_seconds_per_svd(ems, world), "unit": "s", "h2d_bytes_per_step": int(8 * (2 * n - 1)),
               "d2h_bytes_per_step": int(8 * (n + 2 * n * n))}

    # accuracy of the timed result (checkers use torch / cuBLAS, never the library's GEMM)
    acc = None
    if not a.no_check and rank == 0:
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

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peaks, peak_src = load_peaks()
    g = prof["gemm"]
    dominant = max(prof, key=lambda k: prof[k]["ms"])
    if a.prec == "fp64":
        gemm_peak, gemm_unit_src = FP64_DMMA_TFLOPS, "FP64 mma.sync rate from a throughput probe on this GB300"
    else:
        gemm_peak, gemm_unit_src = float(peaks.get("bf16_tflops_sustained", FALLBACK["bf16_tflops_sustained"])), \
            f"bf16_tflops_sustained ({peak_src})"
    achieved = g["work"] / (g["ms"] * 1e-3) / 1e12 if g["ms"] > 0 else 0.0
    roofline = {"bound": "tensor", "achieved": achieved, "peak": gemm_peak, "unit": "TFLOP/s",
                "frac": achieved / gemm_peak if gemm_peak else None, "traffic": None,
                "kernel": "merge products (" + ("DMMA f64" if a.prec == "fp64" else "tcgen05 bf16 slices") + ")",
                "peak_source": gemm_unit_src, "dominant_stage": dominant}
    stages = {k: {"ms_per_step": v["ms"] / a.steps, "launches_per_step": v["launches"] / a.steps,
                  "work_per_step": v["work"] / a.steps} for k, v in prof.items()}
    if prof["secular"].get("roots"):
        stages["secular"]["roots_per_step"] = prof["secular"]["roots"] / a.steps
        stages["secular"]["iters_per_root"] = prof["secular"]["iters"] / prof["secular"]["roots"]
    hbm = float(peaks.get("hbm_gbs", FALLBACK["hbm_gbs"]))
    for k in ("gather", "vectors", "finish", "final"):
        if prof[k]["ms"] > 0:
            stages[k]["GBps"] = prof[k]["work"] / (prof[k]["ms"] * 1e-3) / 1e9
            stages[k]["hbm_frac"] = stages[k]["GBps"] / hbm
    launches = int(sum(v["launches"] for v in prof.values()) / a.steps) * a.steps

    # the root-start comparison: one untimed run with each other start rule
    # (FP64 iterations per root, secular stage time, SVD time)
    root_start = {"mode": a.start, "iters_per_root": stages["secular"].get("iters_per_root"),
                  "secular_ms_per_step": stages["secular"]["ms_per_step"], "mlp_training": train_info}
    for other in ("plain", "analytic", "mlp"):
        if other == a.start or (other == "mlp" and P is None):
            continue
        o_cmp = bdc.make_opts(a.prec, a.leaf, 64, a.slices, seed=other, mlp=P, mixed_min=a.mixed_min)
        bdc.profile_begin()
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        q0.record(st)
        rc = L.bdc_svd_ex(n, bdc._ptr(d), bdc._ptr(e), bdc._ptr(Ut), bdc._ptr(S), bdc._ptr(VTt), n, n,
                          ctypes.byref(o_cmp), bdc._ptr(work), work.numel(), bdc._ptr(info),
                          ctypes.c_void_p(st.cuda_stream))
        q1.record(st)
        torch.cuda.synchronize()
        pp = bdc.profile_end()
        if rc == 0 and pp["secular"].get("roots"):
            root_start[other] = {"iters_per_root": pp["secular"]["iters"] / pp["secular"]["roots"],
                                 "secular_ms": pp["secular"]["ms"], "svd_ms": q0.elapsed_time(q1)}

    cpu = None
    if not a.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_oracle(n, a.kind, a.seed)

    flops_model = 8.0 / 3.0 * n ** 3
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
        "config": {"workload": workload_name(a), "n": n, "prec": a.prec, "leaf": a.leaf,
                   "slices": (a.slices or 7) if a.prec == "exact" else None,
                   "l2": "inputs larger than L2 (U, V and workspace > 10 GB per step)",
                   "start": a.start, "fp32_root_start": True, "parallelism": f"replicas x{world}"},
        "gflops_paper_model": flops_model / (ms * 1e-3) / 1e9,
        "status": status,
        "accuracy": acc,
        "roofline": roofline,
        "stages": stages,
        "root_start": root_start,
        "gpu_launches": launches,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
