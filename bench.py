#!/usr/bin/env python3
"""Benchmark of the mBCG solve at N = 2^20 on one GB300 (or N replicas).

One step = one solve of the whole hot path on the synthetic gp1m problem:
feature prep, rank-k pivoted Cholesky, probe vectors, mBCG on [y | probes]
with the y column driven to a verified true relative residual below tol
(GP_STOP_TRUE), and the Lanczos log-determinant (gp_logml_and_grad without
the gradient).  Inputs are resident in HBM when the timed region starts.
Warm-up steps are the same call capped at two CG steps: every kernel of the
step is loaded and every workspace sized, at a fraction of a solve's cost.

Records beside the timed steps (each once, after the timed region):
  e2e          one step through the same C ABI call with HOST arrays
               (GP_HOST): the library copies X and y in from pinned host
               memory and returns the results;
  training     one full pass with the hyperparameter gradient;
  products     one K-hat V product in the plain FP32 form and one in the
               timed precision, same inputs, same process (mixed vs FP32);
  cpu_baseline the FP64 oracle on a bounded row sample, scaled.
Optional records are skipped when the run's wall time would pass a budget,
so that a slow box still prints its line.

Multi-GPU: the path is replicated, not sharded (each rank solves its own
problem; no collective touches the data path), so `scaling` is "weak".

`--impl reference` times the FP64 oracle on the host cores instead (a
bounded row sample of the same workload, scaled to one solve).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "mBCG solve s at N=1M (mixed vs FP32, 1e-4 resid); K\u0302\u00b7V TFLOP/s; p50/p99 ms"
WORKLOADS = {
    # name: (synth recipe, probes, rank, tol, max_iter, preconditioner form)
    # gp1m/gp256k: clustered features with a near-diagonal K, where the
    # residual-diagonal form of the rank-k preconditioner is the one that
    # converges (the sigma^2 I form needs > 400 steps at k = 100)
    "gp1m": ("gp1m", 15, 100, 1e-4, 400, "resid"),
    "gp256k": ("gp256k", 31, 64, 1e-4, 400, "resid"),
    "gp64k": ("gp64k", 31, 64, 1e-4, 1500, "sigma"),
    "gp2k": ("gp2k", 15, 32, 1e-6, 1000, "sigma"),
}
# K-hat products one solve of each workload needs (split forms, seed 0);
# the reference arm scales its per-product oracle time by this count.
PRODUCTS_PER_SOLVE = {"gp1m": 108, "gp256k": 74, "gp64k": 1217, "gp2k": 60}
# DRAM bytes (read + write) per launch of the fused K-hat V kernel from one
# ncu capture of the current kernel, keyed by (workload, precision); an entry
# is removed whenever the kernel changes after its capture.
KMV_DRAM_BYTES = {
    # kmv_sym_kernel<16> at N = 2^20, d = 64, t = 16: 3.344 GB read + 0.669 GB
    # written in one launch (ncu dram__bytes_read.sum / write.sum, 1 pass)
    ("gp1m", "split_f16"): 3344414208 + 668886528,
}
# TF32 dense tensor peak from the measured BF16 one, by the nominal ratio
# 1.1 / 2.25 PFLOP/s
TF32_PER_BF16 = 1.1 / 2.25
# MUFU throughput per SM-clock measured on this GPU (microbenchmarks of
# ex2.approx.ftz.f32 and sqrt.approx.ftz.f32); one of each per kernel entry
MUFU_EX2_PER_CLK_SM = 30.0
MUFU_SQRT_PER_CLK_SM = 15.0
N_SM = 152
# wall-time budget (s) for the whole run; optional records are skipped past it
WALL_BUDGET_S = 1500.0


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gp1m", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="split_f16",
                    choices=["fp32", "split_tf32", "split_f16", "tf32"])
    ap.add_argument("--precond", default="auto", choices=["auto", "sigma", "resid"])
    ap.add_argument("--stop", default="true", choices=["true", "recurrence"],
                    help="stop rule of y's column (verified true residual, or the CG recurrence)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the training-pass and mixed-vs-FP32 product records")
    ap.add_argument("--seed", type=int, default=0)
    return ap.parse_args(argv)


# ---------------------------------------------------------------- clocks ----
class ClockSampler:
    """nvidia-smi SM clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------------------- helpers ----
def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def tensor_flops_per_entry(precision: str, d: int, t: int) -> float:
    """Tensor-pipe work per kernel entry of one K-hat V product: the cross
    term (2d) and the contraction (2t), each as three products in the split
    forms (hi.hi + hi.lo + lo.hi; TF32 or FP16 parts) and one in the single
    TF32 form.  This is pipe work, not the product's algorithmic work."""
    per = 2.0 * (d + t)
    return 3.0 * per if precision in ("split_tf32", "split_f16") else per


def roofline(precision: str, d: int, t: int, n_rows: int, kmv_ms: float, evaluated: float,
             sm_mhz: float, peaks: dict, peak_src: str, n_sm: int = N_SM):
    """Roofline of the fused K-hat V kernel for one product of N = n_rows rows.

    achieved = the algorithmic work 2 N^2 (d + t) (the GEMM-equivalent flops
    of K(X,X) formed from X~ X~^T and contracted with t vectors) / the
    product's CUDA-event time.  Tensor-core forms divide by the sustained
    dense tensor peak of the operand type (FP16 = the measured BF16 rate,
    TF32 = BF16 x 1.1/2.25): the kernel runs inside a step of seconds.  The
    plain FP32 form divides by the FP32 lanes (152 x 128 x clock, derived).

    `sfu`: the kernel's other bound.  Each evaluated kernel entry takes one
    square root and one base-2 exponential on the MUFU pipe; at the measured
    rates (ex2 30, sqrt 15 per SM-clock) an entry costs 1/30 + 1/15 SM-clock,
    so bound_ms = evaluated x 0.1 / (152 x clock).  `evaluated` is N^2 for
    the full tile grid, about N^2 / 2 when the kernel uses K's symmetry.
    `pipe_tflops`: the tensor pipe's own work rate (3 products per split form)
    against the burst peak, a utilisation figure only."""
    s = kmv_ms * 1e-3
    alg = 2.0 * float(n_rows) ** 2 * (d + t)
    achieved = alg / s / 1e12 if s > 0 else 0.0
    clk = sm_mhz * 1e6
    per_entry_clk = 1.0 / MUFU_EX2_PER_CLK_SM + 1.0 / MUFU_SQRT_PER_CLK_SM
    sfu_ms = evaluated * per_entry_clk / (n_sm * clk) * 1e3
    sfu = {"bound_ms": sfu_ms, "frac": sfu_ms / kmv_ms if kmv_ms > 0 else 0.0,
           "evaluated_entries": evaluated,
           "basis": f"2 MUFU per evaluated entry (ex2 {MUFU_EX2_PER_CLK_SM:.0f}, sqrt "
                    f"{MUFU_SQRT_PER_CLK_SM:.0f} per SM-clock, measured), {n_sm} SMs x {sm_mhz:.0f} MHz"}
    if precision == "fp32":
        peak = n_sm * 128 * clk / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "work": "2 N^2 (d + t) per product",
                "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz (derived)", "sfu": sfu}
    if precision == "split_f16":
        peak = peaks["bf16_tflops_sustained"]
        basis = f"FP16 = BF16 sustained {peak} TFLOP/s (of {peak_src}), same dense rate"
        burst = peaks["bf16_tflops"]
    else:
        peak = peaks["bf16_tflops_sustained"] * TF32_PER_BF16
        basis = f"TF32 = BF16 sustained {peaks['bf16_tflops_sustained']} (of {peak_src}) x 1.1/2.25"
        burst = peaks["bf16_tflops"] * TF32_PER_BF16
    pipe = tensor_flops_per_entry(precision, d, t) * evaluated / s / 1e12 if s > 0 else 0.0
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "work": "2 N^2 (d + t) per product", "peak_basis": basis,
            "sfu": sfu, "pipe_tflops": pipe, "pipe_frac_of_burst": pipe / burst}


def cpu_baseline(w, t, n_products, budget_s=12.0):
    """Oracle streamed K-hat V (FP64, OpenMP) on a row sample, scaled to one
    solve of `n_products` products of the full workload."""
    import numpy as np
    from oracle import cbuild
    from oracle import gp_oracle as go
    rng = np.random.default_rng(0)
    V = rng.choice([-1.0, 1.0], size=(w.N, t))
    # per-row cost from a warm 16-row probe, then a sample sized to the budget
    go.khat_matmul_rows(w.X, V, w.lengthscale, 1.0, w.sigma2, np.arange(2))
    probe = np.sort(rng.choice(w.N, size=16, replace=False))
    t0 = time.perf_counter()
    go.khat_matmul_rows(w.X, V, w.lengthscale, 1.0, w.sigma2, probe)
    per_row = (time.perf_counter() - t0) / len(probe)
    nrows = int(max(16, min(8192, w.N, budget_s / max(per_row, 1e-9))))
    rows = np.sort(rng.choice(w.N, size=nrows, replace=False))
    t0 = time.perf_counter()
    go.khat_matmul_rows(w.X, V, w.lengthscale, 1.0, w.sigma2, rows)
    el = time.perf_counter() - t0
    full_product = el * w.N / nrows
    return {"value": full_product * n_products, "unit": "s", "cores": cbuild.c_threads(),
            "kind": "oracle",
            "sample": (f"FP64 streamed K-hat V of {nrows} sampled rows x N={w.N} x t={t} in "
                       f"{el:.1f} s, scaled by N/rows to one product ({full_product:.1f} s) "
                       f"and by {n_products} products per solve")}


# ------------------------------------------------------------ replicas ----
def replica_seed(rank: int):
    """Rank 0 solves the workload's own seeded problem, rank r > 0 the
    problem seeded 100 + r (independent replicas; nothing is exchanged)."""
    return None if rank == 0 else 100 + rank


def max_over_ranks(value: float, dist, device) -> float:
    """Max of a per-rank scalar over all ranks (the slowest rank sets the
    step time); identity without a process group."""
    if dist is None:
        return value
    import torch
    tt = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


# ----------------------------------------------------------- reference ----
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from synth import make_workload
    recipe, npr, k, tol, maxit, _pc = WORKLOADS[args.workload]
    w = make_workload(recipe, seed=None)
    t = 1 + npr
    nprod = PRODUCTS_PER_SOLVE[args.workload]
    steps = []
    cb = None
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(w, t, nprod, budget_s=4.0)
        if i >= args.warmup:
            steps.append(cb["value"])
    val = sum(steps) / len(steps)
    cb["value"] = val
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": val * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "extrapolated": True,
            "config": {"workload": f"{args.workload}: N={w.N}, d={w.d}, t=1+{npr}, k={k}, tol={tol}"},
            "cpu_baseline": cb,
            "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- ours ----
def log(msg):
    print(f"[bench] {msg}", file=sys.stderr, flush=True)


def run_ours(args):
    import ctypes

    import numpy as np
    import torch

    t_start = time.monotonic()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist = dist_
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    import paper_2109_09817_gb300 as gp
    from synth import make_workload

    recipe, npr, k, tol, maxit, pc_name = WORKLOADS[args.workload]
    if args.precond != "auto":
        pc_name = args.precond
    pc = gp.GP_PC_RESID if pc_name == "resid" else gp.GP_PC_SIGMA
    stop = gp.GP_STOP_TRUE if args.stop == "true" else gp.GP_STOP_RECURRENCE
    w = make_workload(recipe, seed=replica_seed(rank))
    t = 1 + npr
    prec = gp.PRECISIONS[args.precision]
    theta = gp.Theta(w.lengthscale, w.outputscale, w.sigma2)
    stream = torch.cuda.current_stream()
    ctx = gp.Context(local, stream)
    Xh = torch.from_numpy(w.X).pin_memory()
    yh = torch.from_numpy(w.y).pin_memory()
    X = Xh.cuda()
    y = yh.cuda()

    def solve(Xd, yd, max_iter=maxit, grad=False):
        return gp.gp_logml_and_grad(ctx, Xd, theta, yd, n_probes=npr, seed=args.seed, k=k,
                                    tol=tol, max_iter=max_iter, precision=prec,
                                    want_grad=grad, allow_notconv=True, precond=pc, stop=stop)

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    # warm-up: the step's call capped at two CG steps
    for _ in range(args.warmup):
        solve(X, y, max_iter=2)
    barrier()
    log(f"warm-up done at {time.monotonic() - t_start:.1f} s")
    ctx.lib.gp_profile(ctx.h, 1)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip()]
    clocks = ClockSampler(ids[local] if local < len(ids) else local)
    clocks.start()
    l0 = ctx.launches
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    results = []
    for _ in range(args.steps):
        results.append(solve(X, y))
    ev1.record(stream)
    barrier()
    launches = ctx.launches - l0
    clk = clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    nprod = ctypes.c_int64()
    kms = ctypes.c_double()
    kfl = ctypes.c_double()
    kel = ctypes.c_double()
    ctx.lib.gp_profile_read(ctx.h, ctypes.byref(nprod), ctypes.byref(kms), ctypes.byref(kfl),
                            ctypes.byref(kel))
    ctx.lib.gp_profile(ctx.h, 0)
    ms_step = max_over_ranks(ms_total / args.steps, dist, "cuda")
    log(f"timed {args.steps} steps: {ms_step / 1e3:.3f} s per solve, "
        f"wall {time.monotonic() - t_start:.1f} s")

    def budget_left(need_s):
        return time.monotonic() - t_start + need_s < WALL_BUDGET_S

    # end to end: the same C ABI call with HOST arrays (GP_HOST: the library
    # copies X and y from pinned host memory inside the call and returns the
    # results to the host), one step
    e2e = None
    if not args.no_e2e and budget_left(1.5 * ms_step / 1e3):
        barrier()
        t0 = time.perf_counter()
        gp.gp_logml_and_grad_host(ctx, Xh, theta, yh, n_probes=npr, seed=args.seed, k=k, tol=tol,
                                  max_iter=maxit, precision=prec, want_grad=False,
                                  allow_notconv=True, precond=pc, stop=stop)
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        e2e = {"value": e2e_s, "unit": "s", "steps": 1,
               "path": "gp_logml_and_grad with GP_HOST (pinned host X and y)",
               "h2d_bytes_per_step": int(Xh.numel() * 4 + yh.numel() * 4),
               "d2h_bytes_per_step": int(8 * 3 + 4 * 8)}

    r = results[-1]
    kmv_ms = kms.value / max(nprod.value, 1)
    peaks, peak_src = load_peaks()
    sm = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    evaluated = kel.value / max(nprod.value, 1)
    roof = roofline(args.precision, w.d, t, w.N, kmv_ms, evaluated, sm, peaks, peak_src)
    roof.update({"traffic": KMV_DRAM_BYTES.get((args.workload, args.precision)),
                 "kernel": "fused K-hat V (kmv_tc_kernel / kmv_sym_kernel)" if args.precision != "fp32"
                 else "fused K-hat V (kmv_plain_kernel)",
                 "per_launch_ms": kmv_ms, "launches": int(nprod.value),
                 "timing": "CUDA events around every K-hat V product on the context stream, "
                           "timed region"})

    # a full training pass (with the gradient), once
    training = None
    if not args.no_extra and budget_left(2.5 * ms_step / 1e3):
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rt = solve(X, y, grad=True)
        e1.record(stream)
        barrier()
        training = {"s": e0.elapsed_time(e1) / 1e3, "logml": rt["logml"],
                    "what": "prep + pivoted Cholesky + probes + mBCG + Lanczos log-det + gradient"}

    # mixed vs plain FP32: one product each, same inputs
    products = None
    if not args.no_extra and args.precision != "fp32" and budget_left(40.0):
        V = torch.from_numpy(np.random.default_rng(1).choice(
            np.array([-1.0, 1.0], np.float32), size=(t, w.N))).cuda()
        times = {}
        for name in (args.precision, "fp32"):
            gp.gp_kmatmul(ctx, X, theta, V, gp.PRECISIONS[name])   # warm (prep, attributes)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gp.gp_kmatmul(ctx, X, theta, V, gp.PRECISIONS[name])
            e1.record(stream)
            barrier()
            times[name] = e0.elapsed_time(e1) / 1e3
        products = {"t": t, "s": times, "fp32_over_mixed": times["fp32"] / times[args.precision],
                    "fp32_solve_s_projected": times["fp32"] * r["stats"]["n_kmatmul"],
                    "note": "gp_kmatmul calls (prep + split + product); the projection is the "
                            "FP32 product time x the products of one mixed solve"}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    cb = None
    if not args.no_cpu_baseline and budget_left(30.0):
        cb = cpu_baseline(w, t, r["stats"]["n_kmatmul"])
    value = ms_step / 1e3
    st = r["stats"]
    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "split_tf32": "tf32x3/f32", "split_f16": "f16x3/f32",
                  "tf32": "tf32/f32"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: N={w.N}, d={w.d}, t=1+{npr}, k={k}, tol={tol}",
                   "precision": args.precision, "preconditioner": f"rank {k}, {pc_name} form",
                   "step": "prep + pivoted Cholesky + probes + mBCG (y to a verified true residual"
                           " < tol) + Lanczos log-det" if stop else
                           "prep + pivoted Cholesky + probes + mBCG + Lanczos log-det",
                   "warmup_step": "the same call capped at 2 CG steps",
                   "l2": f"inputs larger than L2 (X {w.X.nbytes / 2**20:.0f} MiB, "
                         f"X~ split and vectors rewritten every step)",
                   "parallelism": f"replicas x{world}"},
        "solve": {"iters_max": st["iters_max"], "iters_y": st["iters_y"],
                  "kmatmul_per_step": st["n_kmatmul"], "relres_y_recurrence": st["relres_y"],
                  "relres_y_true": st["true_relres_y"], "true_checks": st["true_checks"],
                  "relres_max_recurrence": st["relres_max"], "rc": r["rc"],
                  "logdet": r["logdet"], "logdet_stderr": r["logdet_stderr"],
                  "kmv_share_of_step": kms.value / ms_total if ms_total else None},
        "roofline": roof, "cpu_baseline": cb, "e2e": e2e, "training": training,
        "products": products, "gpu_launches": int(launches), "clocks": clk,
        "wall_s": time.monotonic() - t_start,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    try:
        return run_ours(args)
    except RuntimeError as e:
        # a solver failure (e.g. a breakdown of single-TF32 products on
        # near-duplicate rows) still prints one line, with the reason
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps({"metric": METRIC, "value": None, "unit": "s", "error": str(e)[:300],
                              "config": {"workload": args.workload, "precision": args.precision}}),
                  flush=True)
        return 1


if __name__ == "__main__":
    sys.exit(main())
