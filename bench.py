#!/usr/bin/env python3
"""Benchmark of the exact-GP training pass on one GB300 (or N replicas).

One step = one pass of the whole path on one synthetic problem:
feature prep, rank-k pivoted Cholesky, probe vectors, mBCG on
[y | probes] to the stop tolerance, Lanczos log-determinant and the
hyperparameter gradient (gp_logml_and_grad).  Inputs are resident in HBM
when the timed region starts; `e2e` repeats the measurement through the
same C ABI call with the inputs copied from pinned host memory every step.

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

METRIC = "mBCG solve s at N=1M (mixed vs FP32, 1e-4 resid); K̂·V TFLOP/s; p50/p99 ms"
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
PRODUCTS_PER_SOLVE = {"gp1m": 97, "gp256k": 120, "gp64k": 1200, "gp2k": 60}
# DRAM bytes (read + write) per launch of the fused tensor-core K-hat V kernel
# from one ncu capture of the full-size launch (profiles/kmv_tc_gp1m.md,
# profiles/kmv_tc_f16_gp1m.md);
# entries are removed whenever the kernel changes after the capture.
# (split TF32: 16.92 + 1.03 GB and split FP16: 4.41 + 0.48 GB were captured,
# and both kernels' epilogues have changed since.)
KMV_DRAM_BYTES = {}
# TF32 dense tensor peak from the measured BF16 one, by the nominal ratio
# 1.1 / 2.25 PFLOP/s
TF32_PER_BF16 = 1.1 / 2.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gp1m", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="split_f16",
                    choices=["fp32", "split_tf32", "split_f16", "tf32"])
    ap.add_argument("--precond", default="auto", choices=["auto", "sigma", "resid"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    return ap.parse_args()


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
    TF32 form."""
    per = 2.0 * (d + t)
    return 3.0 * per if precision in ("split_tf32", "split_f16") else per


def roofline(precision: str, d: int, t: int, entries_per_s: float, sm_mhz: float, peaks: dict,
             peak_src: str, n_sm: int = 152):
    """Roofline of the fused K-hat V kernel.

    Tensor-core forms: achieved = N^2 x tensor FLOPs per entry / kernel time,
    against the dense peak of the operand type: FP16 runs at the BF16 rate
    (the measured BF16 burst), TF32 at the measured BF16 burst x 1.1/2.25.
    Plain FP32
    form: bound by the FMA/ALU pipes at d + t + 12 FP32 ops per entry on 128
    lanes per SM-clock (derived; no measured FP32 peak)."""
    if precision == "fp32":
        ops = d + t + 12
        achieved = entries_per_s * ops / 1e12
        peak = n_sm * 128 * sm_mhz * 1e6 / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "per_entry": f"{ops} FP32 ops",
                "peak_basis": f"152 SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz (derived)"}
    fl = tensor_flops_per_entry(precision, d, t)
    achieved = entries_per_s * fl / 1e12
    if precision == "split_f16":
        peak = peaks["bf16_tflops"]
        basis = f"FP16 = BF16 burst {peaks['bf16_tflops']} ({peak_src}), same dense rate"
    else:
        peak = peaks["bf16_tflops"] * TF32_PER_BF16
        basis = f"TF32 = BF16 burst {peaks['bf16_tflops']} ({peak_src}) x 1.1/2.25"
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "per_entry": f"{fl:.0f} tensor FLOPs", "peak_basis": basis}


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
            "config": {"workload": f"{args.workload}: N={w.N}, d={w.d}, t=1+{npr}, k={k}, tol={tol}"},
            "cpu_baseline": cb,
            "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- ours ----
def run_ours(args):
    import numpy as np
    import torch

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

    def step(Xd, yd):
        return gp.gp_logml_and_grad(ctx, Xd, theta, yd, n_probes=npr, seed=args.seed, k=k,
                                    tol=tol, max_iter=maxit, precision=prec,
                                    allow_notconv=True, precond=pc)

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    for _ in range(args.warmup):
        r = step(X, y)
    barrier()
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
        results.append(step(X, y))
    ev1.record(stream)
    barrier()
    launches = ctx.launches - l0
    clk = clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    import ctypes
    nprod = ctypes.c_int64()
    kms = ctypes.c_double()
    kfl = ctypes.c_double()
    kel = ctypes.c_double()
    ctx.lib.gp_profile_read(ctx.h, ctypes.byref(nprod), ctypes.byref(kms), ctypes.byref(kfl),
                            ctypes.byref(kel))
    ctx.lib.gp_profile(ctx.h, 0)
    ms_step = max_over_ranks(ms_total / args.steps, dist, "cuda")

    # end to end: host inputs copied in every step, results read back
    e2e = None
    if not args.no_e2e:
        Xd = torch.empty_like(X)
        yd = torch.empty_like(y)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            Xd.copy_(Xh, non_blocking=True)
            yd.copy_(yh, non_blocking=True)
            step(Xd, yd)   # returns host scalars and gradient (synchronises)
        barrier()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, dist, "cuda")
        e2e = {"value": e2e_s / max(world, 1), "unit": "s",
               "h2d_bytes_per_step": int(Xh.numel() * 4 + yh.numel() * 4),
               "d2h_bytes_per_step": int(8 * (w.d + 2 + 3))}

    r = results[-1]
    kmv_ms = kms.value / max(nprod.value, 1)
    ent_s = kel.value / max(nprod.value, 1) / (kmv_ms * 1e-3) if nprod.value else 0.0
    peaks, peak_src = load_peaks()
    sm = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    roof = roofline(args.precision, w.d, t, ent_s, sm, peaks, peak_src)
    roof.update({"traffic": KMV_DRAM_BYTES.get((args.workload, args.precision)),
                 "kernel": "fused K-hat V (kmv_tc_kernel)" if args.precision != "fp32"
                 else "fused K-hat V (kmv_plain_kernel)",
                 "per_launch_ms": kmv_ms, "launches": int(nprod.value),
                 "entries_per_s": ent_s,
                 "gemm_equiv_tflops": ent_s * 2.0 * (w.d + t) / 1e12,
                 "timing": "CUDA events around every K-hat V product on the context stream"})
    if rank != 0:
        return 0
    cb = None
    if not args.no_cpu_baseline:
        cb = cpu_baseline(w, t, r["stats"]["n_kmatmul"])
    value = ms_step / 1e3 / max(world, 1)
    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "split_tf32": "tf32x3/f32", "split_f16": "f16x3/f32",
                  "tf32": "tf32/f32"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: N={w.N}, d={w.d}, t=1+{npr}, k={k}, tol={tol}",
                   "precision": args.precision, "preconditioner": f"rank {k}, {pc_name} form",
                   "step": "prep + pivoted Cholesky + probes + mBCG + Lanczos log-det + gradient",
                   "l2": f"inputs larger than L2 (X {w.X.nbytes / 2**20:.0f} MiB)",
                   "parallelism": f"replicas x{world}"},
        "solve": {"iters_max": r["stats"]["iters_max"], "iters_y": r["stats"]["iters_y"],
                  "kmatmul_per_step": r["stats"]["n_kmatmul"], "relres_y": r["stats"]["relres_y"],
                  "relres_max": r["stats"]["relres_max"], "rc": r["rc"],
                  "kmv_share_of_step": kms.value / ms_total if ms_total else None},
        "roofline": roof, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
