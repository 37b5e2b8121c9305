"""Time the fused K-hat V product alone on a named synthetic workload.

    python -m paper_2109_09817_gb300.kmv_bench --workload gp1m --precision split_tf32

Prints one JSON line per precision: per-product device time (CUDA events on
the launching stream, after warm-up), GEMM-equivalent TFLOP/s 2 N^2 (d + t)
and kernel entries per second.  Used for kernel-level timing and profiling
captures; the training-pass benchmark is bench.py at the repository root.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="gp1m")
    ap.add_argument("--N", type=int, default=None)
    ap.add_argument("--t", type=int, default=16)
    ap.add_argument("--precision", default="split_tf32")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    a = ap.parse_args()
    import torch
    import paper_2109_09817_gb300 as gp
    from synth import make_workload
    w = make_workload(a.workload, N=a.N)
    X = torch.from_numpy(w.X).cuda()
    V = torch.randn(a.t, w.N, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    ctx = gp.Context(0)
    th = gp.Theta(w.lengthscale, w.outputscale, w.sigma2)
    for pname in a.precision.split(","):
        prec = gp.PRECISIONS[pname]
        out = torch.empty_like(V)
        for _ in range(a.warmup):
            gp.gp_kmatmul(ctx, X, th, V, prec, out=out)
        torch.cuda.synchronize()
        ctx.lib.gp_profile(ctx.h, 1)
        for _ in range(a.reps):
            gp.gp_kmatmul(ctx, X, th, V, prec, out=out)
        import ctypes
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        fl = ctypes.c_double()
        el = ctypes.c_double()
        ctx.lib.gp_profile_read(ctx.h, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl),
                                ctypes.byref(el))
        ctx.lib.gp_profile(ctx.h, 0)
        per = ms.value / max(n.value, 1)
        print(json.dumps({"workload": a.workload, "N": w.N, "d": w.d, "t": a.t,
                          "precision": pname, "ms_per_product": per,
                          "tflops_gemm_equiv": fl.value / n.value / (per * 1e-3) / 1e12,
                          "gentries_per_s": el.value / n.value / (per * 1e-3) / 1e9}),
              flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
