"""Serving benchmark: continuous batching over two resident models.

    python -m paper_2109_09817_gb300.serve_bench [--offdiag-n 1048576 --diag-n 65536]

Workload (synthetic stand-in for MOB-ML pair energies, Sec. 2.1): a diagonal
model and an off-diagonal model (d = 64 clustered features, fitted through the
server: split-FP16 mBCG, rank-k residual-diagonal preconditioner, and a
rank-r Lanczos variance cache each).  A molecule request has n_occ ~ U{2..60}
occupied orbitals: its n_occ diagonal and n_occ (n_occ - 1) / 2 off-diagonal
pair features go to the two models in one gp_server_molecule call, which
returns the correlation energy (the sum of the pair predictions) and the
variance of that sum.  A fraction of the requests are
solve requests (a new model's alpha) with N ~ logU[1e3, 2e5] drawn from a pool
of pre-generated problems.

Saturation: the closed-loop predict throughput S_p (molecules/s, all requests
queued at once) and the mean solve time T_s give the mixed rate
lambda_sat = 1 / ((1 - f) / S_p + f T_s) for solve fraction f.  Open-loop runs
then offer Poisson arrivals at the requested fractions of lambda_sat.  Prints
one JSON object with p50/p99 latencies and throughput per rate.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import threading
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _pct(v, q):
    import numpy as np
    return float(np.percentile(np.asarray(v, dtype=np.float64), q)) if len(v) else None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--offdiag-n", type=int, default=1 << 20)
    ap.add_argument("--diag-n", type=int, default=65536)
    ap.add_argument("--k", type=int, default=100)
    ap.add_argument("--var-rank", type=int, default=64)
    ap.add_argument("--precision", default="split_f16")
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--fracs", default="0.5,0.8")
    ap.add_argument("--solve-frac", type=float, default=0.1)
    ap.add_argument("--solve-pool", type=int, default=6)
    ap.add_argument("--solve-nmax", type=int, default=200000)
    ap.add_argument("--max-batch-rows", type=int, default=65536)
    ap.add_argument("--seed", type=int, default=5)
    a = ap.parse_args()

    import numpy as np
    import torch
    import paper_2109_09817_gb300 as gp
    from synth import make_workload

    rng = np.random.default_rng(a.seed)
    out = {"workload": (f"serving: diag N={a.diag_n}, offdiag N={a.offdiag_n}, d=64, "
                        f"n_occ~U{{2..60}}, {a.solve_frac:.0%} solves N~logU[1e3,{a.solve_nmax:.0e}]"),
           "data": "synthetic"}
    srv = gp.Server(0, max_batch_rows=a.max_batch_rows)
    models = []
    for name, n, sd in (("diag", a.diag_n, 51), ("offdiag", a.offdiag_n, 52)):
        w = make_workload("gp1m", N=n, seed=sd)
        th = gp.Theta(w.lengthscale, w.outputscale, w.sigma2)
        t0 = time.perf_counter()
        mid = srv.add_model(torch.from_numpy(w.X).cuda(), th, torch.from_numpy(w.y).cuda(), k=a.k,
                            tol=1e-4, max_iter=400, precision=gp.PRECISIONS[a.precision],
                            var_rank=a.var_rank)
        out[f"fit_{name}_s"] = time.perf_counter() - t0
        models.append((mid, w))
    torch.cuda.synchronize()

    def molecule():
        n = int(rng.integers(2, 61))
        rows = []
        for (mid, w), m in zip(models, (n, n * (n - 1) // 2)):
            idx = rng.integers(0, w.N, size=m)
            xp = w.X[idx] + rng.normal(0.0, 0.05, size=(m, w.d)).astype(np.float32)
            rows.append(xp.astype(np.float32))
        return n, rows

    def submit_molecule(rows):
        return srv.molecule(models[0][0], rows[0], models[1][0], rows[1])

    # solve pool: log-uniform sizes
    sizes = np.exp(rng.uniform(np.log(1e3), np.log(a.solve_nmax), size=a.solve_pool)).astype(int)
    pool = []
    for i, n in enumerate(sizes):
        w = make_workload("gp1m", N=int(n), seed=200 + i)
        pool.append((w, gp.Theta(w.lengthscale, w.outputscale, w.sigma2)))

    # closed-loop predict saturation
    mols = [molecule() for _ in range(200)]
    t0 = time.perf_counter()
    tks = [submit_molecule(rows) for _, rows in mols]
    for tk in tks:
        assert srv.wait(tk)[0] == 0
    sp = len(mols) / (time.perf_counter() - t0)
    pairs = sum(n + n * (n - 1) // 2 for n, _ in mols)
    out["predict_saturation_molecules_per_s"] = sp
    out["predict_saturation_pairs_per_s"] = pairs / (time.perf_counter() - t0)
    # mean solve time, closed loop
    ts = []
    for w, th in pool:
        t1 = time.perf_counter()
        tk = srv.solve(w.X, th, w.y, k=min(a.k, w.N), tol=1e-4, max_iter=400)
        rc, _, _ = srv.wait(tk)
        ts.append(time.perf_counter() - t1)
    tsolve = float(np.mean(ts))
    out["solve_pool_sizes"] = [int(s) for s in sizes]
    out["solve_mean_s"] = tsolve
    f = a.solve_frac
    lam_sat = 1.0 / ((1 - f) / sp + f * tsolve)
    out["lambda_sat_req_per_s"] = lam_sat

    runs = []
    for frac in [float(x) for x in a.fracs.split(",")]:
        lam = frac * lam_sat
        n_req = a.requests
        kinds = rng.random(n_req) < f
        gaps = rng.exponential(1.0 / lam, size=n_req)
        items = []
        for i in range(n_req):
            if kinds[i]:
                items.append(("solve", pool[int(rng.integers(0, len(pool)))]))
            else:
                items.append(("mol", molecule()))
        mol_lat, solve_lat, served_pairs, failed = [], [], 0, []
        pending = []
        lock = threading.Lock()
        b0 = srv.stats()

        def waiter():
            while True:
                with lock:
                    item = pending.pop(0) if pending else None
                if item is None:
                    if done_submitting.is_set():
                        with lock:
                            if not pending:
                                return
                    time.sleep(0.0005)
                    continue
                kind, tks, n = item
                lats, bad = [], False
                for t in tks:
                    rc, ms, _ = srv.wait(t)
                    bad = bad or rc != 0
                    lats.append(ms)
                if bad:
                    failed.append(kind)
                else:
                    (solve_lat if kind == "solve" else mol_lat).append(max(lats))

        done_submitting = threading.Event()
        wt = threading.Thread(target=waiter)
        wt.start()
        t_start = time.perf_counter()
        t_next = t_start
        for i, (kind, payload) in enumerate(items):
            t_next += gaps[i]
            dt = t_next - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            if kind == "solve":
                w, th = payload
                tks = [srv.solve(w.X, th, w.y, k=min(a.k, w.N), tol=1e-4, max_iter=400)]
                n = 0
            else:
                n, rows = payload
                tks = [submit_molecule(rows)]
                served_pairs += n + n * (n - 1) // 2
            with lock:
                pending.append((kind, tks, n))
        done_submitting.set()
        wt.join()
        el = time.perf_counter() - t_start
        b1 = srv.stats()
        runs.append({"load_frac": frac, "offered_req_per_s": lam, "requests": n_req,
                     "elapsed_s": el, "molecules_per_s": len(mol_lat) / el,
                     "pairs_per_s": served_pairs / el,
                     "molecule_p50_ms": _pct(mol_lat, 50), "molecule_p99_ms": _pct(mol_lat, 99),
                     "solve_p50_ms": _pct(solve_lat, 50), "solve_p99_ms": _pct(solve_lat, 99),
                     "solves": len(solve_lat), "failed_requests": len(failed),
                     "predict_batches": b1["batches"] - b0["batches"],
                     "predict_requests": b1["predicted"] - b0["predicted"]})
    out["runs"] = runs
    srv.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
