"""Serving loop (gp_server_*): continuous batching of predict requests over
resident models and solve requests on their own stream, through the C ABI.

Each result is checked against the FP64 oracle (predictive mean 1e-4, the
stated tolerance; a solve's alpha by its true relative residual, 1e-4) and
against the same request served alone (1e-4)."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import gp_oracle as go  # noqa: E402
from synth import make_workload  # noqa: E402


@pytest.fixture(scope="module")
def gp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_09817_gb300 as gp_
    return gp_


@pytest.fixture(scope="module")
def served(gp):
    srv = gp.Server(0, max_batch_rows=8192)
    wa = make_workload("gp2k")
    wb = make_workload("gp2k", N=3000, d=16, seed=9)
    ids = []
    for w in (wa, wb):
        th = gp.Theta(w.lengthscale, w.outputscale, w.sigma2)
        ids.append(srv.add_model(torch.from_numpy(w.X).cuda(), th, torch.from_numpy(w.y).cuda(),
                                 k=32, tol=1e-6, max_iter=2000))
    yield srv, (wa, wb), ids
    srv.close()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def test_predict_alone_matches_oracle(gp, served):
    srv, ws, ids = served
    for w, mid in zip(ws, ids):
        tk = srv.predict(mid, w.Xtest[:300])
        rc, lat, mean = srv.wait(tk)
        assert rc == 0 and lat > 0
        ref, _ = go.predict(w.X, w.y.astype(np.float64), w.Xtest[:300], w.lengthscale, 1.0, w.sigma2)
        assert _rel(mean, ref) <= 1e-4


def test_mix_equals_alone_and_batches(gp, served):
    srv, ws, ids = served
    rng = np.random.default_rng(21)
    reqs = []
    for i in range(40):
        m = int(rng.integers(1, 600))
        which = i % 2
        rows = rng.choice(len(ws[which].Xtest), size=m)
        reqs.append((which, ws[which].Xtest[rows]))
    # alone: one request at a time
    alone = []
    for which, xp in reqs:
        rc, _, mean = srv.wait(srv.predict(ids[which], xp))
        assert rc == 0
        alone.append(mean.copy())
    b0 = srv.stats()
    # mix: all predicts submitted at once from 4 threads, with two solves
    ws_solve = [make_workload("gp2k", N=n, d=8, seed=30 + n) for n in (1500, 2500)]
    solve_tk = []
    for w in ws_solve:
        th = gp.Theta(w.lengthscale, w.outputscale, w.sigma2)
        solve_tk.append(srv.solve(w.X, th, w.y, k=32, tol=1e-5, max_iter=3000))
    tickets = [None] * len(reqs)

    def submit(lo):
        for i in range(lo, len(reqs), 4):
            which, xp = reqs[i]
            tickets[i] = srv.predict(ids[which], xp)

    th_ = [threading.Thread(target=submit, args=(lo,)) for lo in range(4)]
    for t in th_:
        t.start()
    for t in th_:
        t.join()
    lat = []
    for i, tk in enumerate(tickets):
        rc, ms, mean = srv.wait(tk)
        assert rc == 0
        lat.append(ms)
        assert _rel(mean, alone[i].astype(np.float64)) <= 1e-4, i
    b1 = srv.stats()
    assert b1["predicted"] - b0["predicted"] == len(reqs)
    assert b1["batches"] - b0["batches"] < len(reqs)     # requests were batched
    for w, tk in zip(ws_solve, solve_tk):
        rc, ms, alpha = srv.wait(tk)
        assert rc == 0 and ms > 0
        res = go.true_relative_residual(w.X, w.lengthscale, 1.0, w.sigma2,
                                        alpha.astype(np.float64)[:, None], w.y[:, None])
        assert res.max() <= 1e-4


def test_server_rejects_bad_requests(gp, served):
    srv, ws, ids = served
    with pytest.raises(gp.GPError):
        srv.predict(7, ws[0].Xtest[:4])
    with pytest.raises(gp.GPError):
        srv.predict(ids[0], np.zeros((9000, ws[0].d), np.float32))   # above max_batch_rows
