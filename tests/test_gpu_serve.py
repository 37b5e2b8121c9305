"""Serving loop (gp_server_*): continuous batching of predict and molecule
requests over resident models and solve requests on their own stream,
through the C ABI.

Each result is checked against the FP64 oracle (predictive mean 1e-4, the
stated tolerance; latent variances from the variance cache 1e-4 absolute;
a molecule's energy and the variance of that sum within 1e-4 of their
scales; a solve's alpha by its true relative residual, 1e-4) and against
the same request served alone (1e-4)."""
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


RANK = 48


def _oracle_cache(w):
    # the server starts its Lanczos cache at K-hat a, which is y up to the
    # fit's 1e-6 tolerance; the oracle starts at y
    Kh = go.khat_matrix(w.X, w.lengthscale, 1.0, w.sigma2)
    R, _ = go.lanczos_variance_cache(Kh, np.asarray(w.y, np.float64), RANK)
    return R


def _molecule_rows(w, n_rows, rng):
    i = rng.choice(len(w.Xtest), size=n_rows, replace=n_rows > len(w.Xtest))
    return w.Xtest[i].astype(np.float32)


@pytest.fixture(scope="module")
def served(gp):
    srv = gp.Server(0, max_batch_rows=8192)
    wa = make_workload("gp2k")
    wb = make_workload("gp2k", N=3000, d=16, seed=9)
    ids = []
    for w in (wa, wb):
        th = gp.Theta(w.lengthscale, w.outputscale, w.sigma2)
        ids.append(srv.add_model(torch.from_numpy(w.X).cuda(), th, torch.from_numpy(w.y).cuda(),
                                 k=32, tol=1e-6, max_iter=2000, var_rank=RANK))
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


def test_predict_variance_from_the_cache(gp, served):
    srv, ws, ids = served
    for w, mid in zip(ws, ids):
        rc, _, (mean, var) = srv.wait(srv.predict(mid, w.Xtest[:200], want_var=True))
        assert rc == 0
        ref = go.cached_variance(w.X, w.Xtest[:200], w.lengthscale, 1.0, _oracle_cache(w))
        np.testing.assert_allclose(var, ref, atol=1e-4)
        _, exact = go.predict(w.X, w.y.astype(np.float64), w.Xtest[:200], w.lengthscale, 1.0, w.sigma2)
        assert np.all(var >= exact - 1e-4)


def test_molecule_energy_matches_oracle(gp, served):
    """E_corr = the sum of a molecule's predictions over both models, and
    the variance of that sum (the two models independent)."""
    srv, (wa, wb), ids = served
    rng = np.random.default_rng(11)
    Ra, Rb = _oracle_cache(wa), _oracle_cache(wb)
    for n_occ in (2, 9, 30):
        Xd = _molecule_rows(wa, n_occ, rng)
        Xo = _molecule_rows(wb, n_occ * (n_occ - 1) // 2, rng)
        rc, lat, (e_mean, e_var) = srv.wait(srv.molecule(ids[0], Xd, ids[1], Xo))
        assert rc == 0 and lat > 0
        ma, va = go.predict_sum(wa.X, wa.y, Xd, wa.lengthscale, 1.0, wa.sigma2)
        mb, vb = go.predict_sum(wb.X, wb.y, Xo, wb.lengthscale, 1.0, wb.sigma2)
        pa, _ = go.predict(wa.X, wa.y, Xd, wa.lengthscale, 1.0, wa.sigma2)
        pb, _ = go.predict(wb.X, wb.y, Xo, wb.lengthscale, 1.0, wb.sigma2)
        assert abs(e_mean - (ma + mb)) <= 1e-4 * (np.abs(pa).sum() + np.abs(pb).sum())
        prior = float(np.sum(go.kernel_matrix(Xd, Xd, wa.lengthscale, 1.0))
                      + np.sum(go.kernel_matrix(Xo, Xo, wb.lengthscale, 1.0)))
        cached = (go.cached_variance_sum(wa.X, Xd, wa.lengthscale, 1.0, Ra)
                  + go.cached_variance_sum(wb.X, Xo, wb.lengthscale, 1.0, Rb))
        assert abs(e_var - cached) <= 1e-4 * prior, (e_var, cached, prior)
        assert e_var >= va + vb - 1e-4 * prior          # the cache bounds from above


def test_mix_equals_alone_and_batches(gp, served):
    srv, ws, ids = served
    rng = np.random.default_rng(21)
    reqs = []
    for i in range(40):
        m = int(rng.integers(1, 600))
        which = i % 2
        rows = rng.choice(len(ws[which].Xtest), size=m)
        reqs.append((which, ws[which].Xtest[rows]))
    mols = [(_molecule_rows(ws[0], n, rng), _molecule_rows(ws[1], n * (n - 1) // 2, rng))
            for n in (3, 12, 25, 40)]
    # alone: one request at a time
    alone = []
    for which, xp in reqs:
        rc, _, mean = srv.wait(srv.predict(ids[which], xp))
        assert rc == 0
        alone.append(mean.copy())
    mol_alone = []
    for xd, xo in mols:
        rc, _, e = srv.wait(srv.molecule(ids[0], xd, ids[1], xo))
        assert rc == 0
        mol_alone.append(e)
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
    mol_tk = [srv.molecule(ids[0], xd, ids[1], xo) for xd, xo in mols]
    for t in th_:
        t.join()
    lat = []
    for i, tk in enumerate(tickets):
        rc, ms, mean = srv.wait(tk)
        assert rc == 0
        lat.append(ms)
        assert _rel(mean, alone[i].astype(np.float64)) <= 1e-4, i
    for (e0m, e0v), tk in zip(mol_alone, mol_tk):
        rc, ms, (em, ev) = srv.wait(tk)
        assert rc == 0
        assert abs(em - e0m) <= 1e-4 * max(1.0, abs(e0m)) and abs(ev - e0v) <= 1e-4 * max(1.0, abs(e0v))
    b1 = srv.stats()
    # each molecule is one part per model
    assert b1["predicted"] - b0["predicted"] == len(reqs) + 2 * len(mols)
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
    with pytest.raises(gp.GPError):
        srv.molecule(ids[0], np.zeros((0, ws[0].d), np.float32), ids[1], ws[1].Xtest[:3])
