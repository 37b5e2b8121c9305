"""Tensor-core (tcgen05) K-hat V against the FP64 oracle, through the C ABI.

Stated tolerances (the FP32-mode gate of 1e-5 applies to GP_FP32_PLAIN and is
tested in test_gpu_parity.py):
* split-TF32 (GP_FP32_SPLIT_TF32): 2e-5.  Its products are exact, but the
  tensor core's FP32 accumulator truncates, and the cross term x_a . x_b is
  accumulated at |x~|^2 ~ 10^2 before the norm expansion cancels it; the
  measured error is 2e-6 (N = 2048) to 1.4e-5 (N = 2^20, rows with ~10^5
  significant neighbours).
* single-pass TF32 (GP_TF32): 1e-2 (~2^-11 relative error in the cross term).
"""
TOL_SPLIT = 2e-5
FORM = "split_tf32"
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import gp_oracle as go  # noqa: E402
from synth import make_workload  # noqa: E402
from _parity import check_kmv, khat_ref, kcross_ref  # noqa: E402


@pytest.fixture(scope="module")
def gp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_09817_gb300 as gp_
    return gp_


@pytest.fixture(scope="module")
def ctx(gp):
    c = gp.Context(0)
    yield c
    c.close()


def _relerr(got, ref):
    num = np.linalg.norm(np.asarray(got, np.float64) - ref, axis=0)
    return float(np.max(num / np.maximum(np.linalg.norm(ref, axis=0), 1e-300)))


def _run(gp, ctx, X, ell, s, sig2, V, prec):
    out = gp.gp_kmatmul(ctx, torch.from_numpy(X).cuda(), gp.Theta(ell, s, sig2),
                        torch.from_numpy(V).cuda(), gp.PRECISIONS[prec])
    ctx.sync()
    return out.cpu().numpy().T


def test_tc_small_first(gp, ctx):
    """Smallest case: one row tile, one column tile."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((64, 32)).astype(np.float32)
    ell = rng.uniform(0.5, 2.0, 32)
    V = rng.standard_normal((16, 64)).astype(np.float32)
    got = _run(gp, ctx, X, ell, 1.0, 1e-4, V, "split_tf32")
    ref, aref = khat_ref(X, V.T, ell, 1.0, 1e-4)
    check_kmv(got, ref, aref, TOL_SPLIT, FORM)


@pytest.mark.parametrize("prec,tol", [("split_tf32", TOL_SPLIT), ("tf32", 1e-2)])
def test_tc_gp2k(gp, ctx, prec, tol):
    w = make_workload("gp2k")
    V = np.random.default_rng(0).standard_normal((16, w.N)).astype(np.float32)
    got = _run(gp, ctx, w.X, w.lengthscale, 1.0, w.sigma2, V, prec)
    ref, aref = khat_ref(w.X, V.T, w.lengthscale, 1.0, w.sigma2)
    check_kmv(got, ref, aref, tol, prec)


@pytest.mark.parametrize("N,d,t", [(1, 3, 1), (129, 5, 3), (257, 33, 17), (1000, 64, 33),
                                   (600, 64, 64), (300, 8, 100), (4100, 20, 16)])
def test_tc_ragged(gp, ctx, N, d, t):
    rng = np.random.default_rng(N * 7 + d + t)
    X = rng.standard_normal((N, d)).astype(np.float32)
    ell = rng.uniform(0.5, 2.0, d)
    V = rng.standard_normal((t, N)).astype(np.float32)
    got = _run(gp, ctx, X, ell, 0.8, 1e-3, V, "split_tf32")
    ref, aref = khat_ref(X, V.T, ell, 0.8, 1e-3)
    check_kmv(got, ref, aref, TOL_SPLIT, FORM)


def test_tc_cross(gp, ctx):
    w = make_workload("gp2k")
    V = np.random.default_rng(2).standard_normal((16, w.N)).astype(np.float32)
    out = gp.gp_kcross_matmul(ctx, torch.from_numpy(w.Xtest).cuda(), torch.from_numpy(w.X).cuda(),
                              gp.Theta(w.lengthscale, 1.0, w.sigma2), torch.from_numpy(V).cuda(),
                              gp.GP_FP32_SPLIT_TF32)
    ref, aref = kcross_ref(w.Xtest, w.X, V.T, w.lengthscale, 1.0)
    check_kmv(out.cpu().numpy().T, ref, aref, TOL_SPLIT, FORM)


@pytest.mark.parametrize("name,t,nrows", [("gp64k", 32, 256), ("gp1m", 16, 48)])
def test_tc_full_size_sampled_rows(gp, ctx, name, t, nrows):
    w = make_workload(name)
    rng = np.random.default_rng(7)
    V = rng.choice([-1.0, 1.0], size=(t, w.N)).astype(np.float32)
    got = _run(gp, ctx, w.X, w.lengthscale, 1.0, w.sigma2, V, "split_tf32")
    rows = np.sort(rng.choice(w.N, size=nrows, replace=False))
    ref, aref = khat_ref(w.X, V.T, w.lengthscale, 1.0, w.sigma2, rows)
    check_kmv(got[rows], ref, aref, TOL_SPLIT, FORM)


def test_tc_matches_plain(gp, ctx):
    """Same product in the two FP32-class forms agree to the tolerance."""
    w = make_workload("gp2k", N=3000, d=64)
    V = np.random.default_rng(4).standard_normal((32, w.N)).astype(np.float32)
    a = _run(gp, ctx, w.X, w.lengthscale, 1.0, w.sigma2, V, "split_tf32")
    b = _run(gp, ctx, w.X, w.lengthscale, 1.0, w.sigma2, V, "fp32")
    assert _relerr(a, b.astype(np.float64)) <= TOL_SPLIT


def test_tc_logml_and_predict(gp, ctx):
    w = make_workload("gp2k")
    X = torch.from_numpy(w.X).cuda()
    y = torch.from_numpy(w.y).cuda()
    th = gp.Theta(w.lengthscale, 1.0, w.sigma2)
    r = gp.gp_logml_and_grad(ctx, X, th, y, n_probes=15, seed=11, k=32, tol=1e-6,
                             precision=gp.GP_FP32_SPLIT_TF32, allow_notconv=True)
    Kh = go.khat_matrix(w.X, w.lengthscale, 1.0, w.sigma2)
    L, _, _ = go.pivoted_cholesky(w.X, w.lengthscale, 1.0, 32)
    Zp = go.probe_vectors(L, w.sigma2, 11, 15)
    tgt = go.same_probe_logdet_target(Kh, L, w.sigma2, Zp)
    assert abs(r["logdet"] - tgt) <= 1e-3 * abs(tgt)
    g_ref = go.same_probe_grad(w.X, w.y.astype(np.float64), w.lengthscale, 1.0, w.sigma2, Zp,
                               go.precond_solve(L, w.sigma2, Zp))
    assert np.abs(r["grad"] - g_ref).max() <= 1e-3 * np.abs(g_ref).max()
    m = gp.gp_model_fit(ctx, X, th, y, k=32, tol=1e-6, precision=gp.GP_FP32_SPLIT_TF32)
    mean, _ = gp.gp_predict(ctx, m, torch.from_numpy(w.Xtest).cuda())
    mr, _ = go.predict(w.X, w.y.astype(np.float64), w.Xtest, w.lengthscale, 1.0, w.sigma2)
    assert np.linalg.norm(mean.cpu().numpy() - mr) <= 1e-4 * np.linalg.norm(mr)
    m.free()


def test_tc_full_size_solve_gp256k(gp, ctx):
    """A solve at full size in the benchmark's configuration (split TF32,
    rank-64 residual-diagonal preconditioner, tol 1e-4): the true relative
    residual of the y column on 1024 rows sampled by the oracle (an estimate
    of the full ratio), gated at 1e-4; the solve verifies its own true
    residual (GP_STOP_TRUE) below 0.8e-4."""
    w = make_workload("gp256k")
    X = torch.from_numpy(w.X).cuda()
    th = gp.Theta(w.lengthscale, 1.0, w.sigma2)
    L, _, _, res_d = gp.gp_pivchol(ctx, X, th, 64, want_resid=True)
    B = w.y[None, :].astype(np.float32)
    r = gp.gp_mbcg(ctx, X, th, L, torch.from_numpy(B).cuda(), tol=1e-4, max_iter=400,
                   precision=gp.GP_FP32_SPLIT_TF32, resid=res_d, allow_notconv=False,
                   stop=gp.GP_STOP_TRUE)
    assert r["rc"] == 0 and r["relres"][0] <= 0.8e-4
    Om = r["Omega"].cpu().numpy().T.astype(np.float64)
    rows = np.sort(np.random.default_rng(8).choice(w.N, size=1024, replace=False))
    res = go.true_relative_residual(w.X, w.lengthscale, 1.0, w.sigma2, Om, B.T, rows)
    assert res.max() <= 1e-4, res


@pytest.mark.parametrize("name,N,d,npr,prec", [("gp2k", 1500, 32, 15, "split_tf32"),
                                              ("gp256k", 1024, 64, 15, "split_tf32"),
                                              ("gp256k", 4096, 64, 31, "split_tf32"),
                                              ("gp256k", 4096, 64, 31, "split_f16")])
def test_tc_backward_matches_oracle(gp, ctx, name, N, d, npr, prec):
    """Tensor-core backward (split TF32, d_pad 32 and 64) against the
    oracle's same-probe gradient, the solve in the pass's precision; at N =
    4096 with 31 probes, the oracle check of the 2^18-row gradient
    configuration (64 lengthscales, s, sigma^2)."""
    w = make_workload(name, N=N, d=d)
    X = torch.from_numpy(w.X).cuda()
    y = torch.from_numpy(w.y).cuda()
    th = gp.Theta(w.lengthscale, 1.0, w.sigma2)
    seed, k = 4, 32
    r = gp.gp_logml_and_grad(ctx, X, th, y, n_probes=npr, seed=seed, k=k, tol=1e-6,
                             max_iter=2000, precision=gp.PRECISIONS[prec],
                             allow_notconv=True, precond=gp.GP_PC_RESID)
    L, pr, _ = go.pivoted_cholesky(w.X, w.lengthscale, 1.0, k)
    rr = go.residual_diagonal(w.X, w.lengthscale, 1.0, L, pr)
    Zp = go.probe_vectors(L, w.sigma2, seed, npr, rr)
    g_ref = go.same_probe_grad(w.X, w.y.astype(np.float64), w.lengthscale, 1.0, w.sigma2, Zp,
                               go.precond_solve(L, w.sigma2, Zp, rr))
    assert np.abs(r["grad"] - g_ref).max() <= 1e-3 * np.abs(g_ref).max()
