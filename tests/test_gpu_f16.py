"""Split-FP16 tensor-core K-hat V (GP_FP32_SPLIT_F16) against the FP64 oracle.

The FP16 form keeps the operand accuracy of the split-TF32 form (hi + lo
carries 22 significant bits of every feature, vector entry and kernel value),
so it is held to the same stated tolerance, 2e-5 (the FP32 accumulator of the
tensor core truncates; see test_gpu_tc.py).  FP16's narrow exponent range is
covered by power-of-two scaling: the tests below also push the features and
the vectors far outside that range, and mix magnitudes inside one vector.
"""
TOL_SPLIT = 2e-5
FORM = "split_f16"
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


def _run(gp, ctx, X, ell, s, sig2, V, prec="split_f16"):
    out = gp.gp_kmatmul(ctx, torch.from_numpy(X).cuda(), gp.Theta(ell, s, sig2),
                        torch.from_numpy(V).cuda(), gp.PRECISIONS[prec])
    ctx.sync()
    return out.cpu().numpy().T


def test_f16_small_first(gp, ctx):
    """Smallest case: one row tile, one column tile."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((64, 32)).astype(np.float32)
    ell = rng.uniform(0.5, 2.0, 32)
    V = rng.standard_normal((16, 64)).astype(np.float32)
    got = _run(gp, ctx, X, ell, 1.0, 1e-4, V)
    ref, aref = khat_ref(X, V.T, ell, 1.0, 1e-4)
    check_kmv(got, ref, aref, TOL_SPLIT, FORM)


def test_f16_gp2k(gp, ctx):
    w = make_workload("gp2k")
    V = np.random.default_rng(0).standard_normal((16, w.N)).astype(np.float32)
    got = _run(gp, ctx, w.X, w.lengthscale, 1.0, w.sigma2, V)
    ref, aref = khat_ref(w.X, V.T, w.lengthscale, 1.0, w.sigma2)
    check_kmv(got, ref, aref, TOL_SPLIT, FORM)


@pytest.mark.parametrize("N,d,t", [(1, 3, 1), (129, 5, 3), (257, 33, 17), (1000, 64, 33),
                                   (600, 64, 64), (300, 8, 100), (4100, 20, 16)])
def test_f16_ragged(gp, ctx, N, d, t):
    rng = np.random.default_rng(N * 7 + d + t)
    X = rng.standard_normal((N, d)).astype(np.float32)
    ell = rng.uniform(0.5, 2.0, d)
    V = rng.standard_normal((t, N)).astype(np.float32)
    got = _run(gp, ctx, X, ell, 0.8, 1e-3, V)
    ref, aref = khat_ref(X, V.T, ell, 0.8, 1e-3)
    check_kmv(got, ref, aref, TOL_SPLIT, FORM)


def test_f16_vector_scales(gp, ctx):
    """Vectors far outside FP16's range, a zero vector, and one vector whose
    entries span 10 decades: each column is scaled on its own."""
    w = make_workload("gp2k", N=1500)
    rng = np.random.default_rng(3)
    V = rng.standard_normal((6, w.N))
    V[0] *= 1e-30
    V[1] *= 1e25
    V[2] = 0.0
    V[3] *= np.exp(rng.uniform(np.log(1e-10), 0.0, w.N))
    V[4] *= 6e4
    V = V.astype(np.float32)
    got = _run(gp, ctx, w.X, w.lengthscale, 1.0, w.sigma2, V)
    ref = go.khat_matmul(w.X, V.T.astype(np.float64), w.lengthscale, 1.0, w.sigma2)
    assert np.all(got[:, 2] == 0.0)
    keep = [0, 1, 3, 4, 5]
    assert _relerr(got[:, keep], ref[:, keep]) <= TOL_SPLIT


@pytest.mark.parametrize("ell_scale", [1e-4, 1e4])
def test_f16_feature_scales(gp, ctx, ell_scale):
    """Prepared features far above FP16's range (lengthscales 1e-4: every
    pair is far apart, K = I) and far below it (lengthscales 1e4: K is close
    to all ones); one power of two scales the whole feature matrix."""
    rng = np.random.default_rng(9)
    N, d = 700, 12
    X = rng.standard_normal((N, d)).astype(np.float32)
    ell = rng.uniform(0.5, 2.0, d) * ell_scale
    V = rng.standard_normal((8, N)).astype(np.float32)
    got = _run(gp, ctx, X, ell, 1.3, 1e-2, V)
    ref = go.khat_matmul(X, V.T.astype(np.float64), ell, 1.3, 1e-2)
    assert np.all(np.isfinite(got))
    assert _relerr(got, ref) <= TOL_SPLIT


def test_f16_duplicates(gp, ctx):
    """Exact and near-duplicate rows: u^2 must cancel to ~0 (norms are taken
    from the same FP16 parts as the cross term)."""
    w = make_workload("gp64k", N=3000)
    V = np.random.default_rng(1).standard_normal((16, w.N)).astype(np.float32)
    X = w.X.copy()
    X[1::7] = X[0::7][: len(X[1::7])]
    got = _run(gp, ctx, X, w.lengthscale, 1.0, w.sigma2, V)
    ref, aref = khat_ref(X, V.T, w.lengthscale, 1.0, w.sigma2)
    check_kmv(got, ref, aref, TOL_SPLIT, FORM)


def test_f16_cross(gp, ctx):
    w = make_workload("gp2k")
    V = np.random.default_rng(2).standard_normal((16, w.N)).astype(np.float32)
    out = gp.gp_kcross_matmul(ctx, torch.from_numpy(w.Xtest).cuda(), torch.from_numpy(w.X).cuda(),
                              gp.Theta(w.lengthscale, 1.0, w.sigma2), torch.from_numpy(V).cuda(),
                              gp.GP_FP32_SPLIT_F16)
    ref, aref = kcross_ref(w.Xtest, w.X, V.T, w.lengthscale, 1.0)
    check_kmv(out.cpu().numpy().T, ref, aref, TOL_SPLIT, FORM)


@pytest.mark.parametrize("name,t,nrows", [("gp64k", 32, 256), ("gp1m", 16, 48)])
def test_f16_full_size_sampled_rows(gp, ctx, name, t, nrows):
    w = make_workload(name)
    rng = np.random.default_rng(7)
    V = rng.choice([-1.0, 1.0], size=(t, w.N)).astype(np.float32)
    got = _run(gp, ctx, w.X, w.lengthscale, 1.0, w.sigma2, V)
    rows = np.sort(rng.choice(w.N, size=nrows, replace=False))
    ref, aref = khat_ref(w.X, V.T, w.lengthscale, 1.0, w.sigma2, rows)
    check_kmv(got[rows], ref, aref, TOL_SPLIT, FORM)


@pytest.mark.parametrize("name,N,t", [("gp256k", 4100, 16), ("gp64k", 2000, 32), ("gp2k", 700, 5),
                                      ("gp2k", 129, 1)])
def test_f16_symmetric_matches_full_grid(gp, ctx, name, N, t):
    """The symmetric kernel (the tiles at and right of the diagonal blocks,
    each contracted twice) against the full-grid kernel (every tile formed
    once; GP_OPT_SYMMETRIC_KMV = 0) on the same product, both against the
    oracle."""
    from paper_2109_09817_gb300 import _lib
    w = make_workload(name, N=N)
    V = np.random.default_rng(N + t).standard_normal((t, w.N)).astype(np.float32)
    th = gp.Theta(w.lengthscale, 1.0, w.sigma2)
    Xd = torch.from_numpy(w.X).cuda()
    Vd = torch.from_numpy(V).cuda()
    sym = gp.gp_kmatmul(ctx, Xd, th, Vd, gp.GP_FP32_SPLIT_F16).cpu().numpy().T
    ctx.set_option(_lib.GP_OPT_SYMMETRIC_KMV, 0)
    try:
        full = gp.gp_kmatmul(ctx, Xd, th, Vd, gp.GP_FP32_SPLIT_F16).cpu().numpy().T
    finally:
        ctx.set_option(_lib.GP_OPT_SYMMETRIC_KMV, 1)
    ref, aref = khat_ref(w.X, V.T, w.lengthscale, 1.0, w.sigma2)
    ce_s, er_s = check_kmv(sym, ref, aref, TOL_SPLIT, FORM)
    ce_f, er_f = check_kmv(full, ref, aref, TOL_SPLIT, FORM)
    assert _relerr(sym, full.astype(np.float64)) <= TOL_SPLIT


def test_f16_matches_split_tf32(gp, ctx):
    w = make_workload("gp2k", N=3000, d=64)
    V = np.random.default_rng(4).standard_normal((32, w.N)).astype(np.float32)
    a = _run(gp, ctx, w.X, w.lengthscale, 1.0, w.sigma2, V, "split_f16")
    b = _run(gp, ctx, w.X, w.lengthscale, 1.0, w.sigma2, V, "split_tf32")
    assert _relerr(a, b.astype(np.float64)) <= TOL_SPLIT


def test_f16_rejects_wide_features(gp, ctx):
    rng = np.random.default_rng(0)
    X = torch.from_numpy(rng.standard_normal((100, 65)).astype(np.float32)).cuda()
    V = torch.ones(1, 100, device="cuda")
    with pytest.raises(gp.GPError) as e:
        gp.gp_kmatmul(ctx, X, gp.Theta(np.ones(65), 1.0, 1e-3), V, gp.GP_FP32_SPLIT_F16)
    assert e.value.code == gp.GP_EINVAL


def test_f16_logml_and_predict(gp, ctx):
    w = make_workload("gp2k")
    X = torch.from_numpy(w.X).cuda()
    y = torch.from_numpy(w.y).cuda()
    th = gp.Theta(w.lengthscale, 1.0, w.sigma2)
    r = gp.gp_logml_and_grad(ctx, X, th, y, n_probes=15, seed=11, k=32, tol=1e-6,
                             precision=gp.GP_FP32_SPLIT_F16, allow_notconv=True)
    Kh = go.khat_matrix(w.X, w.lengthscale, 1.0, w.sigma2)
    L, _, _ = go.pivoted_cholesky(w.X, w.lengthscale, 1.0, 32)
    Zp = go.probe_vectors(L, w.sigma2, 11, 15)
    tgt = go.same_probe_logdet_target(Kh, L, w.sigma2, Zp)
    assert abs(r["logdet"] - tgt) <= 1e-3 * abs(tgt)
    g_ref = go.same_probe_grad(w.X, w.y.astype(np.float64), w.lengthscale, 1.0, w.sigma2, Zp,
                               go.precond_solve(L, w.sigma2, Zp))
    assert np.abs(r["grad"] - g_ref).max() <= 1e-3 * np.abs(g_ref).max()
    m = gp.gp_model_fit(ctx, X, th, y, k=32, tol=1e-6, precision=gp.GP_FP32_SPLIT_F16)
    mean, _ = gp.gp_predict(ctx, m, torch.from_numpy(w.Xtest).cuda())
    mr, _ = go.predict(w.X, w.y.astype(np.float64), w.Xtest, w.lengthscale, 1.0, w.sigma2)
    assert np.linalg.norm(mean.cpu().numpy() - mr) <= 1e-4 * np.linalg.norm(mr)
    m.free()


def test_f16_full_size_solve_gp256k(gp, ctx):
    """Full-size solve in the split-FP16 form (rank-64 residual-diagonal
    preconditioner, tol 1e-4, GP_STOP_TRUE): true relative residual of y on
    1024 rows sampled by the oracle, gated at 1e-4 as for the TF32 form."""
    w = make_workload("gp256k")
    X = torch.from_numpy(w.X).cuda()
    th = gp.Theta(w.lengthscale, 1.0, w.sigma2)
    L, _, _, res_d = gp.gp_pivchol(ctx, X, th, 64, want_resid=True)
    B = w.y[None, :].astype(np.float32)
    r = gp.gp_mbcg(ctx, X, th, L, torch.from_numpy(B).cuda(), tol=1e-4, max_iter=400,
                   precision=gp.GP_FP32_SPLIT_F16, resid=res_d, allow_notconv=False,
                   stop=gp.GP_STOP_TRUE)
    assert r["rc"] == 0 and r["relres"][0] <= 0.8e-4
    Om = r["Omega"].cpu().numpy().T.astype(np.float64)
    rows = np.sort(np.random.default_rng(8).choice(w.N, size=1024, replace=False))
    res = go.true_relative_residual(w.X, w.lengthscale, 1.0, w.sigma2, Om, B.T, rows)
    assert res.max() <= 1e-4, res
