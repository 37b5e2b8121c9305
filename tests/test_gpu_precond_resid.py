"""The diagonal-corrected preconditioner P = L L^T + diag(K - L L^T) + sigma^2 I
(GP_PC_RESID) against the FP64 oracle, through the C ABI.

Same tolerances as test_gpu_parity.py: residual diagonal 1e-9 absolute (FP64
on both sides), solve true residual 1e-4, log-det 1e-3 against the
same-probe target, gradient 1e-3 of the largest component.
"""
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
def ctx(gp):
    c = gp.Context(0)
    yield c
    c.close()


def _theta(gp, w):
    return gp.Theta(w.lengthscale, w.outputscale, w.sigma2)


def test_residual_diagonal_matches_oracle(gp, ctx):
    """diag(K - L L^T) for the pivots the GPU chose: for a fixed ordered
    pivot set P the factor is L = K[:, P] R^{-1} (R^T R = K[P, P]), so the
    expected residual follows from the kernel matrix alone."""
    w = make_workload("gp2k")
    k = 32
    L, piv, rank, res = gp.gp_pivchol(ctx, torch.from_numpy(w.X).cuda(), _theta(gp, w), k,
                                      want_resid=True)
    piv = piv.cpu().numpy()
    assert rank == k and len(set(piv.tolist())) == k
    K = go.kernel_matrix(w.X, w.X, w.lengthscale, 1.0)
    R = np.linalg.cholesky(K[np.ix_(piv, piv)]).T
    Lp = np.linalg.solve(R.T, K[piv, :]).T
    ref = 1.0 - np.sum(Lp ** 2, axis=1)
    got = res.cpu().numpy()
    assert np.all(got[piv] == 0.0)
    ref[piv] = 0.0
    np.testing.assert_allclose(got, ref, atol=1e-9)
    assert got.min() >= 0.0
    # and where the sequences agree, the oracle's own residual diagonal
    Lr, pr, _ = go.pivoted_cholesky(w.X, w.lengthscale, 1.0, k)
    if np.array_equal(pr, piv):
        np.testing.assert_allclose(got, go.residual_diagonal(w.X, w.lengthscale, 1.0, Lr, pr),
                                   atol=1e-9)


def test_mbcg_resid_solves_and_follows_oracle(gp, ctx):
    """Near-duplicate rows: the corrected form converges, with about the
    oracle's number of steps; its true residual is gated at the FP32
    attainable accuracy of this ill-conditioned problem, 2e-4 (see
    test_gpu_parity.py::test_mbcg_iterations_follow_the_oracle)."""
    w = make_workload("gp64k", N=4096)
    X = torch.from_numpy(w.X).cuda()
    th = _theta(gp, w)
    L, piv, rank, res = gp.gp_pivchol(ctx, X, th, 64, want_resid=True)
    B = w.y[None, :].astype(np.float32)
    r = gp.gp_mbcg(ctx, X, th, L, torch.from_numpy(B).cuda(), tol=1e-4, max_iter=2000,
                   resid=res)
    Lr, pr, _ = go.pivoted_cholesky(w.X, w.lengthscale, 1.0, 64)
    rr = go.residual_diagonal(w.X, w.lengthscale, 1.0, Lr, pr)
    Kh = go.khat_matrix(w.X, w.lengthscale, 1.0, w.sigma2)
    ref = go.mbcg(lambda V: Kh @ V, B.T.astype(np.float64),
                  lambda R: go.precond_solve(Lr, w.sigma2, R, rr), 1e-4, 2000)
    assert r["rc"] == 0
    # FP32 products cost steps here: with K-hat rounded to FP32 inside the
    # oracle's own PCG the count goes from 129 to 171 on this workload
    assert abs(int(r["iters"][0]) - int(ref["iters"][0])) <= 0.4 * ref["iters"][0] + 5
    Om = r["Omega"].cpu().numpy().T.astype(np.float64)
    resid = go.true_relative_residual(w.X, w.lengthscale, 1.0, w.sigma2, Om, B.T)
    assert resid.max() <= 2e-4, resid


@pytest.mark.parametrize("prec", ["fp32", "split_tf32"])
def test_logml_and_grad_resid(gp, ctx, prec):
    w = make_workload("gp2k")
    X = torch.from_numpy(w.X).cuda()
    y = torch.from_numpy(w.y).cuda()
    seed, k, npr = 5, 32, 15
    r = gp.gp_logml_and_grad(ctx, X, _theta(gp, w), y, n_probes=npr, seed=seed, k=k,
                             tol=1e-6, max_iter=1000, precision=gp.PRECISIONS[prec],
                             allow_notconv=True, precond=gp.GP_PC_RESID)
    Kh = go.khat_matrix(w.X, w.lengthscale, 1.0, w.sigma2)
    L, pr, _ = go.pivoted_cholesky(w.X, w.lengthscale, 1.0, k)
    rr = go.residual_diagonal(w.X, w.lengthscale, 1.0, L, pr)
    Zp = go.probe_vectors(L, w.sigma2, seed, npr, rr)
    tgt = go.same_probe_logdet_target(Kh, L, w.sigma2, Zp, rr)
    assert abs(r["logdet"] - tgt) <= 1e-3 * abs(tgt)
    yd = w.y.astype(np.float64)
    logml_tgt = go.log_marginal_likelihood(yd @ go.cholesky_solve(Kh, yd), tgt, w.N)
    assert abs(r["logml"] - logml_tgt) <= 1e-3 * abs(logml_tgt)
    g_ref = go.same_probe_grad(w.X, yd, w.lengthscale, 1.0, w.sigma2, Zp,
                               go.precond_solve(L, w.sigma2, Zp, rr))
    assert np.abs(r["grad"] - g_ref).max() <= 1e-3 * np.abs(g_ref).max()


def test_resid_form_needs_fewer_steps_on_near_diagonal_kernel(gp, ctx):
    """Short lengthscales, small noise: K is close to diagonal, the plain
    form's D = sigma^2 I mis-scales every non-pivot row, the corrected form
    does not."""
    w = make_workload("gp2k", N=3000, d=16)
    X = torch.from_numpy(w.X).cuda()
    th = gp.Theta(0.5 * w.lengthscale, 1.0, 1e-4)
    y = torch.from_numpy(w.y).cuda()
    a = gp.gp_logml_and_grad(ctx, X, th, y, n_probes=7, seed=1, k=32, tol=1e-4,
                             max_iter=3000, want_grad=False, precond=gp.GP_PC_SIGMA,
                             allow_notconv=True)
    b = gp.gp_logml_and_grad(ctx, X, th, y, n_probes=7, seed=1, k=32, tol=1e-4,
                             max_iter=3000, want_grad=False, precond=gp.GP_PC_RESID)
    assert b["stats"]["iters_max"] < a["stats"]["iters_max"]
    ell = 0.5 * w.lengthscale
    Kh = go.khat_matrix(w.X, ell, 1.0, 1e-4)
    L, pr, _ = go.pivoted_cholesky(w.X, ell, 1.0, 32)
    rr = go.residual_diagonal(w.X, ell, 1.0, L, pr)
    for r, res in ((a, None), (b, rr)):
        Zp = go.probe_vectors(L, 1e-4, 1, 7, res)
        tgt = go.same_probe_logdet_target(Kh, L, 1e-4, Zp, res)
        assert abs(r["logdet"] - tgt) <= 1e-3 * abs(tgt)


def test_model_predict_resid(gp, ctx):
    w = make_workload("gp2k")
    X = torch.from_numpy(w.X).cuda()
    y = torch.from_numpy(w.y).cuda()
    m = gp.gp_model_fit(ctx, X, _theta(gp, w), y, k=32, tol=1e-6, precond=gp.GP_PC_RESID)
    mean, var = gp.gp_predict(ctx, m, torch.from_numpy(w.Xtest).cuda(), gp.GP_VAR_EXACT)
    mr, vr = go.predict(w.X, w.y.astype(np.float64), w.Xtest, w.lengthscale, 1.0, w.sigma2)
    assert np.linalg.norm(mean.cpu().numpy() - mr) <= 1e-4 * np.linalg.norm(mr)
    np.testing.assert_allclose(var.cpu().numpy(), vr, atol=1e-4)
    m.free()


def test_invalid_precond_form(gp, ctx):
    w = make_workload("gp2k", N=64, d=4)
    X = torch.from_numpy(w.X).cuda()
    y = torch.from_numpy(w.y).cuda()
    with pytest.raises(gp.GPError):
        gp.gp_logml_and_grad(ctx, X, _theta(gp, w), y, n_probes=2, k=4, precond=7)
