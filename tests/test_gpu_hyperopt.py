"""Hyperparameter optimisation on a random subset (Sec. 4), through the C
ABI (GPU): gp_hyperopt ascends the log marginal likelihood, and its
gradient at the final theta matches the oracle's (the same-probe estimator
to 1e-3 of the largest component, the exact gradient to 2e-2: the
estimator's own error on this workload is 0.2-0.6 %); gp_train then fits
all rows with sigma^2 + sigma2_add."""
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


@pytest.mark.parametrize("prec", ["split_tf32", "split_f16"])
def test_hyperopt_ascends_and_gradient_matches_oracle(gp, ctx, prec):
    w = make_workload("gp2k")
    X = torch.from_numpy(w.X).cuda()
    y = torch.from_numpy(w.y).cuda()
    theta0 = gp.Theta(w.lengthscale * 1.6, 0.7, 3e-4)
    subset, seed, steps, npr, k = 1024, 17, 5, 15, 32
    th, hist, grad = gp.gp_hyperopt(ctx, X, y, theta0, subset, seed=seed, steps=steps, lr=0.05,
                                    n_probes=npr, k=k, precond=gp.GP_PC_RESID, tol=1e-6,
                                    max_iter=2000, precision=gp.PRECISIONS[prec])
    assert np.all(np.diff(hist) > 0), hist
    # the oracle at the returned theta on the same subset and probes
    idx = gp.gp_subset_indices(w.N, subset, seed)
    assert len(np.unique(idx)) == subset and np.all(np.diff(idx) > 0)
    Xs, ys = w.X[idx], w.y[idx].astype(np.float64)
    L, pr, _ = go.pivoted_cholesky(Xs, th.lengthscale, th.outputscale, k)
    rr = go.residual_diagonal(Xs, th.lengthscale, th.outputscale, L, pr)
    Zp = go.probe_vectors(L, th.sigma2, seed ^ 0x5eed, npr, rr)
    g_same = go.same_probe_grad(Xs, ys, th.lengthscale, th.outputscale, th.sigma2, Zp,
                                go.precond_solve(L, th.sigma2, Zp, rr))
    g_exact = go.exact_grad(Xs, ys, th.lengthscale, th.outputscale, th.sigma2)
    assert np.abs(grad - g_same).max() <= 1e-3 * np.abs(g_same).max()
    assert np.abs(grad - g_exact).max() <= 2e-2 * np.abs(g_exact).max()
    # the objective went up on the exact log marginal likelihood as well
    def exact_logml(t):
        Kh = go.khat_matrix(Xs, t.lengthscale, t.outputscale, t.sigma2)
        return go.log_marginal_likelihood(ys @ go.cholesky_solve(Kh, ys), go.exact_logdet(Kh), subset)
    assert exact_logml(th) > exact_logml(theta0)


def test_train_fits_all_rows_with_sigma2_add(gp, ctx):
    w = make_workload("gp2k", N=1500, d=16)
    X = torch.from_numpy(w.X).cuda()
    y = torch.from_numpy(w.y).cuda()
    theta0 = gp.Theta(w.lengthscale * 1.3, 1.0, 2e-4)
    model, th, hist = gp.gp_train(ctx, X, y, theta0, 600, seed=3, steps=3, lr=0.05, k=32,
                                  precond=gp.GP_PC_RESID, tol=1e-6, max_iter=2000,
                                  precision=gp.GP_FP32_SPLIT_TF32, sigma2_add=1e-5)
    assert np.all(np.diff(hist) > 0), hist
    mean, _ = gp.gp_predict(ctx, model, torch.from_numpy(w.Xtest[:256]).cuda())
    ref, _ = go.predict(w.X, w.y.astype(np.float64), w.Xtest[:256], th.lengthscale, th.outputscale,
                        th.sigma2 + 1e-5)
    assert np.linalg.norm(mean.cpu().numpy() - ref) <= 1e-4 * np.linalg.norm(ref)
    model.free()


def test_hyperopt_rejects_bad_arguments(gp, ctx):
    w = make_workload("gp2k", N=100, d=4)
    X = torch.from_numpy(w.X).cuda()
    y = torch.from_numpy(w.y).cuda()
    with pytest.raises(gp.GPError):
        gp.gp_hyperopt(ctx, X, y, gp.Theta(w.lengthscale), 101)       # subset > N
    with pytest.raises(gp.GPError):
        gp.gp_hyperopt(ctx, X, y, gp.Theta(-w.lengthscale), 50)       # lengthscale <= 0
