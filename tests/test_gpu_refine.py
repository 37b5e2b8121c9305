"""Mixed-precision iterative refinement (gp_mbcg_refine) against the FP64
oracle, through the C ABI.  The refined solution is judged by what defines
it: the true relative residual ||K-hat Omega - B|| / ||B|| from the oracle's
own FP64 product (tolerance: the requested tol x 2, and always <= 1e-4) and
the dense Cholesky solution (relative error 1e-3)."""
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


def _rhs(w, n_probes, seed):
    rng = np.random.default_rng(seed)
    return np.vstack([w.y, rng.choice([-1.0, 1.0], size=(n_probes, w.N))]).astype(np.float32)


@pytest.mark.parametrize("outer", ["split_tf32", "fp32"])
def test_refine_gp2k(gp, ctx, outer):
    w = make_workload("gp2k")
    X = torch.from_numpy(w.X).cuda()
    th = _theta(gp, w)
    L, _, _ = gp.gp_pivchol(ctx, X, th, 32)
    B = _rhs(w, 15, 3)
    tol = 1e-5
    r = gp.gp_mbcg_refine(ctx, X, th, L, torch.from_numpy(B).cuda(), tol=tol, inner_tol=1e-2,
                          inner_precision=gp.GP_TF32, outer_precision=gp.PRECISIONS[outer])
    assert r["rc"] == 0 and r["outer"] >= 2 and r["inner"] > 0
    assert np.all(r["relres"] < tol)
    Om = r["Omega"].cpu().numpy().T.astype(np.float64)
    res = go.true_relative_residual(w.X, w.lengthscale, 1.0, w.sigma2, Om, B.T)
    assert res.max() <= 2 * tol
    Kh = go.khat_matrix(w.X, w.lengthscale, 1.0, w.sigma2)
    ref = go.cholesky_solve(Kh, B.T.astype(np.float64))
    num = np.linalg.norm(Om - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert num.max() <= 1e-3


def test_refine_clustered_resid_form(gp, ctx):
    """Clustered d = 64 features (the 2^20-row generator at N = 4096) with the
    residual-diagonal preconditioner: single-TF32 inner solves, split-TF32
    outer residuals."""
    w = make_workload("gp256k", N=4096)
    X = torch.from_numpy(w.X).cuda()
    th = _theta(gp, w)
    L, _, _, res_d = gp.gp_pivchol(ctx, X, th, 64, want_resid=True)
    B = _rhs(w, 3, 5)
    r = gp.gp_mbcg_refine(ctx, X, th, L, torch.from_numpy(B).cuda(), tol=1e-4, inner_tol=1e-2,
                          max_iter=3000, resid=res_d)
    assert r["rc"] == 0
    Om = r["Omega"].cpu().numpy().T.astype(np.float64)
    res = go.true_relative_residual(w.X, w.lengthscale, 1.0, w.sigma2, Om, B.T)
    assert res.max() <= 1e-4, res


def test_refine_zero_column_and_notconv(gp, ctx):
    w = make_workload("gp2k", N=500, d=6)
    X = torch.from_numpy(w.X).cuda()
    th = _theta(gp, w)
    B = np.vstack([w.y, np.zeros(w.N)]).astype(np.float32)
    r = gp.gp_mbcg_refine(ctx, X, th, None, torch.from_numpy(B).cuda(), tol=1e-5,
                          inner_tol=1e-2, max_iter=3000)
    Om = r["Omega"].cpu().numpy()
    assert r["rc"] == 0 and np.all(Om[1] == 0.0) and r["relres"][1] == 0.0
    r = gp.gp_mbcg_refine(ctx, X, th, None, torch.from_numpy(B).cuda(), tol=1e-12,
                          inner_tol=1e-1, max_outer=1, max_iter=3000, allow_notconv=True)
    assert r["rc"] == gp.GP_ENOTCONV and r["outer"] == 1


def test_refine_rejects_bad_precision(gp, ctx):
    w = make_workload("gp2k", N=64, d=4)
    X = torch.from_numpy(w.X).cuda()
    B = torch.from_numpy(w.y[None, :].copy()).cuda()
    with pytest.raises(gp.GPError):
        gp.gp_mbcg_refine(ctx, X, _theta(gp, w), None, B, outer_precision=gp.GP_TF32)
