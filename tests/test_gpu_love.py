"""Serving variances against the FP64 oracle, through the C ABI (GPU):
the Lanczos variance cache (gp_model_variance_cache, gp_predict with
GP_VAR_CACHED) against oracle.lanczos_variance_cache / cached_variance, and
per-molecule sums (gp_predict_sum) against oracle.predict_sum /
cached_variance_sum.

Tolerances: latent variances within 1e-4 absolute (outputscale 1), as for
the exact variance in test_gpu_parity.py; the variance of a sum within 1e-4
of the prior variance of that sum, 1^T K(X',X') 1 (the two terms of the
difference are each of that size); sums of means within 1e-4 of the sum of
their magnitudes.
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


def _fit(gp, ctx, w, precision, k=32):
    X = torch.from_numpy(w.X).cuda()
    y = torch.from_numpy(w.y).cuda()
    th = gp.Theta(w.lengthscale, 1.0, w.sigma2)
    return gp.gp_model_fit(ctx, X, th, y, k=k, tol=1e-6, max_iter=3000, precision=precision), y


@pytest.mark.parametrize("prec,rank", [("fp32", 24), ("split_f16", 48)])
def test_cached_variance_matches_oracle_cache(gp, ctx, prec, rank):
    w = make_workload("gp2k", N=1500, d=16)
    m, y = _fit(gp, ctx, w, gp.PRECISIONS[prec])
    got_rank = gp.gp_model_variance_cache(ctx, m, rank, b=y)
    assert got_rank == rank
    Xp = torch.from_numpy(w.Xtest[:200]).cuda()
    mean, var = gp.gp_predict(ctx, m, Xp, gp.GP_VAR_CACHED)
    Kh = go.khat_matrix(w.X, w.lengthscale, 1.0, w.sigma2)
    R, _ = go.lanczos_variance_cache(Kh, np.asarray(w.y, np.float64), rank)
    ref = go.cached_variance(w.X, w.Xtest[:200], w.lengthscale, 1.0, R)
    np.testing.assert_allclose(var.cpu().numpy(), ref, atol=1e-4)
    # a Galerkin cache never understates the exact variance (beyond rounding)
    _, exact = go.predict(w.X, w.y, w.Xtest[:200], w.lengthscale, 1.0, w.sigma2)
    assert np.all(var.cpu().numpy() >= exact - 1e-4)
    m.free()


def test_cached_variance_full_basis_is_exact(gp, ctx):
    w = make_workload("gp2k", N=96, d=4)
    m, y = _fit(gp, ctx, w, gp.GP_FP32_PLAIN, k=8)
    rank = gp.gp_model_variance_cache(ctx, m, 96, b=y)
    assert 1 <= rank <= 96
    Xp = torch.from_numpy(w.Xtest[:64]).cuda()
    _, var = gp.gp_predict(ctx, m, Xp, gp.GP_VAR_CACHED)
    _, vex = gp.gp_predict(ctx, m, Xp, gp.GP_VAR_EXACT)
    _, ref = go.predict(w.X, w.y, w.Xtest[:64], w.lengthscale, 1.0, w.sigma2)
    np.testing.assert_allclose(vex.cpu().numpy(), ref, atol=1e-4)
    np.testing.assert_allclose(var.cpu().numpy(), ref, atol=2e-4)
    m.free()


def test_cached_variance_needs_a_cache(gp, ctx):
    w = make_workload("gp2k", N=200, d=4)
    m, _ = _fit(gp, ctx, w, gp.GP_FP32_PLAIN, k=8)
    with pytest.raises(gp.GPError) as e:
        gp.gp_predict(ctx, m, torch.from_numpy(w.Xtest[:4]).cuda(), gp.GP_VAR_CACHED)
    assert e.value.code == gp.GP_EINVAL
    with pytest.raises(gp.GPError):
        gp.gp_model_variance_cache(ctx, m, 129)
    m.free()


def _molecule(w, n_occ, rng):
    """One synthetic molecule's pair rows: n_occ diagonal-like rows and
    n_occ (n_occ - 1) / 2 rows near them (features of the same mixture)."""
    i = rng.choice(len(w.Xtest), size=n_occ, replace=False)
    rows = [w.Xtest[i]]
    for a in range(n_occ):
        for b in range(a + 1, n_occ):
            rows.append(0.5 * (w.Xtest[i[a]] + w.Xtest[i[b]])[None, :])
    return np.vstack(rows).astype(np.float32)


@pytest.mark.parametrize("prec", ["fp32", "split_f16"])
def test_predict_sum_matches_oracle(gp, ctx, prec):
    w = make_workload("gp2k", N=1200, d=8)
    m, y = _fit(gp, ctx, w, gp.PRECISIONS[prec])
    rank = gp.gp_model_variance_cache(ctx, m, 64, b=y)
    rng = np.random.default_rng(5)
    Kh = go.khat_matrix(w.X, w.lengthscale, 1.0, w.sigma2)
    R, _ = go.lanczos_variance_cache(Kh, np.asarray(w.y, np.float64), rank)
    for n_occ in (2, 7, 15):
        Xm = _molecule(w, n_occ, rng)
        Xd = torch.from_numpy(Xm).cuda()
        ms_e, vs_e = gp.gp_predict_sum(ctx, m, Xd, gp.GP_VAR_EXACT)
        ms_c, vs_c = gp.gp_predict_sum(ctx, m, Xd, gp.GP_VAR_CACHED)
        mean_ref, var_ref = go.predict_sum(w.X, w.y, Xm, w.lengthscale, 1.0, w.sigma2)
        mp_ref, _ = go.predict(w.X, w.y, Xm, w.lengthscale, 1.0, w.sigma2)
        prior = float(np.sum(go.kernel_matrix(Xm, Xm, w.lengthscale, 1.0)))
        assert abs(ms_e - mean_ref) <= 1e-4 * np.sum(np.abs(mp_ref)), (ms_e, mean_ref)
        assert abs(ms_c - ms_e) <= 1e-6 * max(1.0, np.sum(np.abs(mp_ref)))   # FP64 atomics: order varies
        assert abs(vs_e - var_ref) <= 1e-4 * prior, (vs_e, var_ref, prior)
        cref = go.cached_variance_sum(w.X, Xm, w.lengthscale, 1.0, R)
        assert abs(vs_c - cref) <= 1e-4 * prior, (vs_c, cref, prior)
        # one-row molecules reduce to the pointwise prediction
    x1 = torch.from_numpy(w.Xtest[:1]).cuda()
    m1, v1 = gp.gp_predict_sum(ctx, m, x1, gp.GP_VAR_EXACT)
    mean1, var1 = gp.gp_predict(ctx, m, x1, gp.GP_VAR_EXACT)
    assert abs(m1 - float(mean1.cpu()[0])) <= 1e-6 and abs(v1 - float(var1.cpu()[0])) <= 1e-4
    m.free()
