"""Pins of the oracle's Lanczos variance cache (the low-rank cache of
Pleiss et al., 2018), against facts that do not depend on it: with a full
Krylov basis Q T^{-1} Q^T is K-hat^{-1}, so the cached variance equals the
exact posterior variance (Cholesky); with fewer steps it is a Galerkin
approximation, which never overstates k^T K-hat^{-1} k, so the cached
variance bounds the exact one from above and tightens as steps are added;
and its T is the CG/Lanczos tridiagonal of unpreconditioned CG on b."""
import numpy as np

from oracle import gp_oracle as go
from synth import make_workload


def _problem(N=48, d=3, M=20):
    w = make_workload("gp2k", N=N, d=d)
    Xp = w.Xtest[:M]
    Kh = go.khat_matrix(w.X, w.lengthscale, 1.0, 1e-2)
    return w, Xp, Kh


def test_full_basis_gives_exact_variance():
    w, Xp, Kh = _problem()
    rng = np.random.default_rng(0)
    R, T = go.lanczos_variance_cache(Kh, rng.standard_normal(w.N), w.N)
    assert R.shape[1] == w.N
    var = go.cached_variance(w.X, Xp, w.lengthscale, 1.0, R)
    _, exact = go.predict(w.X, w.y, Xp, w.lengthscale, 1.0, 1e-2)
    assert np.max(np.abs(var - exact)) <= 1e-8


def test_partial_basis_bounds_from_above_and_tightens():
    w, Xp, Kh = _problem()
    _, exact = go.predict(w.X, w.y, Xp, w.lengthscale, 1.0, 1e-2)
    prev = None
    for m in (4, 8, 16, 32):
        R, _ = go.lanczos_variance_cache(Kh, np.asarray(w.y, np.float64), m)
        var = go.cached_variance(w.X, Xp, w.lengthscale, 1.0, R)
        assert np.all(var >= exact - 1e-12)
        if prev is not None:
            assert np.all(var <= prev + 1e-12)
        prev = var


def test_cache_tridiagonal_is_the_cg_lanczos_matrix():
    w, _, Kh = _problem()
    b = np.asarray(w.y, np.float64)[:, None]
    m = 10
    res = go.mbcg(lambda V: Kh @ V, b, lambda V: V, 1e-14, m)
    dg, of = go.lanczos_tridiagonal(res["alpha"][0], res["beta"][0], m)
    _, T = go.lanczos_variance_cache(Kh, b[:, 0], m)
    assert np.allclose(np.diag(T), dg, rtol=1e-8, atol=0)
    assert np.allclose(np.abs(np.diag(T, 1)), of, rtol=1e-8, atol=0)


# ------------------------------------------------------ per-molecule sums ----
def _joint_conditional(X, y, Xp, ell, s, sigma2):
    """The posterior of f(X') by conditioning the joint Gaussian of
    (y, f(X')) through one block Cholesky factorisation of its covariance
    [[K-hat, K(X,X')], [K(X',X), K(X',X')]]: with J = C C^T, the posterior
    covariance is C22 C22^T and the posterior mean C21 C11^{-1} y."""
    n = len(X)
    Kh = go.khat_matrix(X, ell, s, sigma2)
    Ks = go.kernel_matrix(X, Xp, ell, s)
    Kss = go.kernel_matrix(Xp, Xp, ell, s)
    J = np.block([[Kh, Ks], [Ks.T, Kss + 1e-12 * np.eye(len(Xp))]])
    C = np.linalg.cholesky(J)
    C11, C21, C22 = C[:n, :n], C[n:, :n], C[n:, n:]
    w = np.linalg.solve(C11, np.asarray(y, np.float64))
    return C21 @ w, C22 @ C22.T


def test_predict_sum_is_the_sum_of_the_joint_posterior():
    w = make_workload("gp2k", N=60, d=3)
    Xp = np.vstack([w.Xtest[:5], w.Xtest[:2] + 1e-2])   # correlated rows
    mean, var = go.predict_sum(w.X, w.y, Xp, w.lengthscale, 1.0, 1e-2)
    mu, cov = _joint_conditional(w.X, w.y, Xp, w.lengthscale, 1.0, 1e-2)
    assert abs(mean - mu.sum()) <= 1e-9 * max(1.0, abs(mu.sum()))
    assert abs(var - cov.sum()) <= 1e-8 * cov.sum()
    # the cross-covariances matter: the sum of the variances alone differs
    assert abs(np.trace(cov) - cov.sum()) > 1e-3 * cov.sum()


def test_predict_sum_of_one_row_is_the_pointwise_prediction():
    w = make_workload("gp2k", N=50, d=4)
    for i in range(3):
        m1, v1 = go.predict_sum(w.X, w.y, w.Xtest[i:i + 1], w.lengthscale, 1.0, 1e-2)
        mp, vp = go.predict(w.X, w.y, w.Xtest[i:i + 1], w.lengthscale, 1.0, 1e-2)
        assert abs(m1 - mp[0]) <= 1e-10 and abs(v1 - vp[0]) <= 1e-10


def test_cached_variance_sum_full_basis_and_bound():
    w, Xp, Kh = _problem()
    _, exact = go.predict_sum(w.X, w.y, Xp, w.lengthscale, 1.0, 1e-2)
    rng = np.random.default_rng(3)
    R, _ = go.lanczos_variance_cache(Kh, rng.standard_normal(w.N), w.N)
    assert abs(go.cached_variance_sum(w.X, Xp, w.lengthscale, 1.0, R) - exact) <= 1e-7 * abs(exact) + 1e-9
    prev = None
    for m in (4, 8, 16):
        R, _ = go.lanczos_variance_cache(Kh, np.asarray(w.y, np.float64), m)
        v = go.cached_variance_sum(w.X, Xp, w.lengthscale, 1.0, R)
        assert v >= exact - 1e-10
        if prev is not None:
            assert v <= prev + 1e-10
        prev = v
