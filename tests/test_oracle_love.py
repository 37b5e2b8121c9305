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
