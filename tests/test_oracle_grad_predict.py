"""Pins for the oracle's derivatives and prediction (CPU only).

* dK-hat/dtheta against central differences of the kernel matrix itself.
* exact dL/dtheta against log-space central differences of Eq. (ll).
* the same-probe gradient estimator equals the exact gradient when the
  probes satisfy Z Z^T / t = P exactly (an algebraic identity).
* prediction: interpolation of y at X' = X for vanishing noise, variance
  bounds 0 <= var <= s, the prior far from the data.
"""
import math

import numpy as np

from oracle import gp_oracle as go


def _data(n=96, d=4, seed=31):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)).astype(np.float32)
    ell = rng.uniform(0.5, 2.0, d)
    y = np.cos(X.astype(np.float64) @ rng.standard_normal(d)) * 0.1
    return X, ell, y


def _logml(X, y, ell, s, sig2):
    Kh = go.khat_matrix(X, ell, s, sig2)
    a = go.cholesky_solve(Kh, y)
    return go.log_marginal_likelihood(y @ a, go.exact_logdet(Kh), len(y))


def test_dkhat_matches_finite_differences_of_K():
    X, ell, _ = _data(n=20)
    s, sig2, h = 1.3, 1e-3, 1e-6
    mats = list(go.dkhat_dtheta(X, ell, s))
    for j in range(len(ell)):
        ep, em = ell.copy(), ell.copy()
        ep[j] += h
        em[j] -= h
        fd = (go.khat_matrix(X, ep, s, sig2) - go.khat_matrix(X, em, s, sig2)) / (2 * h)
        np.testing.assert_allclose(mats[j], fd, atol=1e-8)
    fd = (go.khat_matrix(X, ell, s + h, sig2) - go.khat_matrix(X, ell, s - h, sig2)) / (2 * h)
    np.testing.assert_allclose(mats[-2], fd, atol=1e-8)
    fd = (go.khat_matrix(X, ell, s, sig2 + h) - go.khat_matrix(X, ell, s, sig2 - h)) / (2 * h)
    np.testing.assert_allclose(mats[-1], fd, atol=1e-8)


def test_exact_grad_vs_logspace_central_fd():
    """h = 1e-4 on log(theta) (a natural-space step of 1e-4 on sigma^2 = 1e-4
    would reach sigma^2 = 0)."""
    X, ell, y = _data(n=128, d=4)
    s, sig2, h = 0.9, 1e-3, 1e-4
    g = go.exact_grad(X, y, ell, s, sig2)
    theta = np.concatenate([ell, [s, sig2]])

    def L(th):
        return _logml(X, y, th[:-2], th[-2], th[-1])

    for i in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[i] *= math.exp(h)
        tm[i] *= math.exp(-h)
        fd_log = (L(tp) - L(tm)) / (2 * h)       # dL/dlog(theta_i)
        assert abs(fd_log - theta[i] * g[i]) <= 1e-5 * max(1.0, abs(fd_log)), i


def test_same_probe_grad_is_exact_for_exact_probe_covariance():
    X, ell, y = _data(n=64, d=3, seed=32)
    s, sig2 = 1.0, 1e-2
    N = len(y)
    L, _, _ = go.pivoted_cholesky(X, ell, s, 8)
    P = L @ L.T + sig2 * np.eye(N)
    lp, Qp = np.linalg.eigh(P)
    Phalf = (Qp * np.sqrt(lp)) @ Qp.T
    Q, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((N, N)))
    Zp = Phalf @ Q * math.sqrt(N)                 # Z Z^T / N = P
    g = go.same_probe_grad(X, y, ell, s, sig2, Zp, go.precond_solve(L, sig2, Zp))
    np.testing.assert_allclose(g, go.exact_grad(X, y, ell, s, sig2),
                               rtol=1e-8, atol=1e-9)


def test_predict_interpolates_and_bounds():
    X, ell, y = _data(n=80, d=3, seed=33)
    s = 1.2
    mean, var = go.predict(X, y, X, ell, s, 1e-10)
    np.testing.assert_allclose(mean, y, atol=1e-6)
    assert np.all(var > -1e-8) and np.all(var < 1e-6)
    rng = np.random.default_rng(1)
    Xp = rng.standard_normal((40, 3)).astype(np.float32)
    mean, var = go.predict(X, y, Xp, ell, s, 1e-3)
    assert np.all(var >= -1e-12) and np.all(var <= s + 1e-12)
    far = Xp + 1e3
    mean, var = go.predict(X, y, far, ell, s, 1e-3)
    np.testing.assert_allclose(mean, 0.0, atol=1e-12)
    np.testing.assert_allclose(var, s, rtol=1e-12)
    _, var_obs = go.predict(X, y, far, ell, s, 1e-3, observation_noise=True)
    np.testing.assert_allclose(var_obs, s + 1e-3, rtol=1e-12)
