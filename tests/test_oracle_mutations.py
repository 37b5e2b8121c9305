"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in an oracle function (on the CPU, by replacing
the function for the duration of the test) and runs the pin that should
catch it; the pin must fail.  This shows that the pins constrain the oracle
rather than restating it.
"""
import numpy as np
import pytest

from oracle import gp_oracle as go

import test_oracle_bcg as pins_bcg
import test_oracle_grad_predict as pins_grad
import test_oracle_kernel as pins_kernel
import test_oracle_love as pins_love
import test_oracle_solve as pins_solve

SQRT5 = np.sqrt(5.0)


def _matern_wrong_quadratic(r2, s):
    # 5 r^2 / 2 where the Matern 5/2 kernel has 5 r^2 / 3
    r = np.sqrt(np.asarray(r2, np.float64))
    return s * (1.0 + SQRT5 * r + 2.5 * r * r) * np.exp(-SQRT5 * r)


def _grad_full_trace(X, y, ell, s, sig2):
    # the trace term without its factor 1/2
    Kh = go.khat_matrix(X, ell, s, sig2)
    a = np.linalg.solve(Kh, np.asarray(y, np.float64))
    Kinv = np.linalg.inv(Kh)
    return np.array([0.5 * a @ M @ a - np.trace(Kinv @ M) for M in go.dkhat_dtheta(X, ell, s)])


def _mutants():
    orig_khat = go.khat_matmul
    orig_psolve = go.precond_solve
    orig_tri = go.lanczos_tridiagonal
    orig_piv = go.pivoted_cholesky
    orig_cache = go.lanczos_variance_cache
    orig_trr = go.true_relative_residual

    def khat_no_noise(X, V, ell, s, sig2):
        return orig_khat(X, V, ell, s, 0.0)

    def psolve_sign(L, sig2, V, resid=None):
        # Woodbury correction added instead of subtracted
        if resid is not None:
            return orig_psolve(L, sig2, V, resid)
        return 2.0 * np.asarray(V, np.float64) / sig2 - orig_psolve(L, sig2, V)

    def tri_no_sqrt(alpha, beta, m=None):
        dg, of = orig_tri(alpha, beta, m)
        return dg, of * of

    def piv_reversed(X, ell, s, k, stop_rel=1e-12):
        L, piv, gaps = orig_piv(X, ell, s, k, stop_rel)
        return L, piv[::-1].copy(), gaps

    def cache_untransposed(Khat, b, m):
        R, T = orig_cache(Khat, b, m)
        C = np.linalg.cholesky(T)
        Q = R @ C.T
        return Q @ np.linalg.inv(C), T          # Q C^{-1} instead of Q C^{-T}

    def trr_no_noise(X, ell, s, sig2, Omega, B, rows=None):
        return orig_trr(X, ell, s, 0.0, Omega, B, rows)

    orig_sym = go.sym_precond_factor
    orig_pred = go.predict

    def sym_wrong_root(L, sig2, resid=None):
        # (1 + lam)^{-1} - 1 in place of (1 + lam)^{-1/2} - 1: the factor of
        # P^{-1} itself instead of its square root
        dh, Lt, Cp = orig_sym(L, sig2, resid)
        lam, V = np.linalg.eigh(Lt.T @ Lt)
        lam = np.maximum(lam, 0.0)
        return dh, Lt, (V * (-1.0 / (1.0 + lam))) @ V.T

    def signs_low_bit(seed, counters):
        # the sign taken from the lowest output bit instead of the highest
        with np.errstate(over="ignore"):
            c = np.asarray(counters, dtype=np.uint64)
            z = np.uint64(seed) + (c + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        return np.where((z & np.uint64(1)) == 0, 1.0, -1.0)

    def predict_no_prior(X, y, Xp, ell, s, sig2, observation_noise=False):
        # Eq. (pred) read literally, without the prior term k(x', x')
        mean, var = orig_pred(X, y, Xp, ell, s, sig2, observation_noise)
        return mean, var - s

    orig_psum = go.predict_sum

    def psum_no_cross(X, y, Xp, ell, s, sig2):
        # the variance of the sum taken as the sum of the pointwise variances
        mean, _ = orig_psum(X, y, Xp, ell, s, sig2)
        _, var = orig_pred(X, y, Xp, ell, s, sig2)
        return mean, float(np.sum(var))

    return [
        ("predict_sum", psum_no_cross, pins_love.test_predict_sum_is_the_sum_of_the_joint_posterior),
        ("matern52_of_r2", _matern_wrong_quadratic, pins_kernel.test_matern52_equals_bessel_family),
        ("khat_matmul", khat_no_noise, pins_kernel.test_khat_products_vs_brute_force),
        ("true_relative_residual", trr_no_noise, pins_kernel.test_true_relative_residual_vs_brute_force),
        ("precond_solve", psolve_sign, pins_solve.test_woodbury_and_logdet_vs_dense),
        ("lanczos_tridiagonal", tri_no_sqrt, pins_solve.test_cg_tridiagonal_equals_explicit_lanczos),
        ("pivoted_cholesky", piv_reversed, pins_solve.test_pivchol_matches_lapack_dpstrf),
        ("exact_grad", _grad_full_trace, pins_grad.test_exact_grad_vs_logspace_central_fd),
        ("lanczos_variance_cache", cache_untransposed, pins_love.test_full_basis_gives_exact_variance),
        ("sym_precond_factor", sym_wrong_root, pins_bcg.test_sym_factor_is_inverse_square_root),
        ("splitmix64_signs", signs_low_bit, pins_solve.test_splitmix64_published_outputs),
        ("predict", predict_no_prior, pins_grad.test_predict_interpolates_and_bounds),
    ]


@pytest.mark.parametrize("case", range(len(_mutants())))
def test_pin_catches_planted_mistake(monkeypatch, case):
    name, mutant, pin = _mutants()[case]
    pin()                                   # the pin holds for the oracle as written
    monkeypatch.setattr(go, name, mutant)
    with pytest.raises(AssertionError):
        pin()
