"""Pins for the oracle's solves, preconditioner, mBCG and Lanczos quadrature.

Independent references: LAPACK's pivoted Cholesky (dpstrf), dense inverses
and slogdet, the Krylov-subspace minimisation property that defines CG
iterates, an explicit Lanczos process, matrix logarithms by eigh, and the
published SplitMix64 outputs.
"""
import json
import math
import os

import numpy as np
import scipy.linalg as sla
from scipy.linalg import lapack

from oracle import gp_oracle as go
from synth import make_workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small(n=256, d=6, seed=21, dup=False):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)).astype(np.float32)
    if dup:
        X[n // 2:n // 2 + 8] = X[:8] + 1e-3 * rng.standard_normal((8, d))
    ell = rng.uniform(0.5, 2.0, d)
    y = rng.standard_normal(n) * 1e-2
    return X, ell, y


def test_cholesky_solve_residual():
    X, ell, y = _small()
    Kh = go.khat_matrix(X, ell, 1.0, 1e-4)
    w = go.cholesky_solve(Kh, y)
    assert np.linalg.norm(Kh @ w - y) / np.linalg.norm(y) < 1e-11
    sign, ld = np.linalg.slogdet(Kh)
    assert sign > 0 and abs(go.exact_logdet(Kh) - ld) < 1e-9 * abs(ld)


def test_pivchol_full_rank_reproduces_K():
    X, ell, _ = _small(n=60, d=3)
    K = go.kernel_matrix(X, X, ell, 1.0)
    L, piv, _ = go.pivoted_cholesky(X, ell, 1.0, 60, stop_rel=0.0)
    assert len(piv) == 60 and sorted(piv) == list(range(60))
    assert np.max(np.abs(L @ L.T - K)) < 1e-10


def test_pivchol_matches_lapack_dpstrf():
    """LAPACK dpstrf takes, at each step, the largest remaining diagonal of
    the Schur complement (first index on ties): the same greedy rule."""
    X, ell, _ = _small(n=300, d=5, seed=22)
    K = go.kernel_matrix(X, X, ell, 1.0)
    k = 40
    L, piv, gaps = go.pivoted_cholesky(X, ell, 1.0, k)
    c, lpfull, rank, info = lapack.dpstrf(K.copy(), lower=1, tol=-1.0)
    lpfull = lpfull - 1
    lp = lpfull[:k]
    ok = gaps[1:] > 1e-9  # step 0 is an exact tie (all diagonals equal s)
    assert piv[0] == 0 and lp[0] == 0
    np.testing.assert_array_equal(piv[1:][ok], lp[1:][ok])
    Lref = np.tril(c)[:, :k]
    Lmine = L[lpfull]  # dpstrf stores the factor of P^T K P
    np.testing.assert_allclose(Lmine, Lref, atol=1e-10)


def test_pivchol_argmax_and_trace():
    X, ell, _ = _small(n=120, d=4, seed=23)
    K = go.kernel_matrix(X, X, ell, 1.0)
    L, piv, _ = go.pivoted_cholesky(X, ell, 1.0, 25)
    tr_prev = np.inf
    for j in range(len(piv)):
        res = np.diag(K - L[:, :j] @ L[:, :j].T).copy()
        res[piv[:j]] = 0.0
        assert abs(res[piv[j]] - res.max()) <= 1e-12
        tr = res.sum()
        assert tr <= tr_prev + 1e-12
        tr_prev = tr


def test_woodbury_and_logdet_vs_dense():
    X, ell, _ = _small(n=200, d=4, seed=24)
    sig2 = 1e-3
    L, _, _ = go.pivoted_cholesky(X, ell, 1.0, 20)
    P = L @ L.T + sig2 * np.eye(200)
    V = np.random.default_rng(0).standard_normal((200, 3))
    np.testing.assert_allclose(go.precond_solve(L, sig2, V),
                               np.linalg.solve(P, V), rtol=1e-8, atol=1e-8)
    sign, ld = np.linalg.slogdet(P)
    assert abs(go.precond_logdet(L, sig2, 200) - ld) < 1e-9 * abs(ld)


def test_splitmix64_published_outputs():
    with open(os.path.join(GOLDEN, "splitmix64_seed1234567.json")) as f:
        g = json.load(f)
    M = (1 << 64) - 1

    def mix(z):  # reference scalar SplitMix64 output function
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    outs = [mix((g["seed"] + (i + 1) * 0x9E3779B97F4A7C15) & M) for i in range(5)]
    assert outs == g["outputs"]
    signs = go.splitmix64_signs(g["seed"], np.arange(5))
    np.testing.assert_array_equal(signs, [1.0 if o >> 63 == 0 else -1.0 for o in outs])
    e = go.probe_signs(7, 0, 4096, 8)
    assert set(np.unique(e)) == {-1.0, 1.0}
    assert abs(e.mean()) < 0.03


def _krylov_minimiser(A, b, Minv, m):
    """argmin over x in K_m(M^-1 A, M^-1 b) of ||x - A^-1 b||_A (dense)."""
    v = Minv @ b
    basis = [v / np.linalg.norm(v)]
    for _ in range(m - 1):
        w = Minv @ (A @ basis[-1])
        for q in basis:
            w -= (q @ w) * q
        for q in basis:
            w -= (q @ w) * q
        basis.append(w / np.linalg.norm(w))
    Q = np.array(basis).T
    return Q @ np.linalg.solve(Q.T @ A @ Q, Q.T @ b)


def test_pcg_iterates_are_krylov_minimisers():
    X, ell, y = _small(n=150, d=4, seed=25)
    sig2 = 1e-2
    Kh = go.khat_matrix(X, ell, 1.0, sig2)
    L, _, _ = go.pivoted_cholesky(X, ell, 1.0, 5)
    Pinv = np.linalg.inv(L @ L.T + sig2 * np.eye(150))
    for m in (1, 2, 4, 6):
        res = go.mbcg(lambda V: Kh @ V, y[:, None],
                      lambda R: go.precond_solve(L, sig2, R), 0.0, m)
        ref = _krylov_minimiser(Kh, y, Pinv, m)
        np.testing.assert_allclose(res["U"][:, 0], ref, rtol=1e-7, atol=1e-9)
    # identity preconditioner: plain CG
    for m in (1, 3, 5):
        res = go.mbcg(lambda V: Kh @ V, y[:, None], lambda R: R.copy(), 0.0, m)
        ref = _krylov_minimiser(Kh, y, np.eye(150), m)
        np.testing.assert_allclose(res["U"][:, 0], ref, rtol=1e-7, atol=1e-9)


def test_mbcg_converges_to_cholesky_and_batches_independently():
    X, ell, y = _small(n=256, d=5, seed=26, dup=True)
    sig2 = 1e-4
    Kh = go.khat_matrix(X, ell, 1.0, sig2)
    L, _, _ = go.pivoted_cholesky(X, ell, 1.0, 16)
    Zp = go.probe_vectors(L, sig2, 5, 4)
    B = np.column_stack([y, Zp])
    ps = lambda R: go.precond_solve(L, sig2, R)  # noqa: E731
    res = go.mbcg(lambda V: Kh @ V, B, ps, 1e-10, 2000)
    ref = go.cholesky_solve(Kh, B)
    assert np.all(res["relres"] < 1e-10)
    err = np.linalg.norm(res["U"] - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() < 1e-6
    # each column alone follows the same recurrence (early coefficients agree
    # to rounding; later ones drift with the loss of orthogonality)
    one = go.mbcg(lambda V: Kh @ V, B[:, 2:3], ps, 1e-10, 2000)
    np.testing.assert_allclose(one["alpha"][0][:8], res["alpha"][2][:8], rtol=1e-8)
    np.testing.assert_allclose(one["U"][:, 0], res["U"][:, 2], rtol=1e-6, atol=1e-9)


def _dense_lanczos(A, w, m):
    q = w / np.linalg.norm(w)
    Q = [q]
    a, b = [], []
    for j in range(m):
        v = A @ Q[-1]
        a.append(Q[-1] @ v)
        v = v - a[-1] * Q[-1] - (b[-1] * Q[-2] if j > 0 else 0.0)
        for _ in range(2):
            for qq in Q:
                v -= (qq @ v) * qq
        if j < m - 1:
            b.append(np.linalg.norm(v))
            Q.append(v / b[-1])
    return np.array(a), np.array(b)


def test_cg_tridiagonal_equals_explicit_lanczos():
    X, ell, y = _small(n=120, d=4, seed=27)
    sig2 = 1e-2
    Kh = go.khat_matrix(X, ell, 1.0, sig2)
    L, _, _ = go.pivoted_cholesky(X, ell, 1.0, 6)
    P = L @ L.T + sig2 * np.eye(120)
    lp, Qp = np.linalg.eigh(P)
    Pmh = (Qp / np.sqrt(lp)) @ Qp.T
    A = Pmh @ Kh @ Pmh
    z = go.probe_vectors(L, sig2, 3, 1)[:, 0]
    m = 8
    res = go.mbcg(lambda V: Kh @ V, z[:, None],
                  lambda R: go.precond_solve(L, sig2, R), 0.0, m)
    dg, of = go.lanczos_tridiagonal(res["alpha"][0], res["beta"][0], m)
    a, b = _dense_lanczos(A, Pmh @ z, m)
    np.testing.assert_allclose(dg, a, rtol=1e-8)
    np.testing.assert_allclose(of, b, rtol=1e-7)


def test_full_lanczos_quadrature_is_exact():
    """After n = N steps, ||w||^2 e1^T log(T) e1 = w^T log(A) w."""
    rng = np.random.default_rng(28)
    N = 10  # small and well conditioned, so n steps keep orthogonality
    X = rng.standard_normal((N, 3)).astype(np.float32)
    ell = np.array([0.6, 0.9, 1.4])
    sig2 = 0.5
    Kh = go.khat_matrix(X, ell, 1.0, sig2)
    z = rng.choice([-1.0, 1.0], N)
    res = go.mbcg(lambda V: Kh @ V, z[:, None], lambda R: R.copy(), 0.0, N)
    dg, of = go.lanczos_tridiagonal(res["alpha"][0], res["beta"][0], N)
    lam_t = sla.eigh_tridiagonal(dg, of, eigvals_only=True)
    np.testing.assert_allclose(np.sort(lam_t), np.linalg.eigvalsh(Kh), rtol=1e-8)
    quad = res["rz0"][0] * go.quadrature_log(dg, of)
    ref = z @ sla.logm(Kh).real @ z
    assert abs(quad - ref) < 1e-9 * abs(ref)


def test_slq_logdet_matches_same_probe_target_and_exact():
    w = make_workload("gp2k", N=512, d=8)
    ell, s, sig2 = w.lengthscale, 1.0, w.sigma2
    Kh = go.khat_matrix(w.X, ell, s, sig2)
    L, _, _ = go.pivoted_cholesky(w.X, ell, s, 16)
    Zp = go.probe_vectors(L, sig2, 9, 24)
    res = go.mbcg(lambda V: Kh @ V, Zp, lambda R: go.precond_solve(L, sig2, R),
                  1e-10, 1000)
    est = go.slq_logdet(res, L, sig2, 512)
    tgt = go.same_probe_logdet_target(Kh, L, sig2, Zp)
    exact = go.exact_logdet(Kh)
    assert abs(est - tgt) < 1e-7 * abs(tgt)
    # Hutchinson error for this probe count: loose statistical bound
    assert abs(tgt - exact) < 0.05 * abs(exact)


def test_diagonal_corrected_preconditioner_vs_dense():
    """P = L L^T + diag(K - L L^T) + sigma^2 I: Woodbury solve and log|P|
    against dense linear algebra; the residual diagonal against its
    definition; probes with covariance P (sample covariance check)."""
    X, ell, _ = _small(n=180, d=4, seed=29)
    sig2 = 1e-3
    K = go.kernel_matrix(X, X, ell, 1.0)
    L, piv, _ = go.pivoted_cholesky(X, ell, 1.0, 12)
    res = go.residual_diagonal(X, ell, 1.0, L, piv)
    ref = np.diag(K - L @ L.T).copy()
    ref[piv] = 0.0
    np.testing.assert_allclose(res, ref, atol=1e-12)
    P = L @ L.T + np.diag(res + sig2)
    V = np.random.default_rng(1).standard_normal((180, 3))
    np.testing.assert_allclose(go.precond_solve(L, sig2, V, res), np.linalg.solve(P, V),
                               rtol=1e-8, atol=1e-8)
    sign, ld = np.linalg.slogdet(P)
    assert abs(go.precond_logdet(L, sig2, 180, res) - ld) < 1e-9 * abs(ld)
    Z = go.probe_vectors(L, sig2, 4, 4000, res)
    C = Z @ Z.T / 4000
    assert np.abs(C - P).max() < 0.15 * np.abs(P).max()


def test_diagonal_corrected_pcg_on_near_diagonal_kernel():
    """On a near-diagonal K (well separated points) the corrected form needs
    no more CG steps than no preconditioner, while L L^T + sigma^2 I needs more."""
    rng = np.random.default_rng(30)
    X = (3.0 * rng.standard_normal((400, 6))).astype(np.float32)
    ell = np.ones(6)
    sig2 = 1e-4
    Kh = go.khat_matrix(X, ell, 1.0, sig2)
    y = rng.standard_normal((400, 1))
    L, piv, _ = go.pivoted_cholesky(X, ell, 1.0, 20)
    res = go.residual_diagonal(X, ell, 1.0, L, piv)
    it = lambda ps: go.mbcg(lambda V: Kh @ V, y, ps, 1e-8, 2000)["iters"][0]  # noqa: E731
    none = it(lambda R: R.copy())
    sig = it(lambda R: go.precond_solve(L, sig2, R))
    cor = it(lambda R: go.precond_solve(L, sig2, R, res))
    assert cor <= none + 1 and sig > cor
