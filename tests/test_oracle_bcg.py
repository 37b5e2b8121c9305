"""Pins for the oracle's AltBBMM pieces (CPU only): the symmetric
preconditioner factor against dense linear algebra, block CG against PCG
(block size 1 is PCG), against the Cholesky solution, and against the
block-Krylov minimisation that defines it, computed by an explicit dense
projection."""
import numpy as np
import scipy.linalg as sla

from oracle import gp_oracle as go


def _problem(n=160, d=4, seed=41, sig2=1e-3, k=12, resid=False):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)).astype(np.float32)
    ell = rng.uniform(0.6, 1.6, d)
    Kh = go.khat_matrix(X, ell, 1.0, sig2)
    L, piv, _ = go.pivoted_cholesky(X, ell, 1.0, k)
    res = go.residual_diagonal(X, ell, 1.0, L, piv) if resid else None
    return X, ell, Kh, L, res, sig2


def test_sym_factor_is_inverse_square_root():
    for resid in (False, True):
        X, ell, Kh, L, res, sig2 = _problem(resid=resid)
        fac = go.sym_precond_factor(L, sig2, res)
        n = L.shape[0]
        S = go.sym_precond_apply(fac, np.eye(n))
        St = go.sym_precond_apply(fac, np.eye(n), transpose=True)
        np.testing.assert_allclose(St, S.T, atol=1e-10)
        P = L @ L.T + np.diag(go.precond_diag(L, sig2, res))
        np.testing.assert_allclose(S @ S.T, np.linalg.inv(P), rtol=1e-8, atol=1e-8 / sig2)
        np.testing.assert_allclose(S.T @ P @ S, np.eye(n), atol=1e-8)


def test_block_size_one_is_pcg():
    """In exact arithmetic CG on S^T K-hat S equals PCG with P = (S S^T)^{-1}:
    same iterates step by step."""
    X, ell, Kh, L, res, sig2 = _problem(seed=42)
    fac = go.sym_precond_factor(L, sig2)
    b = np.random.default_rng(1).standard_normal((len(Kh), 1))
    for k in (1, 3, 7, 12):
        a = go.bcg(lambda V: Kh @ V, b, fac, 0.0, k)
        p = go.mbcg(lambda V: Kh @ V, b, lambda R: go.precond_solve(L, sig2, R), 0.0, k)
        np.testing.assert_allclose(a["Omega"], p["U"], rtol=1e-7, atol=1e-9 * np.abs(p["U"]).max())


def test_bcg_converges_to_cholesky():
    X, ell, Kh, L, res, sig2 = _problem(seed=43, resid=True)
    fac = go.sym_precond_factor(L, sig2, res)
    B = np.random.default_rng(2).standard_normal((len(Kh), 6))
    r = go.bcg(lambda V: Kh @ V, B, fac, 1e-10, 500)
    assert np.all(r["relres"] < 1e-10)
    np.testing.assert_allclose(r["Omega"], go.cholesky_solve(Kh, B), rtol=1e-6,
                               atol=1e-8 * np.abs(go.cholesky_solve(Kh, B)).max())
    # the recurrence residual is the true residual
    true = np.linalg.norm(B - Kh @ r["Omega"], axis=0) / np.linalg.norm(B, axis=0)
    assert true.max() < 1e-8


def test_bcg_minimises_over_the_block_krylov_space():
    """After k steps every column's A-norm error (A = S^T K-hat S) is the
    minimum over the block Krylov space span{A^j R0 : j < k} (Sec. 3.1), by a
    dense projection onto an orthonormal basis of that space."""
    X, ell, Kh, L, res, sig2 = _problem(n=120, seed=44, k=8)
    fac = go.sym_precond_factor(L, sig2)
    n = len(Kh)
    S = go.sym_precond_apply(fac, np.eye(n))
    A = S.T @ Kh @ S
    B = np.random.default_rng(3).standard_normal((n, 3))
    Bh = S.T @ B
    Wstar = np.linalg.solve(A, Bh)
    for k in (1, 2, 4):
        r = go.bcg(lambda V: Kh @ V, B, fac, 0.0, k)
        W = np.linalg.solve(S, r["Omega"])
        blocks = [Bh]
        for _ in range(k - 1):
            blocks.append(A @ blocks[-1])
        Qb, _ = np.linalg.qr(np.hstack(blocks))
        # A-orthogonal projection of W* onto span(Qb)
        Wp = Qb @ np.linalg.solve(Qb.T @ A @ Qb, Qb.T @ A @ Wstar)
        np.testing.assert_allclose(W, Wp, rtol=1e-6, atol=1e-8 * np.abs(Wp).max())


def test_block_beats_single_column_on_y():
    """The block space contains each column's own Krylov space, so the y
    column's A-norm error after k block steps is at most PCG's (Sec. 3.1)."""
    X, ell, Kh, L, res, sig2 = _problem(n=200, seed=45, k=10)
    fac = go.sym_precond_factor(L, sig2)
    n = len(Kh)
    S = go.sym_precond_apply(fac, np.eye(n))
    A = S.T @ Kh @ S
    rng = np.random.default_rng(4)
    B = np.hstack([rng.standard_normal((n, 1)), rng.standard_normal((n, 7))])
    wstar = np.linalg.solve(Kh, B[:, :1])
    for k in (2, 5, 9):
        blk = go.bcg(lambda V: Kh @ V, B, fac, 0.0, k)["Omega"][:, :1]
        one = go.bcg(lambda V: Kh @ V, B[:, :1], fac, 0.0, k)["Omega"]
        ea = (blk - wstar).T @ Kh @ (blk - wstar)
        eb = (one - wstar).T @ Kh @ (one - wstar)
        assert ea[0, 0] <= eb[0, 0] * (1 + 1e-8) + 1e-14
