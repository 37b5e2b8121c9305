"""Plain FP64 definitions of the exact-GP path of arXiv 2109.09817.

TEST INFRASTRUCTURE ONLY (see the package docstring).  No blocking, fusion
or reordering beyond what each definition states; NumPy/SciPy library
primitives (matmul, Cholesky, eigh) serve as single steps.

Notation follows the paper: X in R^{N x d}, y in R^N, noise sigma^2,
K-hat = K(X, X) + sigma^2 I (Sec. 2.2), test points X' in R^{M x d}.
Hyperparameters theta = (lengthscale l in R^d, outputscale s, sigma^2).

Readings where the paper is silent (all listed in the design notes):
* Sec. 4 names the Matern 5/2 kernel without its formula: the standard
  form with one lengthscale per feature (ARD) is used,
  k = s (1 + sqrt5 r + 5 r^2/3) exp(-sqrt5 r), r^2 = sum_j ((x_j-x'_j)/l_j)^2.
* Eq. (pred) prints Var = K(X',X) K-hat^{-1} K(X,X'); it is read as the
  posterior variance of the latent f, k(x',x') - k*^T K-hat^{-1} k*.
* The trace probes are z = L e1 + sigma e2 with Rademacher e1 (k), e2 (N),
  so that Cov(z) = P = L L^T + sigma^2 I; the signs come from SplitMix64
  (Steele, Lea & Flood 2014) indexed by (seed, stream, probe, row).
* Pivot ties are broken by the lowest index; a pivot is taken out of the
  candidate set by zeroing its residual diagonal; the factorisation stops
  early when the largest residual diagonal is <= 1e-12 * s.
* Preconditioner form.  Sec. 3.2 uses the pivoted Cholesky factor as
  P = L L^T + sigma^2 I; Sec. 3.2 also notes that better preconditioners may
  exist.  Besides that form the oracle provides the diagonal-corrected
  P = L L^T + D, D = diag(K - L L^T) + sigma^2 I (the residual diagonal of
  the same factorisation), which equals the first form when K is close to
  rank k and stays well conditioned when K is close to diagonal.
* Serving variances at sizes where one solve per test row is out of reach
  use a low-rank Lanczos cache of K-hat^{-1} (Pleiss et al., 2018); the
  paper does not say how it serves variances.
* A molecule's correlation energy is the sum of its pair energies (Sec. 2.1,
  MOB-ML); its predictive variance is read as the variance of the sum of
  the latent values at the molecule's feature rows, 1^T Cov 1 with Cov the
  posterior covariance of Eq. (pred) (cross-covariances included), and the
  diagonal and off-diagonal models as independent GPs whose variances add.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from .cbuild import c_kernel_block, c_khat_rows, c_kcross

SQRT5 = math.sqrt(5.0)
F64 = np.float64

__all__ = [
    "matern52_of_r2", "sqdist", "kernel_matrix", "khat_matrix", "khat_matmul",
    "khat_matmul_rows", "kcross_matmul", "cholesky_solve", "exact_logdet",
    "log_marginal_likelihood", "pivoted_cholesky", "precond_solve",
    "precond_logdet", "splitmix64_signs", "probe_signs", "probe_vectors",
    "residual_diagonal", "precond_diag",
    "mbcg", "lanczos_tridiagonal", "quadrature_log", "slq_logdet",
    "same_probe_logdet_target", "dkhat_dtheta", "exact_grad",
    "same_probe_grad", "predict", "true_relative_residual",
    "sym_precond_factor", "sym_precond_apply", "bcg",
    "lanczos_variance_cache", "cached_variance", "predict_sum", "cached_variance_sum",
]


# ----------------------------------------------------------------------------
# Kernel (Sec. 4 "Matern 5/2 kernel"; K : R^d x R^d -> R, Sec. 2.2)
# ----------------------------------------------------------------------------
def matern52_of_r2(r2, s):
    """k as a function of the squared scaled distance r^2 (Sec. 4)."""
    r2 = np.asarray(r2, dtype=F64)
    r = np.sqrt(r2)
    return s * (1.0 + SQRT5 * r + (5.0 / 3.0) * r2) * np.exp(-SQRT5 * r)


def sqdist(X1, X2, lengthscale, block=256):
    """r^2_ab = sum_j ((x1_aj - x2_bj) / l_j)^2 by direct differences."""
    Z1 = np.asarray(X1, F64) / np.asarray(lengthscale, F64)
    Z2 = np.asarray(X2, F64) / np.asarray(lengthscale, F64)
    out = np.empty((Z1.shape[0], Z2.shape[0]), dtype=F64)
    for i in range(0, Z1.shape[0], block):
        diff = Z1[i:i + block, None, :] - Z2[None, :, :]
        out[i:i + block] = np.einsum("abj,abj->ab", diff, diff)
    return out


def kernel_matrix(X1, X2, lengthscale, s):
    """K(X1, X2) (Sec. 2.2, Eq. pred), dense FP64."""
    return matern52_of_r2(sqdist(X1, X2, lengthscale), s)


def khat_matrix(X, lengthscale, s, sigma2):
    """K-hat = K(X, X) + sigma^2 I (Sec. 2.2, after Eq. pred)."""
    K = c_kernel_block(X, X, lengthscale, s)
    K[np.diag_indices_from(K)] += sigma2
    return K


def khat_matmul(X, V, lengthscale, s, sigma2):
    """K-hat @ V, the blackbox product CG needs (Sec. 3.1); dense FP64."""
    K = khat_matrix(X, lengthscale, s, sigma2)
    return K @ np.asarray(V, F64)


def khat_matmul_rows(X, V, lengthscale, s, sigma2, rows):
    """Rows of K-hat @ V formed one row of K-hat at a time (Sec. 3.2: O(N)
    memory); used for row samples at sizes where K cannot be stored."""
    return c_khat_rows(X, lengthscale, s, sigma2, V, rows)


def kcross_matmul(Xp, X, V, lengthscale, s):
    """K(X', X) @ V (Eq. pred), streamed FP64."""
    return c_kcross(Xp, X, lengthscale, s, V)


def true_relative_residual(X, lengthscale, s, sigma2, Omega, B, rows=None):
    """Per-column ||K-hat w - b|| / ||b|| (Sec. 3.1's convergence measure),
    with K-hat w formed by the oracle.  With ``rows`` the norms are taken
    over that row sample only (an estimate of the full ratio)."""
    Omega = np.asarray(Omega, F64).reshape(len(B), -1)
    B = np.asarray(B, F64).reshape(len(B), -1)
    if rows is None:
        rows = np.arange(len(B))
    KO = khat_matmul_rows(X, Omega, lengthscale, s, sigma2, rows)
    res = KO - B[rows]
    return np.linalg.norm(res, axis=0) / np.linalg.norm(B[rows], axis=0)


# ----------------------------------------------------------------------------
# Cholesky exact GP (Sec. 2.2: the O(N^3) route; Eq. ll)
# ----------------------------------------------------------------------------
def cholesky_solve(Khat, B):
    """K-hat^{-1} B by a dense Cholesky factorisation (Sec. 2.2)."""
    c = sla.cho_factor(Khat, lower=True)
    return sla.cho_solve(c, np.asarray(B, F64))


def exact_logdet(Khat):
    """log|K-hat| = 2 sum log diag(chol K-hat) (Sec. 2.2)."""
    Lc = np.linalg.cholesky(Khat)
    return 2.0 * np.sum(np.log(np.diag(Lc)))


def log_marginal_likelihood(yKinvy, logdet, N):
    """Eq. (ll): L = -1/2 y^T K-hat^{-1} y - 1/2 log|K-hat| - N/2 log 2 pi."""
    return -0.5 * yKinvy - 0.5 * logdet - 0.5 * N * math.log(2.0 * math.pi)


# ----------------------------------------------------------------------------
# Pivoted Cholesky preconditioner (Sec. 3.2, refs. bach2013sharp and
# harbrecht2012low): greedy rank-k factor K ~ L L^T, P = L L^T + sigma^2 I
# ----------------------------------------------------------------------------
def pivoted_cholesky(X, lengthscale, s, k, stop_rel=1e-12):
    """Greedy pivoted Cholesky of K(X, X) in FP64.

    Returns (L (N x rank), pivots (rank,), gaps (rank,)) where gaps[j] is
    (largest - second largest) / s of the residual diagonal at step j.
    """
    X = np.asarray(X)
    N = X.shape[0]
    k = min(k, N)
    dres = np.full(N, float(s), dtype=F64)          # diag of K - L L^T
    L = np.zeros((N, k), dtype=F64)
    piv, gaps = [], []
    for j in range(k):
        p = int(np.argmax(dres))                     # first maximum
        top = dres[p]
        if top <= stop_rel * s:
            break
        rest = np.delete(dres, p)
        gaps.append((top - (rest.max() if rest.size else 0.0)) / s)
        col = c_kernel_block(X, X[p:p + 1], lengthscale, s)[:, 0]
        col = col - L[:, :j] @ L[p, :j]
        L[:, j] = col / math.sqrt(top)
        dres = dres - L[:, j] ** 2
        dres[p] = 0.0
        piv.append(p)
    r = len(piv)
    return L[:, :r], np.asarray(piv, dtype=np.int64), np.asarray(gaps)


def residual_diagonal(X, lengthscale, s, L, piv):
    """diag(K - L L^T) with the pivots' entries set to zero (their residual
    is removed by the factorisation)."""
    d = float(s) - np.sum(np.asarray(L, F64) ** 2, axis=1)
    d[np.asarray(piv, dtype=np.int64)] = 0.0
    return d


def precond_diag(L, sigma2, resid=None):
    """The diagonal D of P = L L^T + D: sigma^2 (form of Sec. 3.2) or
    resid + sigma^2 (diagonal-corrected form)."""
    N = L.shape[0]
    if resid is None:
        return np.full(N, float(sigma2))
    return np.asarray(resid, F64) + sigma2


def precond_solve(L, sigma2, V, resid=None):
    """P^{-1} V with P = L L^T + D, by the Woodbury identity:
    P^{-1} v = D^{-1} v - D^{-1} L (I_k + L^T D^{-1} L)^{-1} L^T D^{-1} v.
    With D = sigma^2 I this is (v - L (sigma^2 I_k + L^T L)^{-1} L^T v)/sigma^2."""
    V = np.asarray(V, F64)
    Dinv = 1.0 / precond_diag(L, sigma2, resid)
    DV = Dinv[:, None] * V if V.ndim == 2 else Dinv * V
    C = np.eye(L.shape[1]) + L.T @ (Dinv[:, None] * L)
    W = np.linalg.solve(C, L.T @ DV)
    LW = L @ W
    return DV - (Dinv[:, None] * LW if V.ndim == 2 else Dinv * LW)


def precond_logdet(L, sigma2, N, resid=None):
    """log|P| = sum_a log D_a + log|I_k + L^T D^{-1} L|."""
    D = precond_diag(L, sigma2, resid)
    C = np.eye(L.shape[1]) + L.T @ (L / D[:, None])
    sign, ld = np.linalg.slogdet(C)
    assert sign > 0
    return float(np.sum(np.log(D)) + ld)


# ----------------------------------------------------------------------------
# Probe vectors (Sec. 3.2: stochastic estimates of the log-determinant and
# of the derivative traces)
# ----------------------------------------------------------------------------
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_signs(seed, counters):
    """Rademacher signs from the n-th SplitMix64 output, n = counter + 1.

    SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): state_n = seed + n*gamma,
    output = mix(state_n) with the published 64-bit finaliser.  The sign is
    +1 when the output's top bit is 0, else -1.
    """
    with np.errstate(over="ignore"):
        c = np.asarray(counters, dtype=np.uint64)
        z = np.uint64(seed) + (c + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return np.where((z >> np.uint64(63)) == 0, 1.0, -1.0)


def probe_signs(seed, stream, n_rows, n_probes):
    """(n_rows x n_probes) signs; counter = stream<<56 | probe<<32 | row."""
    rows = np.arange(n_rows, dtype=np.uint64)[:, None]
    cols = np.arange(n_probes, dtype=np.uint64)[None, :]
    ctr = (np.uint64(stream) << np.uint64(56)) | (cols << np.uint64(32)) | rows
    return splitmix64_signs(seed, ctr)


def probe_vectors(L, sigma2, seed, n_probes, resid=None):
    """z_c = L e1_c + D^{1/2} e2_c, e1 in {+-1}^k (stream 1), e2 in {+-1}^N
    (stream 0), so that Cov(z) = P = L L^T + D."""
    N, k = L.shape
    e2 = probe_signs(seed, 0, N, n_probes)
    e1 = probe_signs(seed, 1, k, n_probes)
    return L @ e1 + np.sqrt(precond_diag(L, sigma2, resid))[:, None] * e2


# ----------------------------------------------------------------------------
# mBCG (Sec. 3.2, ref. gardner2018gpytorch): preconditioned CG (Sec. 3.1)
# run on t right-hand sides at once, sharing one K-hat product per step,
# recording the CG coefficients from which Lanczos tridiagonals follow.
# ----------------------------------------------------------------------------
def mbcg(matmul, B, psolve, tol, max_iter):
    """Solve K-hat U = B column by column with PCG, all columns together.

    Stop rule (Sec. 4): a column stops when ||r_c|| / ||b_c|| < tol; the
    solve stops when every column has stopped or after max_iter steps.
    Returns dict with U, alpha/beta lists per column, iters, relres, rz0.
    """
    B = np.asarray(B, F64)
    N, t = B.shape
    U = np.zeros_like(B)
    R = B.copy()
    Z = psolve(R)
    D = Z.copy()
    rz = np.sum(R * Z, axis=0)
    rz0 = rz.copy()
    bnorm = np.linalg.norm(B, axis=0)
    active = bnorm > 0
    alphas = [[] for _ in range(t)]
    betas = [[] for _ in range(t)]
    iters = np.zeros(t, dtype=np.int64)
    relres = np.where(active, 1.0, 0.0)
    for it in range(max_iter):
        if not active.any():
            break
        W = matmul(D)
        dw = np.sum(D * W, axis=0)
        cols = np.nonzero(active)[0]
        alpha = rz[cols] / dw[cols]
        U[:, cols] += D[:, cols] * alpha
        R[:, cols] -= W[:, cols] * alpha
        for c, a in zip(cols, alpha):
            alphas[c].append(a)
        relres[cols] = np.linalg.norm(R[:, cols], axis=0) / bnorm[cols]
        Z = psolve(R)
        rz_new = np.sum(R * Z, axis=0)
        for c in cols:
            iters[c] = it + 1
            if relres[c] < tol:
                active[c] = False
                continue
            beta = rz_new[c] / rz[c]
            betas[c].append(beta)
            D[:, c] = Z[:, c] + D[:, c] * beta
            rz[c] = rz_new[c]
    return dict(U=U, alpha=alphas, beta=betas, iters=iters, relres=relres,
                rz0=rz0)


# ----------------------------------------------------------------------------
# AltBBMM (Sec. 3.2): block CG (BCG, Sec. 3.1) with symmetric preconditioning
# S^T K-hat S, S S^T = P^{-1}, and the Nystrom preconditioner.  Reading: the
# Nystrom landmarks are the greedy pivoted-Cholesky pivots, so the low-rank
# part of P is the same L L^T as in BBMM; P = L L^T + D as above.
# ----------------------------------------------------------------------------
def sym_precond_factor(L, sigma2, resid=None):
    """Factors of S = D^{-1/2} (I + Lt Lt^T)^{-1/2} with Lt = D^{-1/2} L, so
    that S S^T = P^{-1}.  With Lt^T Lt = V diag(lam) V^T,
    (I + Lt Lt^T)^{-1/2} = I + Lt Cp Lt^T, Cp = V diag(g(lam)) V^T,
    g(lam) = ((1 + lam)^{-1/2} - 1) / lam = -1 / (sqrt(1+lam) (1 + sqrt(1+lam))).
    Returns (dh = D^{-1/2}, Lt, Cp)."""
    L = np.asarray(L, F64)
    dh = 1.0 / np.sqrt(precond_diag(L, sigma2, resid))
    Lt = dh[:, None] * L
    lam, V = np.linalg.eigh(Lt.T @ Lt)
    lam = np.maximum(lam, 0.0)
    r = np.sqrt(1.0 + lam)
    g = -1.0 / (r * (1.0 + r))
    return dh, Lt, (V * g) @ V.T


def sym_precond_apply(fac, V, transpose=False):
    """S V (transpose=False: dh o (G V)) or S^T V (G (dh o V)), with
    G = I + Lt Cp Lt^T symmetric."""
    dh, Lt, Cp = fac
    V = np.asarray(V, F64)
    dv = dh[:, None] if V.ndim == 2 else dh
    if transpose:
        V = dv * V
    GV = V + Lt @ (Cp @ (Lt.T @ V))
    return GV if transpose else dv * GV


def bcg(matmul, B, fac, tol, max_iter):
    """Block CG (O'Leary's recurrences) on A = S^T K-hat S, right-hand sides
    S^T B; Omega = S W solves K-hat Omega = B for all s columns together.

    Per step: Dt = S D, W = K-hat Dt, Q = S^T W, alpha = (D^T Q)^{-1} (Rh^T Rh),
    Omega += Dt alpha, R -= W alpha, Rh -= Q alpha,
    beta = (Rh^T Rh)^{-1} (Rh'^T Rh'), D = Rh' + D beta.
    R = B - K-hat Omega is carried by its recurrence; the solve stops when all
    s relative residuals ||R_c|| / ||B_c|| are below tol (Sec. 4) or after
    max_iter steps.  Returns dict(Omega, iters, relres)."""
    B = np.asarray(B, F64)
    N, s = B.shape
    Om = np.zeros_like(B)
    R = B.copy()
    Rh = sym_precond_apply(fac, R, transpose=True)
    D = Rh.copy()
    rho = Rh.T @ Rh
    bnorm = np.linalg.norm(B, axis=0)
    relres = np.ones(s)
    it = 0
    while it < max_iter and np.any(relres >= tol):
        Dt = sym_precond_apply(fac, D)
        W = matmul(Dt)
        Q = sym_precond_apply(fac, W, transpose=True)
        alpha = np.linalg.solve(D.T @ Q, rho)
        Om += Dt @ alpha
        R -= W @ alpha
        Rh -= Q @ alpha
        rho_new = Rh.T @ Rh
        beta = np.linalg.solve(rho, rho_new)
        D = Rh + D @ beta
        rho = rho_new
        relres = np.linalg.norm(R, axis=0) / bnorm
        it += 1
    return dict(Omega=Om, iters=it, relres=relres)


def lanczos_tridiagonal(alpha, beta, m=None):
    """The m x m Lanczos matrix T of PCG (the CG/Lanczos relation):
    T_jj = 1/a_j + b_{j-1}/a_{j-1},  T_{j,j+1} = sqrt(b_j)/a_j."""
    a = np.asarray(alpha, F64)
    b = np.asarray(beta, F64)
    m = len(a) if m is None else m
    diag = np.empty(m)
    off = np.empty(max(m - 1, 0))
    for j in range(m):
        diag[j] = 1.0 / a[j] + (b[j - 1] / a[j - 1] if j > 0 else 0.0)
        if j < m - 1:
            off[j] = math.sqrt(b[j]) / a[j]
    return diag, off


def quadrature_log(diag, off):
    """e1^T log(T) e1 = sum_i q_{0i}^2 log(lambda_i) (Gauss quadrature of the
    Lanczos matrix T)."""
    if len(diag) == 0:
        return 0.0
    lam, Q = sla.eigh_tridiagonal(diag, off)
    return float(np.sum(Q[0, :] ** 2 * np.log(lam)))


def slq_logdet(res, L, sigma2, N, resid=None):
    """log|K-hat| ~ log|P| + (1/t) sum_c ||w_c||^2 e1^T log(T_c) e1 with
    ||w_c||^2 = z_c^T P^{-1} z_c = r0^T z0 (Sec. 3.2: mBCG estimates of
    the log marginal likelihood).  ``res`` is ``mbcg`` output on the probe
    columns only."""
    t = len(res["alpha"])
    acc = 0.0
    for c in range(t):
        dg, of = lanczos_tridiagonal(res["alpha"][c], res["beta"][c],
                                     int(res["iters"][c]))
        acc += res["rz0"][c] * quadrature_log(dg, of)
    return precond_logdet(L, sigma2, N, resid) + acc / t


def same_probe_logdet_target(Khat, L, sigma2, Zp, resid=None):
    """The value the stochastic estimate converges to for these probes:
    log|P| + (1/t) sum_c z_c^T P^{-1/2} log(A) P^{-1/2} z_c,
    A = P^{-1/2} K-hat P^{-1/2}, by dense eigendecompositions."""
    N = Khat.shape[0]
    P = L @ L.T + np.diag(precond_diag(L, sigma2, resid))
    lp, Qp = np.linalg.eigh(P)
    Pmh = (Qp / np.sqrt(lp)) @ Qp.T
    A = Pmh @ Khat @ Pmh
    la, Qa = np.linalg.eigh(0.5 * (A + A.T))
    Wt = Qa.T @ (Pmh @ Zp)
    quad = np.sum(Wt ** 2 * np.log(la)[:, None], axis=0)
    return float(np.sum(np.log(lp)) + quad.mean())


# ----------------------------------------------------------------------------
# Derivatives (Sec. 2.2 "hyperparameters ... learned by maximizing" Eq. ll;
# Sec. 3.2 "marginal likelihood and its derivatives")
# dL/dtheta = 1/2 a^T dK a - 1/2 tr(K-hat^{-1} dK),  a = K-hat^{-1} y
# ----------------------------------------------------------------------------
def dkhat_dtheta(X, lengthscale, s):
    """Dense dK-hat/dtheta for theta = (l_1..l_d, s, sigma^2).

    dk/dl_j = s (5/3) (1 + sqrt5 r) exp(-sqrt5 r) (x_j - x'_j)^2 / l_j^3,
    dk/ds = k / s, dK-hat/dsigma^2 = I.  Yields the d + 2 matrices one at a
    time, so that only one of them is held at once.
    """
    X = np.asarray(X, F64)
    ell = np.asarray(lengthscale, F64)
    r2 = sqdist(X, X, ell)
    r = np.sqrt(r2)
    g = s * (5.0 / 3.0) * (1.0 + SQRT5 * r) * np.exp(-SQRT5 * r)
    for j in range(X.shape[1]):
        dj = (X[:, j:j + 1] - X[None, :, j]) ** 2 / ell[j] ** 3
        yield g * dj
    yield matern52_of_r2(r2, s) / s
    yield np.eye(X.shape[0])


def exact_grad(X, y, lengthscale, s, sigma2):
    """Exact dL/dtheta in natural parameters (l_1..l_d, s, sigma^2)."""
    Khat = khat_matrix(X, lengthscale, s, sigma2)
    Kinv = np.linalg.inv(Khat)
    a = Kinv @ np.asarray(y, F64)
    return np.array([0.5 * a @ dK @ a - 0.5 * np.sum(Kinv * dK)
                     for dK in dkhat_dtheta(X, lengthscale, s)])


def same_probe_grad(X, y, lengthscale, s, sigma2, Zp, PinvZ):
    """The estimator's value for fixed probes with exact solves:
    1/2 a^T dK a - 1/(2t) sum_c (K-hat^{-1} z_c)^T dK (P^{-1} z_c)."""
    Khat = khat_matrix(X, lengthscale, s, sigma2)
    a = cholesky_solve(Khat, y)
    U = cholesky_solve(Khat, Zp)
    t = Zp.shape[1]
    out = []
    for dK in dkhat_dtheta(X, lengthscale, s):
        tr = np.sum(U * (dK @ PinvZ)) / t
        out.append(0.5 * a @ dK @ a - 0.5 * tr)
    return np.array(out)


# ----------------------------------------------------------------------------
# Prediction (Eq. pred)
# ----------------------------------------------------------------------------
def predict(X, y, Xp, lengthscale, s, sigma2, observation_noise=False):
    """mean = K(X',X) K-hat^{-1} y; var_i = k(x'_i,x'_i) - k_i^T K-hat^{-1} k_i
    (+ sigma^2 when ``observation_noise``)."""
    Khat = khat_matrix(X, lengthscale, s, sigma2)
    Ks = kernel_matrix(Xp, X, lengthscale, s)
    c = sla.cho_factor(Khat, lower=True)
    mean = Ks @ sla.cho_solve(c, np.asarray(y, F64))
    var = s - np.sum(Ks * sla.cho_solve(c, Ks.T).T, axis=1)
    if observation_noise:
        var = var + sigma2
    return mean, var


# ----------------------------------------------------------------------------
# Variance cache for serving (the low-rank Lanczos cache of Pleiss et al.,
# 2018, "LOVE"; a reading for the latent variance of Eq. (pred) at sizes
# where one solve per test row is out of reach)
# ----------------------------------------------------------------------------
def lanczos_variance_cache(Khat, b, m):
    """m steps of Lanczos on K-hat started at b, with full
    reorthogonalisation in FP64: Q^T K-hat Q = T, Q orthonormal (N x m'),
    m' <= m (fewer when b's Krylov space is exhausted).  K-hat^{-1} is
    approximated by Q T^{-1} Q^T = R R^T with R = Q C^{-T}, T = C C^T.
    Returns (R, T)."""
    Khat = np.asarray(Khat, F64)
    b = np.asarray(b, F64)
    N = Khat.shape[0]
    Q = np.zeros((N, m))
    alpha = np.zeros(m)
    beta = np.zeros(m)
    q = b / np.linalg.norm(b)
    q_prev = np.zeros(N)
    steps = 0
    for j in range(m):
        Q[:, j] = q
        w = Khat @ q - (beta[j - 1] * q_prev if j > 0 else 0.0)
        alpha[j] = q @ w
        w = w - alpha[j] * q
        for _ in range(2):                      # full reorthogonalisation
            w = w - Q[:, :j + 1] @ (Q[:, :j + 1].T @ w)
        steps = j + 1
        beta[j] = np.linalg.norm(w)
        if beta[j] <= 1e-12 * abs(alpha[0]):
            break
        q_prev, q = q, w / beta[j]
    Q = Q[:, :steps]
    T = np.diag(alpha[:steps]) + np.diag(beta[:steps - 1], 1) + np.diag(beta[:steps - 1], -1)
    C = np.linalg.cholesky(T)
    R = sla.solve_triangular(C, Q.T, lower=True).T      # Q C^{-T}
    return R, T


def cached_variance(X, Xp, lengthscale, s, R):
    """var_i ~ k(x'_i, x'_i) - |R^T k_i|^2 with k_i = K(X, x'_i)."""
    Ks = kernel_matrix(Xp, X, lengthscale, s)
    return s - np.sum((Ks @ R) ** 2, axis=1)


# ----------------------------------------------------------------------------
# Per-molecule sums (Sec. 2.1: E_corr is the sum of a molecule's pair
# energies; Eq. (pred) for each pair's latent value)
# ----------------------------------------------------------------------------
def predict_sum(X, y, Xp, lengthscale, s, sigma2):
    """Mean and variance of S = sum_i f(x'_i) over the M rows of X' under the
    posterior of Eq. (pred): E[S] = 1^T K(X',X) K-hat^{-1} y and
    Var[S] = 1^T K(X',X') 1 - c^T K-hat^{-1} c with c = K(X,X') 1, i.e. the
    sum of every entry of the posterior covariance (variances and the
    cross-covariances between the molecule's rows)."""
    Khat = khat_matrix(X, lengthscale, s, sigma2)
    Ks = kernel_matrix(Xp, X, lengthscale, s)
    Kss = kernel_matrix(Xp, Xp, lengthscale, s)
    ch = sla.cho_factor(Khat, lower=True)
    ones = np.ones(len(Xp))
    mean = ones @ (Ks @ sla.cho_solve(ch, np.asarray(y, F64)))
    c = Ks.T @ ones
    var = ones @ Kss @ ones - c @ sla.cho_solve(ch, c)
    return float(mean), float(var)


def cached_variance_sum(X, Xp, lengthscale, s, R):
    """Var[S] with the Lanczos cache K-hat^{-1} ~ R R^T:
    1^T K(X',X') 1 - |R^T K(X,X') 1|^2."""
    Ks = kernel_matrix(Xp, X, lengthscale, s)
    Kss = kernel_matrix(Xp, Xp, lengthscale, s)
    ones = np.ones(len(Xp))
    u = R.T @ (Ks.T @ ones)
    return float(ones @ Kss @ ones - u @ u)
