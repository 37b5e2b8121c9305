"""Pins for the oracle's kernel and K-hat products (CPU only).

Each check compares against something other than the oracle's own formula:
the general Matern family through the modified Bessel function, brute-force
Python loops, invariants (k(x,x)=s, symmetry, positive definiteness,
monotonicity, ARD scale invariance).
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
from oracle import gp_oracle as go


def _bessel_matern(r, s, nu=2.5):
    """General Matern: s 2^{1-nu}/Gamma(nu) (sqrt(2 nu) r)^nu K_nu(sqrt(2 nu) r)."""
    z = math.sqrt(2 * nu) * r
    return s * 2 ** (1 - nu) / special.gamma(nu) * z ** nu * special.kv(nu, z)


def test_matern52_equals_bessel_family():
    r = np.linspace(1e-3, 12.0, 400)
    for s in (1.0, 0.37):
        got = go.matern52_of_r2(r * r, s)
        ref = np.array([_bessel_matern(x, s) for x in r])
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-300)
    # r -> 0 limit of the Bessel form is s
    assert abs(_bessel_matern(1e-6, 2.0) - 2.0) < 1e-9
    assert go.matern52_of_r2(0.0, 2.0) == 2.0


def test_matern52_monotone_decreasing():
    r2 = np.linspace(0, 200, 2001)
    k = go.matern52_of_r2(r2, 1.0)
    assert np.all(np.diff(k) < 0)
    assert np.all(k > 0)


def _brute_kernel(X1, X2, ell, s):
    out = np.zeros((len(X1), len(X2)))
    for a in range(len(X1)):
        for b in range(len(X2)):
            r2 = 0.0
            for j in range(X1.shape[1]):
                u = (float(X1[a, j]) - float(X2[b, j])) / ell[j]
                r2 += u * u
            out[a, b] = _bessel_matern(math.sqrt(r2), s) if r2 > 0 else s
    return out


def test_kernel_matrix_vs_brute_force():
    rng = np.random.default_rng(11)
    X = rng.standard_normal((17, 5)).astype(np.float32)
    Xp = rng.standard_normal((9, 5)).astype(np.float32)
    ell = rng.uniform(0.5, 2.0, 5)
    ref = _brute_kernel(X, Xp, ell, 1.3)
    np.testing.assert_allclose(go.kernel_matrix(X, Xp, ell, 1.3), ref,
                               rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(oracle.cbuild.c_kernel_block(X, Xp, ell, 1.3),
                               ref, rtol=1e-11, atol=1e-14)


def test_khat_products_vs_brute_force():
    rng = np.random.default_rng(12)
    N, d, t = 23, 4, 3
    X = rng.standard_normal((N, d)).astype(np.float32)
    V = rng.standard_normal((N, t))
    ell = rng.uniform(0.5, 2.0, d)
    s, sig2 = 0.8, 1e-2
    K = _brute_kernel(X, X, ell, s)
    ref = np.zeros((N, t))
    for a in range(N):
        for c in range(t):
            acc = sig2 * V[a, c]
            for b in range(N):
                acc += K[a, b] * V[b, c]
            ref[a, c] = acc
    np.testing.assert_allclose(go.khat_matmul(X, V, ell, s, sig2), ref,
                               rtol=1e-11, atol=1e-13)
    rows = np.array([0, 5, 22, 7])
    np.testing.assert_allclose(go.khat_matmul_rows(X, V, ell, s, sig2, rows),
                               ref[rows], rtol=1e-11, atol=1e-13)
    Xp = rng.standard_normal((6, d)).astype(np.float32)
    Kp = _brute_kernel(Xp, X, ell, s)
    np.testing.assert_allclose(go.kcross_matmul(Xp, X, V, ell, s), Kp @ V,
                               rtol=1e-11, atol=1e-13)


def test_khat_invariants():
    rng = np.random.default_rng(13)
    X = rng.standard_normal((200, 6)).astype(np.float32)
    ell = rng.uniform(0.5, 2.0, 6)
    s, sig2 = 1.7, 1e-4
    Kh = go.khat_matrix(X, ell, s, sig2)
    np.testing.assert_array_equal(np.diag(Kh), np.full(200, s + sig2))
    np.testing.assert_array_equal(Kh, Kh.T)
    lam = np.linalg.eigvalsh(Kh)
    assert lam.min() >= sig2 - 1e-12


def test_ard_scale_invariance():
    rng = np.random.default_rng(14)
    X = rng.standard_normal((30, 3))
    ell = np.array([0.7, 1.1, 1.9])
    c = np.array([2.0, 0.5, 4.0])  # powers of two: exact rescaling
    K1 = go.kernel_matrix(X, X, ell, 1.0)
    K2 = go.kernel_matrix(X * c, X * c, ell * c, 1.0)
    np.testing.assert_allclose(K1, K2, rtol=1e-14, atol=1e-15)


def test_true_relative_residual_vs_brute_force():
    """The solve checker: ||K-hat w - b|| / ||b|| per column with K-hat from
    brute-force loops, full and on a row sample."""
    rng = np.random.default_rng(14)
    N, d = 21, 3
    X = rng.standard_normal((N, d)).astype(np.float32)
    ell = rng.uniform(0.5, 2.0, d)
    Kh = _brute_kernel(X, X, ell, 0.9) + 1e-2 * np.eye(N)
    W = rng.standard_normal((N, 2))
    B = Kh @ W + 1e-3 * rng.standard_normal((N, 2))
    ref = np.linalg.norm(Kh @ W - B, axis=0) / np.linalg.norm(B, axis=0)
    np.testing.assert_allclose(go.true_relative_residual(X, ell, 0.9, 1e-2, W, B), ref,
                               rtol=1e-9)
    rows = np.array([0, 3, 7, 20])
    refr = np.linalg.norm((Kh @ W - B)[rows], axis=0) / np.linalg.norm(B[rows], axis=0)
    np.testing.assert_allclose(go.true_relative_residual(X, ell, 0.9, 1e-2, W, B, rows), refr,
                               rtol=1e-9)
    # the exact solution has zero residual
    assert go.true_relative_residual(X, ell, 0.9, 1e-2, np.linalg.solve(Kh, B), B).max() < 1e-10
