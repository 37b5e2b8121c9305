"""The integral form of the Lanczos quadrature (the device's evaluation of
e1^T log(T) e1, Sec. 3.2), checked on the CPU against the eigendecomposition.

For a positive definite tridiagonal T with eigenpairs (lambda_i, q_i),
e1^T log(T) e1 = sum_i q_{0i}^2 log(lambda_i).  The device evaluates it as
int_R [sig(u) - e^u e1^T (T + e^u I)^{-1} e1] du (sig the logistic function)
with a trapezoid rule of step 0.25, the resolvent entry from the bottom-up
continued fraction of T + s I, and the range cut where the tails' exact bounds
e^{u_lo} (1 + e1^T T^{-1} e1) and e^{-u_hi} (1 + T_00) reach 1e-16.  This
test restates those steps in NumPy FP64 and compares them with
scipy.linalg.eigh_tridiagonal; tests/test_gpu_lanczos.py compares the kernel
itself with the oracle.
"""
import math

import numpy as np
import scipy.linalg as sla


def _tridiagonal(al, be):
    m = len(al)
    a = np.empty(m)
    off = np.zeros(max(m - 1, 0))
    for j in range(m):
        a[j] = 1.0 / al[j] + (be[j - 1] / al[j - 1] if j > 0 else 0.0)
        if j < m - 1:
            off[j] = math.sqrt(be[j]) / al[j]
    return a, off


def _resolvent00(a, b2, s):
    # e1^T (T + s I)^{-1} e1 by the bottom-up continued fraction
    d = a[-1] + s
    for j in range(len(a) - 2, -1, -1):
        d = a[j] + s - b2[j] / d
    return 1.0 / d


def _integral_form(a, off, h=0.25, tol=1e-16):
    b2 = off ** 2
    g0 = _resolvent00(a, b2, 0.0)
    ulo = math.log(tol / (1.0 + g0))
    uhi = math.log((1.0 + a[0]) / tol)
    u = ulo + h * np.arange(int(math.ceil((uhi - ulo) / h)) + 1)
    s = np.exp(u)
    r = _resolvent00(a, b2, s)
    return h * float(np.sum(1.0 / (1.0 + np.exp(-u)) - s * r))


def _eig_form(a, off):
    lam, q = sla.eigh_tridiagonal(a, off)
    return float(np.sum(q[0] ** 2 * np.log(lam)))


def test_integral_form_matches_eigendecomposition():
    rng = np.random.default_rng(3)
    for m in (1, 2, 7, 64, 400, 1500):
        al = np.exp(rng.uniform(-4.0, 3.0, m))
        be = np.exp(rng.uniform(-6.0, 0.5, m))
        a, off = _tridiagonal(al, be)
        ref = _eig_form(a, off)
        got = _integral_form(a, off)
        assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (m, got, ref)


def test_integral_form_over_ten_decades():
    rng = np.random.default_rng(4)
    al = np.exp(rng.uniform(-12.0, 8.0, 800))
    be = np.exp(rng.uniform(-10.0, 2.0, 800))
    a, off = _tridiagonal(al, be)
    lam = sla.eigh_tridiagonal(a, off, eigvals_only=True)
    assert lam.max() / lam.min() > 1e9
    ref = _eig_form(a, off)
    assert abs(_integral_form(a, off) - ref) <= 1e-11 * max(1.0, abs(ref))


def test_one_by_one_is_the_log():
    # m = 1: the quadrature is log T_00 exactly
    for t00 in (1e-6, 0.3, 1.0, 42.0, 1e7):
        assert abs(_integral_form(np.array([t00]), np.zeros(0)) - math.log(t00)) < 1e-12 * max(1.0, abs(math.log(t00)))


def test_step_and_tails_matter():
    # a coarser step or a range cut short by ten units both break the
    # agreement, so the 1e-12 match above is not accidental
    rng = np.random.default_rng(5)
    al = np.exp(rng.uniform(-4.0, 3.0, 200))
    be = np.exp(rng.uniform(-6.0, 0.5, 200))
    a, off = _tridiagonal(al, be)
    ref = _eig_form(a, off)
    assert abs(_integral_form(a, off, h=2.0) - ref) > 1e-6
    assert abs(_integral_form(a, off, tol=1e-4) - ref) > 1e-8
