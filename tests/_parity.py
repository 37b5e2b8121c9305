"""Comparison helpers for the CUDA-vs-oracle parity tests.

Two measures of a K-hat V result `got` (N x t) against the oracle's `ref`:
* column_relerr: max over columns of ||got_c - ref_c|| / ||ref_c|| (the
  stated tolerance of each precision form);
* element_ratio: max over entries of |got_ac - ref_ac| / sum_b |K-hat_ab| |V_bc|,
  the error of each entry against the scale of the sum that forms it.  A few
  bad rows (a wrong diagonal, a near-duplicate row whose u^2 cancels) are
  hidden inside a column norm but not here.
The absolute-value sums come from the same oracle call on |V| (K-hat's
entries are non-negative for the Matern kernel, so sum_b |K-hat_ab| |V_bc| =
(K-hat |V|)_ac).
"""
import numpy as np

from oracle import gp_oracle as go

# element_ratio bounds per precision form.  u^2 = n_a + n_b - 2 x~_a . x~_b
# is formed by the norm expansion, so its rounding is absolute, about
# 2^-22 (n_a + n_b) in the split forms; at u ~ 0 (duplicate rows, K ~ s) the
# kernel's slope dK/du^2 = -(ln 2)^2 / 6 turns that into an entry error of a
# few 1e-5 of K when |x~|^2 ~ 1e3 (measured 4.4e-5 on the near-duplicate
# rows of the 65,536-row generator).  Rows dominated by such a pair carry
# that ratio; the split forms are held to 1e-4, FP32 (2 bits more) to 2e-5.
ELEM_TOL = {"fp32": 2e-5, "split_tf32": 1e-4, "split_f16": 1e-4, "tf32": 2e-2}


def column_relerr(got, ref):
    num = np.linalg.norm(np.asarray(got, np.float64) - ref, axis=0)
    return float(np.max(num / np.maximum(np.linalg.norm(ref, axis=0), 1e-300)))


def element_ratio(got, ref, absref):
    err = np.abs(np.asarray(got, np.float64) - ref)
    return float(np.max(err / np.maximum(absref, 1e-300)))


def khat_ref(X, V_rows, ell, s, sig2, rows=None):
    """Oracle K-hat V and K-hat |V| (V_rows: N x t, FP64), optionally on a
    row sample."""
    V = np.asarray(V_rows, np.float64)
    both = np.hstack([V, np.abs(V)])
    if rows is None:
        r = go.khat_matmul(X, both, ell, s, sig2)
    else:
        r = go.khat_matmul_rows(X, both, ell, s, sig2, rows)
    t = V.shape[1]
    return r[:, :t], r[:, t:]


def kcross_ref(Xp, X, V_rows, ell, s):
    V = np.asarray(V_rows, np.float64)
    r = go.kcross_matmul(Xp, X, np.hstack([V, np.abs(V)]), ell, s)
    t = V.shape[1]
    return r[:, :t], r[:, t:]


def check_kmv(got, ref, absref, col_tol, form):
    """Both measures; returns them for messages."""
    ce = column_relerr(got, ref)
    er = element_ratio(got, ref, absref)
    assert ce <= col_tol, f"column error {ce:.3e} > {col_tol:.1e}"
    assert er <= ELEM_TOL[form], f"element error ratio {er:.3e} > {ELEM_TOL[form]:.1e}"
    return ce, er
