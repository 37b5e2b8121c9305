"""Operand-representation error of each tensor-core form, on the CPU.

The tensor-core products see the features, the kernel values and the vectors
only through their split parts.  This test rebuilds those parts in NumPy (TF32
round-to-nearest-away, FP16 and BF16 round-to-nearest-even, the power-of-two
scaling of the FP16 form), forms K-hat V from them with FP64 arithmetic, and
compares with the oracle.  It isolates the representation error from the
tensor core's FP32 accumulation (which the GPU parity tests include; about
1e-5 at N = 2^20) and backs the choice of forms:
* split TF32 and split FP16 keep 22 significant bits: ~2e-7, far below the
  2e-5 tolerance;
* a split-BF16 form keeps 16 bits: ~50 times more error, which together
  with the accumulation error no longer fits under 2e-5; single TF32 (11
  bits) misses it outright;
* without its power-of-two scaling, the FP16 form would lose vectors and
  features outside FP16's range.
No CUDA code is involved.
"""
import numpy as np
import pytest

from oracle import gp_oracle as go
from synth import make_workload

C_FEAT = np.sqrt(5.0) * np.log2(np.e)   # x~ = c (x - mu) / l: u = c r
LN2 = np.log(2.0)
TOL = 2e-5


# ---- roundings of FP32 values ---------------------------------------------
def tf32_rna(x):
    b = np.asarray(x, np.float32).view(np.uint32)
    return ((b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def bf16_rne(x):
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def fp16_rne(x):
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float32)


def split(x, rnd):
    """hi = rnd(x), lo = rnd(x - hi) (x - hi exact in FP32)."""
    x = np.asarray(x, np.float32)
    hi = rnd(x)
    lo = rnd((x - hi).astype(np.float32))
    return hi.astype(np.float64), lo.astype(np.float64)


def fp16_scaled_split(x, axis=None):
    """FP16 split of 2^e x with max |x| 2^e in [2^14, 2^15), one e per
    `axis` slice (None: one for the whole array); returns unscaled parts."""
    x = np.asarray(x, np.float32)
    m = np.max(np.abs(x), axis=axis, keepdims=True)
    e = np.where(m > 0, 15 - np.frexp(np.where(m > 0, m, 1.0))[1], 0)
    xs = np.ldexp(x, e).astype(np.float32)
    hi, lo = split(xs, fp16_rne)
    return np.ldexp(hi, -e), np.ldexp(lo, -e)


def prepared(X, ell):
    mu = X.astype(np.float64).mean(axis=0)
    return ((X - mu) * (C_FEAT / ell)).astype(np.float32)


def khatv_from_parts(xh, xl, kparts, V, vparts, s, sigma2, single=False):
    """K-hat V from split parts, FP64 arithmetic.  Norms come from the same
    parts as the cross term (as on the GPU)."""
    xr = xh + (0.0 if single else xl)
    n = np.sum(xr * xr, axis=1)
    S = xh @ xh.T if single else xh @ xh.T + xh @ xl.T + xl @ xh.T
    u2 = np.maximum(n[:, None] + n[None, :] - 2.0 * S, 0.0)
    u = np.sqrt(u2)
    K = (1.0 + LN2 * u + (LN2 * u) ** 2 / 3.0) * np.exp2(-u)
    np.fill_diagonal(K, 1.0)
    kh, kl = kparts(K)
    vh, vl = vparts(V)
    O = kh @ vh.T if single else kh @ vh.T + kh @ vl.T + kl @ vh.T
    return s * O + sigma2 * np.asarray(V, np.float64).T


def relerr(got, ref):
    return float(np.max(np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)))


def form_error(name, X, ell, V, s, sigma2, scaled=True):
    Xt = prepared(X, ell)
    if name == "split_tf32":
        xh, xl = split(Xt, tf32_rna)
        kp = lambda K: (tf32_rna(K).astype(np.float64),
                        bf16_rne(K - tf32_rna(K)).astype(np.float64))
        # K_lo is rounded to BF16 for its product with V_hi (the GPU also
        # rounds that V_hi to BF16, a 2^-20 effect left out here)
        vp = lambda V: split(V, tf32_rna)
        out = khatv_from_parts(xh, xl, kp, V, vp, s, sigma2)
    elif name == "split_f16":
        if scaled:
            xh, xl = fp16_scaled_split(Xt)
            kp = lambda K: tuple(np.ldexp(p, -14) for p in split(np.ldexp(K, 14), fp16_rne))
            vp = lambda V: fp16_scaled_split(V, axis=1)
        else:
            xh, xl = split(Xt, fp16_rne)
            kp = lambda K: split(K, fp16_rne)
            vp = lambda V: split(V, fp16_rne)
        out = khatv_from_parts(xh, xl, kp, V, vp, s, sigma2)
    elif name == "split_bf16":
        xh, xl = split(Xt, bf16_rne)
        out = khatv_from_parts(xh, xl, lambda K: split(K, bf16_rne), V,
                               lambda V: split(V, bf16_rne), s, sigma2)
    elif name == "tf32":
        xh = tf32_rna(Xt).astype(np.float64)
        out = khatv_from_parts(xh, None, lambda K: (tf32_rna(K).astype(np.float64), None), V,
                               lambda V: (tf32_rna(V).astype(np.float64), None), s, sigma2,
                               single=True)
    else:
        raise ValueError(name)
    ref = go.khat_matmul(X, np.asarray(V, np.float64).T, ell, s, sigma2)
    return relerr(out, ref)


@pytest.fixture(scope="module")
def problem():
    w = make_workload("gp2k", N=1024)
    V = np.random.default_rng(3).standard_normal((4, w.N)).astype(np.float32)
    return w, V


def test_split_tf32_and_f16_keep_22_bits(problem):
    w, V = problem
    e_tf32 = form_error("split_tf32", w.X, w.lengthscale, V, 1.0, w.sigma2)
    e_f16 = form_error("split_f16", w.X, w.lengthscale, V, 1.0, w.sigma2)
    assert e_tf32 < 0.1 * TOL, e_tf32
    assert e_f16 < 0.1 * TOL, e_f16


def test_sixteen_and_eleven_bit_forms_lose_the_margin(problem):
    w, V = problem
    e_f16 = form_error("split_f16", w.X, w.lengthscale, V, 1.0, w.sigma2)
    e_bf16 = form_error("split_bf16", w.X, w.lengthscale, V, 1.0, w.sigma2)
    e_tf32 = form_error("tf32", w.X, w.lengthscale, V, 1.0, w.sigma2)
    assert e_bf16 > 20 * e_f16 and e_bf16 > 0.25 * TOL, (e_bf16, e_f16)
    assert e_tf32 > 10 * TOL, e_tf32


def test_f16_scaling_covers_extreme_vectors(problem):
    w, V = problem
    for factor in (1e-30, 1e25):
        Vx = (V.astype(np.float64) * factor).astype(np.float32)
        assert form_error("split_f16", w.X, w.lengthscale, Vx, 1.0, w.sigma2) < 0.1 * TOL
    # without the per-vector scale, 1e-30 underflows to zero and 1e25
    # overflows in FP16
    with np.errstate(over="ignore", invalid="ignore"):
        Vs = (V.astype(np.float64) * 1e-30).astype(np.float32)
        assert form_error("split_f16", w.X, w.lengthscale, Vs, 1.0, w.sigma2, scaled=False) > 0.5
        Vb = (V.astype(np.float64) * 1e25).astype(np.float32)
        assert not np.isfinite(form_error("split_f16", w.X, w.lengthscale, Vb, 1.0, w.sigma2,
                                          scaled=False))


def test_f16_scaling_covers_features_beyond_fp16_range():
    """Lengthscales of 1e-5: |x~| ~ 3e5 > 65504, every pair far apart (K = I)."""
    rng = np.random.default_rng(9)
    X = rng.standard_normal((400, 12)).astype(np.float32)
    ell = rng.uniform(0.5, 2.0, 12) * 1e-5
    V = rng.standard_normal((3, 400)).astype(np.float32)
    assert form_error("split_f16", X, ell, V, 1.3, 1e-2) < 0.1 * TOL
    with np.errstate(over="ignore", invalid="ignore"):
        assert not np.isfinite(form_error("split_f16", X, ell, V, 1.3, 1e-2, scaled=False))
