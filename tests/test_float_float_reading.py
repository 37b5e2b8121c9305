"""The float-float arithmetic of the Woodbury apply (reading 15), checked on
the CPU.

The device carries the preconditioner's factor L and D^{-1} as FP32 pairs
hi + lo and accumulates sum_a L_a y_a with a float-float multiply-add: the
product's rounding error recovered by an FMA (Dekker's two-product), the
sum's by Knuth's two-sum, the cross terms a_hi b_lo + a_lo b_hi in the low
word.  This test restates that step sequence with NumPy float32 scalars (every
operation rounded to FP32; an FMA as the exact double product plus one
rounding) and checks the accuracy it was chosen for: about 44 significant
bits, enough to survive the cancellation in z = D^{-1} r - L C^{-1} L^T D^{-1} r
that plain FP32 loses.
"""
import math

import numpy as np

F32 = np.float32


def _fma32(a, b, c):
    # a b is exact in FP64 for FP32 operands; one rounding of the sum
    return F32(float(a) * float(b) + float(c))


def _split(v):
    hi = F32(v)
    return hi, F32(v - float(hi))


def _ff_mac(sh, sl, ah, al, bh, bl):
    p = F32(ah * bh)
    e = _fma32(ah, bh, -p)
    e = _fma32(ah, bl, e)
    e = _fma32(al, bh, e)
    s = F32(sh + p)
    bb = F32(s - sh)
    err = F32(F32(sh - F32(s - bb)) + F32(p - bb))
    sl = F32(sl + F32(err + e))
    return s, sl


def _ff_dot(x, y):
    sh, sl = F32(0.0), F32(0.0)
    for xv, yv in zip(x, y):
        xh, xl = _split(xv)
        yh, yl = _split(yv)
        sh, sl = _ff_mac(sh, sl, xh, xl, yh, yl)
    return float(sh) + float(sl)


def test_float_float_dot_keeps_about_44_bits():
    rng = np.random.default_rng(11)
    x = rng.standard_normal(3000) * np.exp(rng.uniform(-3, 3, 3000))
    y = rng.standard_normal(3000)
    exact = math.fsum(float(a) * float(b) for a, b in zip(x, y))   # FP64 products, exactly summed
    scale = math.fsum(abs(float(a) * float(b)) for a, b in zip(x, y))
    ff = _ff_dot(x, y)
    f32 = float(np.sum((x.astype(F32) * y.astype(F32)).astype(F32), dtype=F32))
    assert abs(ff - exact) <= 2.0 ** -40 * scale
    # plain FP32 is some seven digits worse
    assert abs(f32 - exact) > 1e3 * abs(ff - exact)


def test_float_float_survives_the_woodbury_cancellation():
    # r - acc where acc agrees with r to seven digits: the difference keeps
    # most of its digits in float-float and none in FP32
    rng = np.random.default_rng(12)
    n = 64
    L = rng.standard_normal(n)
    w = rng.standard_normal(n)
    acc_exact = math.fsum(float(a) * float(b) for a, b in zip(L, w))
    r = acc_exact * (1.0 + 3e-7)
    diff_exact = r - acc_exact
    diff_ff = r - _ff_dot(L, w)
    diff_f32 = float(F32(r)) - float(np.sum((L.astype(F32) * w.astype(F32)).astype(F32), dtype=F32))
    assert abs(diff_ff - diff_exact) <= 1e-4 * abs(diff_exact)
    assert abs(diff_f32 - diff_exact) > 1e-2 * abs(diff_exact)
