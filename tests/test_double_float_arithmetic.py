"""The double-float arithmetic of the wide-block Rayleigh-Ritz eigensolver, checked on the CPU
with exact rational arithmetic (a model of the design, independent of the GPU library and of
the oracle).

A real number is carried as hi + lo, two FP32 numbers with |lo| <= ulp(hi) / 2.  A product
of two such numbers is p = fl(ah bh) plus the error terms fma(ah, bh, -p) (exact),
+ ah bl + al bh (rounded); a sum of products keeps its error terms apart and folds them in
once (two-sum on the leading parts, a final fast two-sum).  Claims checked here: two-sum is
exact, the product's error term recovers ah bh - p exactly, and a rotation update
a x + b y of complex double-float values (real a, b; the form the eigensolver applies) is
within 2^-44 of the exact result relative to |a||x| + |b||y|, i.e. about 47 significand
bits, against FP64's 53.
"""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32


def _r(x):
    """Round a float64 (or exact float32 product held in float64) to FP32."""
    return f32(x)


def _fma(a, b, c):
    """fmaf(a, b, c) for FP32 a, b, c: the sum a b + c is formed exactly with fractions and
    rounded to FP32 through FP64 (a double rounding that can differ from fmaf in the last
    bit; exact whenever the result is representable, as for the product's error term)."""
    v = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    return _r(float(v))


def _two_sum(a, b):
    s = _r(float(a) + float(b))
    bb = _r(float(s) - float(a))
    err = _r(float(_r(float(a) - float(_r(float(s) - float(bb))))) + float(_r(float(b) - float(bb))))
    return s, err


def _prod(ah, al, bh, bl):
    p = _r(float(ah) * float(bh))
    e = _fma(ah, bh, -p)
    e = _fma(ah, bl, e)
    e = _fma(al, bh, e)
    return p, e


def _acc(a, b):
    s, err = _two_sum(a[0], b[0])
    return s, _r(float(_r(float(a[1]) + float(b[1]))) + float(err))


def _norm(a):
    s = _r(float(a[0]) + float(a[1]))
    return s, _r(float(a[1]) - float(_r(float(s) - float(a[0]))))


def _split(x):
    h = _r(x)
    return h, _r(x - float(h))


def _val(d):
    return Fraction(float(d[0])) + Fraction(float(d[1]))


def test_two_sum_is_exact():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        a, b = f32(rng.standard_normal() * 2.0 ** rng.integers(-20, 20)), f32(rng.standard_normal())
        s, e = _two_sum(a, b)
        assert Fraction(float(s)) + Fraction(float(e)) == Fraction(float(a)) + Fraction(float(b))


def test_product_error_term_recovers_the_rounding_exactly():
    rng = np.random.default_rng(2)
    for _ in range(2000):
        a, b = f32(rng.standard_normal()), f32(rng.standard_normal() * 1e3)
        p = _r(float(a) * float(b))
        assert Fraction(float(p)) + Fraction(float(_fma(a, b, -p))) == Fraction(float(a)) * Fraction(float(b))


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_rotation_update_carries_about_47_bits(seed):
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(400):
        th = rng.uniform(0, np.pi / 2)
        a, b = _split(np.cos(th)), _split(-np.sin(th) if rng.random() < 0.5 else np.sin(th))
        x = (_split(rng.standard_normal()), _split(rng.standard_normal()))   # re, im
        y = (_split(rng.standard_normal() * 10), _split(rng.standard_normal() * 10))
        out = []
        for part in range(2):  # re and im: a x_part + b y_part
            s = _acc(_prod(a[0], a[1], x[part][0], x[part][1]), _prod(b[0], b[1], y[part][0], y[part][1]))
            out.append(_norm(s))
        for part in range(2):
            exact = _val(a) * _val(x[part]) + _val(b) * _val(y[part])
            scale = abs(_val(a) * _val(x[part])) + abs(_val(b) * _val(y[part]))
            err = abs(_val(out[part]) - exact)
            worst = max(worst, float(err / scale))
    assert worst <= 2.0 ** -44, worst
    assert worst > 2.0 ** -60  # the representation is not exact: the bound is about attained order
