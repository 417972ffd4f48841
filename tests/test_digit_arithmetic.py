"""The arithmetic of the split-BF16 digit products, checked on the CPU with exact rational
arithmetic (a model of the design, independent of the GPU library and of the oracle).

A value x with |x| < 2^e is written as 2^e sum_{k<=S} d_k 2^{-7k}: |x| 2^{-e} rounded to
7S fractional bits (half up), split into base-128 digits and re-centred from the least
significant end.  Claims checked here: the digits are small integers (exact in bf16),
the representation error is at most 2^{e-7S-1}, an exact FP32 chunk of 960 digit products
cannot overflow 2^24, and keeping the slice pairs s + t <= S + 1 of a product leaves an
error of order 2^{-7S} of the row and column scales (dropping one more diagonal does not).
"""
from fractions import Fraction

import numpy as np
import pytest


def _exponent(vmax: float) -> int:
    """Smallest e with vmax < 2^e (0 for vmax == 0)."""
    if vmax == 0.0:
        return 0
    m, ex = np.frexp(vmax)  # vmax = m 2^ex, m in [0.5, 1)
    return int(ex)


def _digits(x: float, e: int, S: int):
    """Balanced digits of x (|x| < 2^e) from integer operations on the significand."""
    m, ex = np.frexp(abs(x))
    mant = int(np.ldexp(m, 53))          # |x| = mant 2^(ex - 53), mant < 2^53
    eu = int(ex) - 53
    sh_last = e - eu - 7 * S
    if sh_last >= 1:
        mant += 1 << (sh_last - 1)       # round half up at the last digit
    d = []
    for k in range(1, S + 1):
        sh = e - eu - 7 * k
        w = mant >> sh if sh >= 0 else mant << (-sh)
        d.append(w if k == 1 else w & 127)
    for k in range(S, 1, -1):
        if d[k - 1] >= 64:
            d[k - 1] -= 128
            d[k - 2] += 1
    return [-v for v in d] if x < 0 else d


def _value(d, e):
    return sum(Fraction(dk) * Fraction(2) ** (e - 7 * (k + 1)) for k, dk in enumerate(d))


@pytest.mark.parametrize("S", [1, 2, 3, 5, 7, 8])
def test_digits_are_small_integers_and_reconstruct_within_half_a_unit(S):
    rng = np.random.default_rng(40 + S)
    xs = np.concatenate([rng.standard_normal(300) * np.exp(rng.uniform(-30, 30, 300)),
                         [1.0, -1.0, 0.5, 2.0 ** -40, 1 - 2.0 ** -53, -(1 - 2.0 ** -52)]])
    for x in xs:
        e = _exponent(abs(x)) + int(rng.integers(0, 3))  # rows share e: |x| may be well below 2^e
        d = _digits(float(x), e, S)
        mag = d if x >= 0 else [-v for v in d]              # digits of |x|
        assert 0 <= mag[0] <= 129 and all(-64 <= v <= 63 for v in mag[1:])
        assert all(abs(v) <= 256 for v in d)            # integers of <= 8 bits: exact in bf16
        err = abs(_value(d, e) - Fraction(float(x)))
        assert err <= Fraction(2) ** (e - 7 * S - 1)


def test_exact_fp32_chunk_cannot_overflow():
    # |d_1| <= 129, |d_k| <= 64: the largest digit product is 129^2; 960 of them stay below
    # 2^24, where every integer is exact in FP32
    assert 960 * 129 * 129 < 2 ** 24
    assert 961 * 129 * 129 > 2 ** 24 - 2 ** 20  # 960 is near the limit: chunks cannot grow much


def _product_model(A, B, S, keep):
    """sum over kept pairs of 2^{e_i + f_j - 7(s+t)} (D_s^A D_t^B)_ij, exactly."""
    M, K = A.shape
    N = B.shape[1]
    e = [_exponent(float(np.max(np.abs(A[i])))) for i in range(M)]
    f = [_exponent(float(np.max(np.abs(B[:, j])))) for j in range(N)]
    DA = [[_digits(float(A[i, k]), e[i], S) for k in range(K)] for i in range(M)]
    DB = [[_digits(float(B[k, j]), f[j], S) for k in range(K)] for j in range(N)]
    C = [[Fraction(0)] * N for _ in range(M)]
    for i in range(M):
        for j in range(N):
            acc = Fraction(0)
            for s in range(1, S + 1):
                for t in range(1, S + 1):
                    if not keep(s, t):
                        continue
                    chunk = sum(DA[i][k][s - 1] * DB[j][k][t - 1] for k in range(K))  # exact integer
                    acc += Fraction(chunk) * Fraction(2) ** (e[i] + f[j] - 7 * (s + t))
            C[i][j] = acc
    return C, e, f


@pytest.mark.parametrize("S", [2, 4, 7, 8])
def test_pairs_up_to_s_plus_t_equal_S_plus_1_give_the_stated_error(S):
    rng = np.random.default_rng(50 + S)
    M, N, K = 4, 3, 24
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-6, 6, (M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-6, 6, (1, N)))
    exact = [[sum(Fraction(float(A[i, k])) * Fraction(float(B[k, j])) for k in range(K))
              for j in range(N)] for i in range(M)]
    C, e, f = _product_model(A, B, S, lambda s, t: s + t <= S + 1)
    worst = 0.0
    for i in range(M):
        for j in range(N):
            bound = Fraction(K * (S + 3)) * Fraction(2) ** (e[i] + f[j] - 7 * S)
            worst = max(worst, float(abs(C[i][j] - exact[i][j]) / bound))
    assert worst <= 1.0
    if S <= 4:
        # dropping the diagonal s + t = S + 1 as well breaks the bound
        C2, _, _ = _product_model(A, B, S, lambda s, t: s + t <= S)
        worst2 = max(float(abs(C2[i][j] - exact[i][j]) /
                           (Fraction(K * (S + 3)) * Fraction(2) ** (e[i] + f[j] - 7 * S)))
                     for i in range(M) for j in range(N))
        assert worst2 > 1.0


@pytest.mark.parametrize("S", [2, 4, 7])
def test_gauss_form_error_is_the_sum_of_its_three_products_bounds(S):
    """The Gauss form of a complex product, A B = (Ar Br - Ai Bi) + i((Ar + Ai)(Br + Bi)
    - Ar Br - Ai Bi), with each real product taken by the kept slice pairs at its own row and
    column scales: the real part's error is within the bounds of two products, the imaginary
    part's within those of three; the scales of Ar + Ai and Br + Bi are at most twice the
    embedding's (max over |Re|, |Im| of the row or column), so the whole is within six times
    the embedding's bound K (S + 3) 2^{e_i + f_j - 7S}."""
    rng = np.random.default_rng(70 + S)
    M, N, K = 3, 3, 20
    A = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))) * np.exp(rng.uniform(-5, 5, (M, 1)))
    B = (rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))) * np.exp(rng.uniform(-5, 5, (1, N)))
    keep = lambda s, t: s + t <= S + 1  # noqa: E731
    Ar, Ai, Br, Bi = A.real.copy(), A.imag.copy(), B.real.copy(), B.imag.copy()
    P0, e0, f0 = _product_model(Ar, Br, S, keep)
    P1, e1, f1 = _product_model(Ai, Bi, S, keep)
    P2, e2, f2 = _product_model(Ar + Ai, Br + Bi, S, keep)
    bound = lambda e, f, i, j: Fraction(K * (S + 3)) * Fraction(2) ** (e[i] + f[j] - 7 * S)  # noqa: E731
    e_emb = [_exponent(float(np.max(np.maximum(np.abs(Ar[i]), np.abs(Ai[i]))))) for i in range(M)]
    f_emb = [_exponent(float(np.max(np.maximum(np.abs(Br[:, j]), np.abs(Bi[:, j]))))) for j in range(N)]
    for i in range(M):
        for j in range(N):
            re_x = sum(Fraction(float(Ar[i, k])) * Fraction(float(Br[k, j])) -
                       Fraction(float(Ai[i, k])) * Fraction(float(Bi[k, j])) for k in range(K))
            im_x = sum(Fraction(float(Ar[i, k])) * Fraction(float(Bi[k, j])) +
                       Fraction(float(Ai[i, k])) * Fraction(float(Br[k, j])) for k in range(K))
            # the FP64 rounding of the sums Ar + Ai, Br + Bi is a perturbation of the
            # operands below 2^-53 of their scales, far inside the 2^-7S bounds for S <= 7
            re_err = abs(P0[i][j] - P1[i][j] - re_x)
            im_err = abs(P2[i][j] - P0[i][j] - P1[i][j] - im_x)
            b0, b1, b2 = bound(e0, f0, i, j), bound(e1, f1, i, j), bound(e2, f2, i, j)
            rounding = Fraction(K * 4) * Fraction(2) ** (e_emb[i] + f_emb[j] - 52)
            assert re_err <= b0 + b1
            assert im_err <= b0 + b1 + b2 + rounding
            emb = bound(e_emb, f_emb, i, j)
            assert b0 + b1 + b2 <= 6 * emb
