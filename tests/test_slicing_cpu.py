"""Host checks of the error-free slicing behind the FP64-class tensor-core products.

The tall products after the sketch (T = Y R^-1, H = Y D, Psi H, the Gram T* T, X) are formed
from BF16 slices: each row of the left operand and each column of the right one is scaled
by its largest power of two 2^e and cut into eight base-64 digits, the slice products of
the levels a + b <= 9 are summed exactly, and the levels are combined in double-float
(Ozaki, Ogita, Oishi and Rump 2012; the method computes these products in FP64).  These
tests restate the digit rules in exact rational arithmetic and check the properties the
scheme rests on:

* the digits reproduce the value rounded at 2^-48 of its scale, with |t_1| <= 64 and
  |t_a| <= 32 after (FP64 values: 48-bit integer split into two 24-bit halves; FP32 values:
  digits taken directly);
* a pre-scaled slice t 2^-6(a-1) is exact in BF16;
* every level sum stays below 2^24 for K <= 1536 real terms, so FP32 accumulation of a
  level is exact whatever the order;
* the product of the truncated sums is within 2^-46.53 of |row scale| |column scale| per
  term of the exact product (remainders 2^-49 per operand, dropped levels 10..16).
"""
import math
import random
from fractions import Fraction

import numpy as np

S, BETA, LEV_MAX = 8, 6, 9


def exp_of(v):
    """Exponent e with |v| < 2^e (frexp's), 0 for zero."""
    return 0 if v == 0 else math.frexp(v)[1]


def _digits4(y):
    """Four base-64 digits of y (|y| <= 1, a multiple of 2^-24), rounding half to even."""
    t = []
    for _ in range(4):
        y *= 64
        r = round(y)   # Fraction: half to even, as rintf
        y -= r
        t.append(int(r))
    assert y == 0
    return t


def digits_fp64(v, e):
    """Digits of y = v 2^-e for an FP64 v: Y = y 2^48 rounded half away from zero, split as
    Y = H 2^24 + L with L in [-2^23, 2^23), then four digits of each half."""
    y = Fraction(v) * Fraction(2) ** (48 - e)
    mag = math.floor(abs(y) + Fraction(1, 2))
    Y = -mag if v < 0 else mag
    L = Y & 0xFFFFFF
    if L >= 0x800000:
        L -= 0x1000000
    H = (Y - L) >> 24
    return _digits4(Fraction(H, 1 << 24)) + _digits4(Fraction(L, 1 << 24)), Y


def digits_fp32(v, e):
    """Digits of y = v 2^-e for an FP32 v, taken directly (exact in FP32: y has 24 bits)."""
    y = Fraction(float(np.float32(v))) * Fraction(2) ** (-e)
    t = []
    for _ in range(S):
        y *= 64
        r = round(y)
        y -= r
        t.append(int(r))
    return t


def value_of(t, e):
    return sum(Fraction(ta) * Fraction(2) ** (-BETA * (a + 1)) for a, ta in enumerate(t)) * Fraction(2) ** e


def _samples(rng, n):
    vals = [0.0, 1.0, -1.0, 0.5, -0.75, 2.0 ** -60, -(2.0 ** 40) * (1 - 2.0 ** -53)]
    for _ in range(n):
        vals.append(rng.uniform(-1, 1) * 2.0 ** rng.randint(-40, 40))
    return vals


def test_fp64_digits_reproduce_the_rounded_value_within_bounds():
    rng = random.Random(3)
    for v in _samples(rng, 400):
        e = exp_of(v) + rng.randint(0, 12)   # a row scale at or above the element's own
        t, Y = digits_fp64(v, e)
        assert abs(t[0]) <= 64 and all(abs(x) <= 32 for x in t[1:]), (v, e, t)
        assert value_of(t, e) == Fraction(Y) * Fraction(2) ** (e - 48)
        assert abs(value_of(t, e) - Fraction(v)) <= Fraction(2) ** (e - 49)


def test_fp64_digits_at_the_split_ties():
    # Y with L = -2^23 (kept) and L = 2^23 (moved into H): both halves stay within bounds
    for H, L in ((12345, -(1 << 23)), (-777, 1 << 23), ((1 << 24) - 1, (1 << 23) - 1), (0, 1 << 23)):
        Y = H * (1 << 24) + L
        v = float(Fraction(Y) * Fraction(2) ** -48)   # exact: |Y| < 2^48
        t, Y2 = digits_fp64(v, 0)
        assert Y2 == Y
        assert abs(t[0]) <= 64 and all(abs(x) <= 32 for x in t[1:])
        assert value_of(t, 0) == Fraction(v)


def test_fp32_digits_reproduce_the_value_rounded_at_2_pow_minus_48():
    rng = random.Random(5)
    for v in _samples(rng, 400):
        v32 = float(np.float32(v))
        e = exp_of(v32) + rng.randint(0, 30)
        t = digits_fp32(v32, e)
        assert abs(t[0]) <= 64 and all(abs(x) <= 32 for x in t[1:]), (v32, e, t)
        assert abs(value_of(t, e) - Fraction(v32)) <= Fraction(2) ** (e - 49)
        if exp_of(v32) - 24 >= e - 48:   # all 24 bits lie above 2^-48 of the scale: exact
            assert value_of(t, e) == Fraction(v32)


def test_prescaled_slices_are_exact_in_bf16():
    for a in range(S):
        for t in range(-64, 65):
            x = np.float32(t * 2.0 ** (-BETA * a))
            assert float(x) == t * 2.0 ** (-BETA * a)
            assert int(x.view(np.uint32)) & 0xFFFF == 0   # the BF16 pattern is the upper half


def test_every_level_sum_is_exact_in_fp32_for_k_up_to_1536():
    for lev in range(2, LEV_MAX + 1):
        bound = sum((64 if a == 1 else 32) * (64 if lev - a == 1 else 32)
                    for a in range(1, S + 1) if 1 <= lev - a <= S)
        assert bound * 1536 < 2 ** 24, lev
    assert 10240 * 1638 < 2 ** 24 <= 10240 * 1639   # level 9 sets the limit


def _sliced_product(A, B, a_fp32):
    """C from the slices of A (rows) and B (columns): exact level sums for levels 2..9."""
    m, K = A.shape
    N = B.shape[1]
    ea = [max(exp_of(float(x)) for x in A[i]) for i in range(m)]
    fb = [max(exp_of(float(x)) for x in B[:, j]) for j in range(N)]
    ta = [[(digits_fp32(A[i, k], ea[i]) if a_fp32 else digits_fp64(float(A[i, k]), ea[i])[0])
           for k in range(K)] for i in range(m)]
    ub = [[digits_fp64(float(B[k, j]), fb[j])[0] for k in range(K)] for j in range(N)]
    C = [[Fraction(0)] * N for _ in range(m)]
    for i in range(m):
        for j in range(N):
            total = Fraction(0)
            for lev in range(2, LEV_MAX + 1):
                s = 0
                for a in range(1, S + 1):
                    b = lev - a
                    if 1 <= b <= S:
                        s += sum(ta[i][k][a - 1] * ub[j][k][b - 1] for k in range(K))
                assert abs(s) < 2 ** 24
                total += Fraction(s) * Fraction(2) ** (-BETA * lev)
            C[i][j] = total * Fraction(2) ** (ea[i] + fb[j])
    return C, ea, fb


def test_sliced_product_is_within_the_truncation_bound():
    rng = np.random.default_rng(11)
    m, K, N = 3, 48, 4
    for a_fp32 in (False, True):
        A = rng.standard_normal((m, K)) * np.exp2(rng.integers(-20, 20, size=(m, 1)))
        A *= np.exp2(rng.integers(-8, 1, size=(m, K)))   # spread within each row
        if a_fp32:
            A = A.astype(np.float32)
        B = rng.standard_normal((K, N)) * np.exp2(rng.integers(-20, 20, size=(1, N)))
        C, ea, fb = _sliced_product(A, B, a_fp32)
        per_term = Fraction(2) ** -48 + sum(
            Fraction((64 if a == 1 else 32) * (64 if lev - a == 1 else 32)) * Fraction(2) ** (-BETA * lev)
            for lev in range(LEV_MAX + 1, 2 * S + 1) for a in range(1, S + 1) if 1 <= lev - a <= S)
        assert float(per_term) < 2.0 ** -46.5
        for i in range(m):
            for j in range(N):
                exact = sum(Fraction(float(A[i, k])) * Fraction(float(B[k, j])) for k in range(K))
                err = abs(C[i][j] - exact)
                assert err <= K * per_term * Fraction(2) ** (ea[i] + fb[j]), (i, j)
                # typical: far below the worst case (relative to the scale of the terms)
                scale = sum(abs(Fraction(float(A[i, k])) * Fraction(float(B[k, j]))) for k in range(K))
                assert float(err / scale) < 1e-13
