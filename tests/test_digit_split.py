"""The arithmetic of the digit-split kernel sums, emulated step by step on the CPU.

The tensor-core coupling and near field write each double-float kernel entry
K = kh + kl (|kl| <= ulp(kh)/2), scaled by 2^-E into (-1/2, 1/2), and each
vector value q' in (-1/2, 1/2) as six round-to-nearest 8-bit digits; digit
products are summed exactly per level L = s + t on the tensor cores, and the
level sums are folded into double-float (levels 0-2 by TwoSums, levels 3-5 as
a float32 tail).  This file checks the
claims that exactness rests on, with the kernel's float32 operations emulated:
every emulated operation below is exact in float64 before one rounding to
float32 (products by powers of two, sums of at most ~41 significant bits), so
the emulation rounds as the GPU's single-rounding FMA does.

  * entry digits: |a_s| <= 128 except the fourth (it also takes lo(K)),
    |a_3| <= 256; every digit is an integer exact in bf16 (<= 8 significant
    bits); the six digits give K 2^-E to 3 * 2^-49 (the last remainder,
    2^-49, plus the one rounding where lo(K) enters the fourth digit, 2^-48);
  * vector digits (FP64): |b_t| <= 128, reconstruction to 2^-49;
  * level sums: at most 6 products per source, one of them with a_3, so 128
    sources stay below 2^24 (exact FP32 integers);
  * the fold of the six level sums (integers below 2^24) into a double-float
    value is off by at most 2^-22 units of level 0, i.e. 2^-46 of a
    full-scale level sum: the TwoSums of levels 0-2 are exact, and only the
    float32 tail (levels 3-5, weight 2^-24) and the low part round.
"""
from fractions import Fraction

import numpy as np

F = np.float32
SHIFT = F(12582912.0)  # 1.5 * 2^23: x + SHIFT - SHIFT rounds |x| < 2^22 to an integer


def fma(a, b, c):
    return F(np.float64(a) * np.float64(b) + np.float64(c))


def entry_digits(kh, kl, E):
    """The kernel's split of K = kh + kl at exponent E (float32 operations)."""
    sc0 = F(2.0 ** (8 - E))
    d = []
    d0 = F(fma(kh, sc0, SHIFT) - SHIFT)
    r = fma(kh, sc0, -d0)
    d.append(d0)
    for s in range(1, 6):
        if s == 3:
            x = fma(r, F(256.0), F(kl * F(sc0 * F(16777216.0))))
            ds = F(F(x + SHIFT) - SHIFT)
            r = F(x - ds)
        else:
            ds = F(fma(r, F(256.0), SHIFT) - SHIFT)
            r = fma(r, F(256.0), -ds)
        d.append(ds)
    return d


def vector_digits(q):
    """The FP64 split of q' in (-1/2, 1/2)."""
    x, d = float(q), []
    for _ in range(6):
        x *= 256.0
        di = float(np.rint(x))
        x -= di
        d.append(di)
    return d


def bf16_exact(v):
    v = abs(int(v))
    return v == 0 or v.bit_length() - (v & -v).bit_length() + 1 <= 8


def _two_sum_ordered(a, b):
    big, small = (a, b) if abs(a) >= abs(b) else (b, a)
    s = F(a + b)
    return s, F(small - F(s - big))


def test_entry_digits_bounds_and_reconstruction():
    rng = np.random.default_rng(9100)
    worst3, worst, err = 0.0, 0.0, 0.0
    for _ in range(20000):
        K = rng.uniform(0.05, 1.0) * 2.0 ** int(rng.integers(-20, 20))
        kh = F(K)
        kl = F(K - float(kh))
        bound = K * rng.uniform(1.0, 4.0)           # any valid upper bound of |K| over the row
        E = int(np.floor(np.log2(bound * (1 + 1e-6)))) + 2  # bound 2^-E in [1/4, 1/2)
        d = entry_digits(kh, kl, E)
        assert all(float(x).is_integer() and bf16_exact(x) for x in d)
        worst3 = max(worst3, abs(float(d[3])))
        worst = max(worst, max(abs(float(x)) for i, x in enumerate(d) if i != 3))
        rec = sum(Fraction(float(x)) * Fraction(1, 2 ** (8 * (i + 1))) for i, x in enumerate(d))
        exact = (Fraction(float(kh)) + Fraction(float(kl))) * Fraction(2) ** (-E)
        err = max(err, abs(float(rec - exact)))
    assert worst <= 128 and worst3 <= 256
    assert err <= 3 * 2.0 ** -49


def test_vector_digits_bounds_and_reconstruction():
    rng = np.random.default_rng(9101)
    for q in np.concatenate([rng.uniform(-0.5, 0.5, 5000), [0.4999999999, -0.4999999999, 0.0, 2.0 ** -60]]):
        d = vector_digits(q)
        assert all(abs(x) <= 128 and bf16_exact(x) for x in d)
        rec = sum(Fraction(x) * Fraction(1, 2 ** (8 * (i + 1))) for i, x in enumerate(d))
        assert abs(float(rec - Fraction(float(q)))) <= 2.0 ** -49


def test_level_sums_stay_below_2_pow_24():
    # worst case: every digit at its largest magnitude, all of one sign
    a = [128, 128, 128, 256, 128, 128]
    b = [128] * 6
    per_source = max(sum(a[s] * b[L - s] for s in range(6) if 0 <= L - s < 6) for L in range(6))
    assert per_source == 7 * 2 ** 14
    assert 128 * per_source < 2 ** 24


def test_fold_of_level_sums_is_double_float_accurate():
    """The flush: C_0 + 2^-8 C_1 + 2^-16 C_2 by ordered TwoSums, the tail
    C_3 + 2^-8 C_4 + 2^-16 C_5 in float32 at weight 2^-24."""
    rng = np.random.default_rng(9102)
    worst = 0.0
    for _ in range(5000):
        C = [F(int(v)) for v in rng.integers(-(2 ** 24) + 1, 2 ** 24, 6)]
        tail = fma(C[5], F(1.0 / 65536.0), fma(C[4], F(1.0 / 256.0), C[3]))
        h, l = _two_sum_ordered(C[0], F(C[1] * F(1.0 / 256.0)))
        h, e2 = _two_sum_ordered(h, F(C[2] * F(1.0 / 65536.0)))
        l = fma(tail, F(1.0 / 16777216.0), F(l + e2))
        got = Fraction(float(h)) + Fraction(float(l))
        exact = sum(Fraction(int(c)) * Fraction(1, 2 ** (8 * i)) for i, c in enumerate(C))
        worst = max(worst, float(abs(got - exact)))
    assert worst <= 2.0 ** -22
