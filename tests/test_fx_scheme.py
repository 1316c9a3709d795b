"""CPU checks of the exact integer-digit products used for the FP64 passes over dense constraint
rows and the small E Y E products (not in the paper).

A value x with |x| 2^adj < 2^F is written as N = rint(x 2^(52 + adj - F)) = hi 2^26 + lo, with N
formed by integer shifts of the IEEE fields; a dot product sums hi hi' and hi lo' + lo hi' exactly
in 64-bit integers (at most 1024 terms per accumulator) and converts once to FP64.  These tests
emulate that arithmetic with Python integers and check it against exact rational arithmetic:
the rounding is to nearest, the digits stay in range, no accumulator overflows, and the result is
within K 2^-53 max|a| max|x| of the exact dot product (about what FP64 summation attains)."""
import math
import random
import struct
from fractions import Fraction

import numpy as np


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def expo(x):
    """e with |x| < 2^e, from the IEEE fields (x finite, nonzero)."""
    b = bits(abs(x))
    ex = (b >> 52) & 0x7FF
    if ex:
        return ex - 1022
    m = b & ((1 << 52) - 1)
    return (m.bit_length() - 1) - 1073


def fixed(x, adj, F):
    """rint(x 2^(52 + adj - F)) by integer shifts (halves away from zero)."""
    b = bits(x)
    ex = (b >> 52) & 0x7FF
    mnt = b & ((1 << 52) - 1)
    if ex:
        mnt |= 1 << 52
    if mnt == 0:
        return 0
    sh = (ex if ex else 1) - 1023 + adj - F
    if sh >= 0:
        n = mnt << sh
    elif sh <= -64:
        n = 0
    else:
        n = (mnt + (1 << (-sh - 1))) >> (-sh)
    return -n if b >> 63 else n


def split(n):
    hi = (n + (1 << 25)) >> 26
    return hi, n - (hi << 26)


def to_double(t):
    """The int64 accumulator converted to FP64 (round to nearest)."""
    assert -(1 << 63) <= t < (1 << 63)
    return float(t)


def digit_dot(a, x):
    e = max(expo(v) for v in a if v != 0)
    f = max(expo(v) for v in x if v != 0)
    acc, t1, t2, cnt = 0.0, 0, 0, 0
    for u, v in zip(a, x):
        h, l = split(fixed(u, 0, e))
        xh, xl = split(fixed(v, 0, f))
        assert abs(h) <= 1 << 26 and -(1 << 25) <= l < (1 << 25)
        t1 += h * xh
        t2 += h * xl + l * xh
        cnt += 1
        if cnt == 1024:
            acc += to_double(t1) * 2.0 ** -52 + to_double(t2) * 2.0 ** -78
            t1 = t2 = cnt = 0
    acc += to_double(t1) * 2.0 ** -52 + to_double(t2) * 2.0 ** -78
    return math.ldexp(acc, e + f)


def test_fixed_point_rounding_and_digits():
    rng = random.Random(3)
    for t in range(20000):
        x = rng.gauss(0.0, 1.0) * 10.0 ** rng.uniform(-300, 300)
        if t % 100 == 0:
            x = 5e-324 * rng.randint(1, 10 ** 15) * rng.choice([1, -1])   # subnormal
        e = expo(x)
        assert 2.0 ** (e - 1) <= abs(x) < 2.0 ** e
        adj = rng.randint(-5, 5)
        F = e + adj + rng.randint(0, 70)
        n = fixed(x, adj, F)
        exact = Fraction(x) * Fraction(2) ** (52 + adj - F)
        assert abs(n) <= 2 ** 52 and abs(Fraction(n) - exact) <= Fraction(1, 2)
        hi, lo = split(n)
        assert hi * 2 ** 26 + lo == n and abs(hi) <= 2 ** 26 and -(2 ** 25) <= lo < 2 ** 25


def test_digit_dot_product_error_bound():
    rng = np.random.default_rng(1)
    worst = 0.0
    for trial in range(16):
        K = int(rng.integers(1, 2500))
        a = rng.standard_normal(K) * 10.0 ** rng.uniform(-8, 8) * np.exp(rng.uniform(-3, 3, K))
        x = rng.standard_normal(K) * np.exp(rng.uniform(-5, 5, K))
        if trial % 5 == 0:
            a[rng.integers(0, K)] = 0.0
        got = digit_dot([float(v) for v in a], [float(v) for v in x])
        exact = sum(Fraction(float(u)) * Fraction(float(v)) for u, v in zip(a, x))
        bound = K * 2.0 ** -53 * float(np.max(np.abs(a))) * float(np.max(np.abs(x)))
        worst = max(worst, float(abs(Fraction(got) - exact)) / bound)
    assert worst <= 1.0, worst


def test_digit_dot_is_exact_on_small_integers():
    """Integer data whose products and sums are exact in FP64 come out exactly."""
    rng = np.random.default_rng(2)
    for _ in range(8):
        K = int(rng.integers(1, 3000))
        a = rng.integers(-1000, 1000, K).astype(float)
        x = rng.integers(-1000, 1000, K).astype(float)
        if not a.any() or not x.any():
            continue
        assert digit_dot(list(a), list(x)) == float(int(np.dot(a.astype(np.int64), x.astype(np.int64))))
