"""Host-side pins of arithmetic identities the GPU kernels rely on.

The LU kernels form each multiplier x / piv as l = x * y with y = 1 / piv
(computed once per step), then one FMA correction l' = l + (x - piv*l) * y
(Markstein's quotient refinement).  The kernels' pivot choices depend on the
multipliers, so the claim that l' is the correctly rounded quotient -- in
particular that equal rows still cancel exactly -- is checked here in exact
rational arithmetic, independently of any GPU.
"""
import random
from fractions import Fraction

import numpy as np


def _fma(a, b, c):
    # one rounding of the exact a*b + c (float(Fraction) rounds to nearest even)
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _refined_quotient(x, p):
    y = 1.0 / p
    l = x * y
    return _fma(_fma(-p, l, x), y, l)


def test_refined_quotient_is_correctly_rounded_random():
    rng = random.Random(7)
    for _ in range(20000):
        p = rng.uniform(0.5, 1.0) * 2.0 ** rng.randint(-40, 40) * rng.choice((-1.0, 1.0))
        x = rng.uniform(-1.0, 1.0) * 2.0 ** rng.randint(-40, 40)
        assert _refined_quotient(x, p) == x / p, (x, p)


def test_refined_quotient_exact_cases():
    rng = random.Random(11)
    for _ in range(5000):
        p = rng.uniform(-1e3, 1e3)
        if p == 0.0:
            continue
        for k in (1.0, -1.0, 2.0, 0.5, 3.0, 0.0):
            x = k * p
            q = _refined_quotient(x, p)
            assert q == x / p, (x, p)
        # an equal row cancels exactly: x - l * piv == 0 with l = 1
        assert _fma(-_refined_quotient(p, p), p, p) == 0.0


def test_refined_quotient_hard_significands():
    # divisors whose significand is all ones or a power of two plus one ulp
    ps = [np.nextafter(2.0, 0.0), np.nextafter(1.0, 2.0), 3.0, 1.0 / 3.0, np.nextafter(1.0, 0.0) * 7.0]
    rng = random.Random(3)
    for p in ps:
        for _ in range(2000):
            x = rng.uniform(-4.0, 4.0)
            assert _refined_quotient(x, float(p)) == x / float(p), (x, p)


# ------------------------------------------------------------- slice digits
# The slicing kernel (split_kernel) writes the seven balanced base-256 digits
# q_p in [-128, 127] of a 54-bit fixed-point integer X (X = sum_p q_p
# 256^(6-p)) as the bytes of X + sum_p 128 256^p, each minus 128, and each
# digit's bf16 as the upper half of the FP32 (2^23 + byte) - (2^23 + 128).
# Both are checked here against the definition: digits taken one at a time
# from the least significant end.
_BIAS = sum(128 << (8 * p) for p in range(7))


def _digits_by_definition(X):
    out = [0] * 7
    for p in range(6, -1, -1):
        q = ((X + 128) & 255) - 128
        X = (X - q) >> 8
        out[p] = q
    assert X == 0
    return out


def _digits_by_bytes(X):
    Z = X + _BIAS
    assert 0 <= Z < 1 << 64
    return [((Z >> (8 * (6 - p))) & 255) - 128 for p in range(7)]


def test_balanced_digits_are_the_biased_bytes():
    rng = random.Random(5)
    edge = [0, 1, -1, 127, 128, -128, -129, (1 << 54) - 1, -((1 << 54) - 1), 1 << 53, -(1 << 53)]
    for X in edge + [rng.randint(-(1 << 54) + 1, (1 << 54) - 1) for _ in range(50000)]:
        d = _digits_by_definition(X)
        assert d == _digits_by_bytes(X), X
        assert all(-128 <= q <= 127 for q in d) and abs(d[0]) <= 64
        assert sum(q << (8 * (6 - p)) for p, q in enumerate(d)) == X


def test_digit_to_bf16_by_an_exact_fp32_subtraction():
    for b in range(256):
        f = np.float32(np.uint32(0x4B000000 | b).view(np.float32)) - np.float32(8388736.0)
        assert float(f) == b - 128
        bits = int(np.float32(f).view(np.uint32))
        assert bits & 0xFFFF == 0                              # exact in bf16
        assert (b != 128) or bits == 0                         # +0, not -0
