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
