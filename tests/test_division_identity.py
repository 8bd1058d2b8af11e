"""The FMA-based division the set-up kernels use for quotients that share a divisor (the direct
interpolation weights of a row, all divided by its modified diagonal):
with y = RN(1/b), q0 = RN(a y), q1 = RN(q0 + RN(a - b q0) y) and q = RN(q1 + (a - b q1) y), the
result is RN(a/b) -- the oracle's correctly rounded division -- away from overflow and underflow
(q1 is a faithful quotient, so its remainder is exact, and Markstein's theorem applies).

Checked here in exact rational arithmetic on the host (no GPU code involved): Python floats give
correctly rounded 1/b, a*y and a/b, and Fraction forms each FMA's exact value and its single
rounding.  Operands span the exponent range the kernels use the identity in (|x| in
[2^-822, 2^776]; outside it they divide), with cases near powers of two and small-integer
ratios, where rounding is most delicate.  A single correction step is not enough in general:
q0 can be two ulps off, and then its remainder is not a floating-point number (checked too).
"""
import math
import random
from fractions import Fraction

import pytest


def fma_rn(x: float, y: float, z: float) -> float:
    """RN(x * y + z) with one rounding (what an FMA computes)."""
    return float(Fraction(x) * Fraction(y) + Fraction(z))


def two_step(a: float, b: float) -> float:
    y = 1.0 / b
    q0 = a * y
    q1 = fma_rn(fma_rn(-q0, b, a), y, q0)
    r1_exact = Fraction(a) - Fraction(b) * Fraction(q1)
    r1 = fma_rn(-q1, b, a)
    assert Fraction(r1) == r1_exact, "the faithful quotient's remainder must be exact"
    return fma_rn(r1, y, q1)


def log_uniform(rng: random.Random, lo: int, hi: int) -> float:
    return math.ldexp(1.0 + rng.random(), rng.randint(lo, hi)) * rng.choice((-1.0, 1.0))


def cases(seed):
    rng = random.Random(seed)
    out = []
    for _ in range(15000):  # quotients inside the safe range
        b = log_uniform(rng, -300, 300)
        out.append((b * log_uniform(rng, -300, 300), b))
    for _ in range(3000):  # divisors near powers of two, operands of a few bits
        b = math.ldexp(1.0, rng.randint(-60, 60)) * (1.0 + rng.choice((-1, 1)) * rng.randint(1, 64) * 2.0 ** -52)
        out.append((float(rng.randint(1, 1 << 20)) * rng.choice((-1.0, 1.0)), b))
    for _ in range(3000):  # full-width integer operands
        out.append((float(rng.randint(1, 1 << 53)), float(rng.randint(1, 1 << 53))))
    for n in range(1, 150):  # small-integer ratios such as 1/3, 2/3, 5/7
        for d in (3, 5, 6, 7, 9, 11, 13, 49, 97):
            out.append((float(n), float(d)))
    return [(a, b) for a, b in out if a != 0.0]


@pytest.mark.parametrize("seed", [0, 1])
def test_two_step_division_is_correctly_rounded(seed):
    for a, b in cases(seed):
        assert two_step(a, b) == a / b, (a, b)


def test_one_step_remainder_can_be_inexact():
    """Why the kernels correct twice: after one step from q0 = RN(a y) the remainder a - b q0
    is sometimes not a floating-point number (q0 two ulps off), outside Markstein's hypotheses."""
    inexact = 0
    for a, b in cases(0):
        q0 = a * (1.0 / b)
        r = Fraction(a) - Fraction(b) * Fraction(q0)
        inexact += Fraction(float(r)) != r
    assert inexact > 0


def test_interpolation_weight_shape():
    """The weights' own shape: -(alpha a_ij) / a~_ii with alpha = sn / sp, on values like the
    Poisson levels' (couplings near -1, diagonals 2-6 and their coarse-level sums)."""
    rng = random.Random(7)
    for _ in range(15000):
        alpha = -rng.uniform(0.5, 30.0) / -rng.uniform(0.5, 30.0)
        num = -(alpha * -rng.uniform(1e-3, 10.0))
        at = rng.uniform(0.5, 60.0)
        assert two_step(num, at) == num / at
