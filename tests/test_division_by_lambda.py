"""The FP64 collision divides by a lattice velocity lambda that is no power of
two (the Euler scheme's lambda = 3) without a division instruction: with r the
correctly rounded reciprocal of lambda, q0 = RN(x r), e = RN(x - q0 lambda) (one
FMA, exact) and q = RN(e r + q0) (one FMA).  Markstein's theorem (IBM J. Res.
Dev. 34(1), 1990) says q is the correctly rounded quotient; this checks the
identity with exact rational arithmetic standing in for the three roundings,
so the kernel's FP64 path stays bit for bit the oracle's division."""
from fractions import Fraction

import numpy as np
import pytest


def rn(q: Fraction) -> float:
    """Round a rational to the nearest double, ties to even (CPython's int
    true division is correctly rounded)."""
    return float(q)


def markstein(x: float, lam: float, r: float) -> float:
    q0 = rn(Fraction(x) * Fraction(r))
    e = rn(Fraction(x) - Fraction(q0) * Fraction(lam))
    return rn(Fraction(e) * Fraction(r) + Fraction(q0))


LAMBDAS = [3.0, 1.5, 5.0, 7.0, 0.3, 2.5, 1.7, 9.81, 3.0000001, 6.0, 0.1]


@pytest.mark.parametrize("lam", LAMBDAS)
def test_one_correction_step_gives_the_correctly_rounded_quotient(lam):
    rng = np.random.default_rng(int(lam * 1000))
    r = 1.0 / lam  # correctly rounded reciprocal
    xs = list(rng.uniform(-1.0, 1.0, 1500) * 2.0 ** rng.integers(-900, 900, 1500))
    # exact multiples, values next to powers of two and to multiples of lambda
    for k in range(1, 200):
        m = k * lam
        xs += [m, np.nextafter(m, 0.0), np.nextafter(m, np.inf), -m, float(2.0 ** (k % 60 - 30))]
        xs += [np.nextafter(2.0 ** (k % 60 - 30), 0.0), np.nextafter(2.0 ** (k % 60 - 30), np.inf)]
    for x in xs:
        x = float(x)
        assert markstein(x, lam, r) == x / lam, (x, lam)


def test_the_identity_fails_without_the_correction():
    """The product alone is not enough: for lambda = 3 some quotients differ
    from x * RN(1/3), so the check above can tell a missing correction."""
    r = 1.0 / 3.0
    rng = np.random.default_rng(3)
    xs = rng.uniform(0.5, 2.0, 2000)
    assert any(rn(Fraction(float(x)) * Fraction(r)) != float(x) / 3.0 for x in xs)
