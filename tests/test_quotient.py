"""The noise-variance quotient: RN(a / b) from the host's y = RN(1 / b) and one
Markstein correction (P. Markstein, IBM J. Res. Dev. 34(1), 1990), as the
kernel computes it: q0 = RN(a y), r = RN(a - b q0) (exact: one fused
multiply-add), q = RN(q0 + r y).  The rounding of every step is replayed with
exact rational arithmetic (float(Fraction) rounds to nearest even) and the
result is compared with the correctly rounded quotient."""
from fractions import Fraction

import numpy as np


def rn(x: Fraction) -> float:
    return float(x)


def markstein(a: float, b: float) -> float:
    y = rn(Fraction(1) / Fraction(b))
    q0 = rn(Fraction(a) * Fraction(y))
    r_exact = Fraction(a) - Fraction(b) * Fraction(q0)
    r = rn(r_exact)
    assert Fraction(r) == r_exact              # the remainder is exact
    return rn(Fraction(q0) + Fraction(r) * Fraction(y))


def test_markstein_quotient_is_correctly_rounded():
    rng = np.random.default_rng(2005)
    dens = []
    for w in (1, 3, 5, 7, 9, 15):
        for H, W in ((1, 1), (7, 9), (512, 512), (1620, 1620), (4096, 4096), (65535, 65535), (3, 60000)):
            dens.append(float(w ** 4 * H * W))
    checked = 0
    for b in dens:
        assert b < 2.0 ** 53
        for _ in range(300):
            # numerators: sums of local variances, from tiny to 2^100
            a = float(rng.integers(1, 2 ** 62)) * 2.0 ** int(rng.integers(-10, 40))
            assert markstein(a, b) == rn(Fraction(a) / Fraction(b))
            checked += 1
    assert checked == len(dens) * 300


def test_markstein_on_hard_ratios():
    # numerators just around multiples of the denominator and of half-ulps
    for b in (25.0 * 1620 * 1620, 625.0 * 4096 * 4096, 50625.0 * 65535 * 65535):
        for k in (1, 3, 1 << 20, (1 << 52) + 1):
            for da in (-2.0, -1.0, 0.0, 1.0, 2.0):
                a = float(k) * b + da
                assert markstein(a, b) == rn(Fraction(a) / Fraction(b))
