"""Error bound of the reciprocal the FP64 basis smoothing uses for its
partition-of-unity scale (Sec. 5.1: every cell's basis values are divided by
their sum).

The kernel seeds r0 = 1 / x from the FP32 reciprocal of x's mantissa (seed
error below 2^-21 relative) and takes one third-order step of the series
1 / x = r0 (1 + e + e^2 + ...), e = 1 - x r0, as three fused multiply-adds.
Here the same three steps run in exact rational arithmetic with one rounding
to double per fused multiply-add, from seeds at the worst admitted error, and
the result must lie within one unit in the last place of 1 / x (the series'
truncation error e^3 is below 2^-63 relative)."""
from fractions import Fraction

import numpy as np


def _fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _seed(x, rel):
    """1 / x perturbed by rel, rounded to a 24-bit significand (an FP32 value
    scaled by a power of two)."""
    r = 1.0 / x * (1.0 + rel)
    m, e = np.frexp(r)
    return float(np.ldexp(np.round(m * 2.0**24) / 2.0**24, e))


def _series(x, r0):
    e = _fma(-x, r0, 1.0)
    return _fma(r0, _fma(e, e, e), r0)


def test_series_reciprocal_within_one_ulp():
    rng = np.random.default_rng(7)
    xs = np.ldexp(1.0 + rng.random(600), rng.integers(-1000, 1000, 600))
    xs = np.concatenate([xs, [1.0, 0.5, 0.75, 1.0 - 2.0**-52, 1.0 + 2.0**-52, 3.0, 6.135294117647059]])
    exact_hits = 0
    total = 0
    for x in xs:
        x = float(x)
        ref = Fraction(1) / Fraction(x)
        ulp = float(np.spacing(float(ref)))
        for rel in (2.0**-21, -2.0**-21, 2.0**-23, -3.0e-7, 0.0):
            r = _series(x, _seed(x, rel))
            err = abs(Fraction(r) - ref) / Fraction(ulp)
            assert err <= 1, (x, rel, float(err))
            exact_hits += r == float(ref)
            total += 1
    assert exact_hits >= 0.99 * total   # nearly always the correctly rounded quotient
