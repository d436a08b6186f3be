"""The numpy FP32 fma emulation against exact rational arithmetic."""
from fractions import Fraction

import numpy as np

from fp32util import fma32


def exact_round_f32(fr: Fraction) -> np.float32:
    """Round a rational to float32 (nearest, ties to even) by bracketing."""
    x = np.float32(float(fr))  # within one ulp
    cands = [np.nextafter(x, np.float32(-np.inf)), x, np.nextafter(x, np.float32(np.inf))]
    best = min(cands, key=lambda v: (abs(Fraction(float(v)) - fr),
                                     int(np.frombuffer(np.float32(v).tobytes(), np.uint32)[0]) & 1))
    return np.float32(best)


def test_fma32_matches_exact_rounding():
    rng = np.random.default_rng(0)
    a = rng.uniform(-2, 2, 3000).astype(np.float32)
    b = rng.uniform(-2, 2, 3000).astype(np.float32)
    c = (rng.uniform(-2, 2, 3000) * 10.0 ** rng.integers(-8, 3, 3000)).astype(np.float32)
    got = fma32(a, b, c)
    for i in range(a.size):
        want = exact_round_f32(Fraction(float(a[i])) * Fraction(float(b[i])) + Fraction(float(c[i])))
        assert got[i] == want, (a[i], b[i], c[i])


def test_fma32_midpoint_cases():
    # a*b + c lands within 2^-60 of a float32 midpoint: the float64 sum is the
    # midpoint, the exact value is not, and the error term must decide.
    one = np.float32(1.0)
    eps = np.float32(2.0 ** -24)
    a = np.array([one + np.float32(2.0 ** -23)] * 2, np.float32)
    b = np.array([one + eps * 0 + np.float32(2.0 ** -23), one - np.float32(2.0 ** -23)], np.float32)
    c = np.array([np.float32(2.0 ** -30), np.float32(-(2.0 ** -30))], np.float32)
    got = fma32(a, b, c)
    for i in range(2):
        want = exact_round_f32(Fraction(float(a[i])) * Fraction(float(b[i])) + Fraction(float(c[i])))
        assert got[i] == want
