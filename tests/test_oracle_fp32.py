"""Pins for the binary32 emulation (oracle.fp32) against exact rationals."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import fp32


def round_to_f32(x: Fraction) -> np.float32:
    """Correct round-to-nearest-even of an exact rational to binary32,
    chosen among the three binary32 values nearest to float(x)."""
    r0 = np.float32(float(x))
    cands = [np.nextafter(r0, np.float32(-np.inf)), r0, np.nextafter(r0, np.float32(np.inf))]
    best = None
    for c in cands:
        if not np.isfinite(c):
            continue
        err = abs(Fraction(float(c)) - x)
        if best is None or err < best[0]:
            best = (err, c)
        elif err == best[0]:
            # tie: keep the even significand
            if int(np.array(c, np.float32).view(np.uint32)) % 2 == 0:
                best = (err, c)
    return best[1]


def _rand32(rng, n, lo=-8, hi=8):
    m = rng.uniform(1.0, 2.0, n) * rng.choice([-1, 1], n)
    e = rng.integers(lo, hi, n)
    return (m * 2.0 ** e).astype(np.float32)


def test_fma32_matches_exact_rounding_random():
    rng = np.random.default_rng(1)
    a, b, c = _rand32(rng, 3000), _rand32(rng, 3000), _rand32(rng, 3000)
    got = fp32.fma32(a, b, c)
    for k in range(len(a)):
        x = Fraction(float(a[k])) * Fraction(float(b[k])) + Fraction(float(c[k]))
        assert got[k] == round_to_f32(x), k


def test_fma32_double_rounding_cases():
    # a*b = +-(2^-24 - 2^-70): added to c in [1, 2) the binary64 sum rounds
    # onto the binary32 midpoint c +- 2^-24 while the exact value lies just
    # inside it, so ties-to-even on the binary64 sum is wrong for half of
    # the significand parities.
    rng = np.random.default_rng(7)
    n = 400
    c = rng.uniform(1.0, 2.0, n).astype(np.float32)
    a = np.full(n, 1.0 + 2.0 ** -23, dtype=np.float32)
    b = (rng.choice([-1.0, 1.0], n) * 2.0 ** -24 * (1.0 - 2.0 ** -23)).astype(np.float32)
    got = fp32.fma32(a, b, c)
    naive = (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)
    exact = np.array([round_to_f32(Fraction(float(a[k])) * Fraction(float(b[k])) + Fraction(float(c[k])))
                      for k in range(n)], np.float32)
    np.testing.assert_array_equal(got, exact)
    assert np.count_nonzero(naive != exact) > n // 8


@pytest.mark.parametrize("op,ref", [
    (fp32.add32, lambda x, y: x + y),
    (fp32.sub32, lambda x, y: x - y),
    (fp32.mul32, lambda x, y: x * y),
])
def test_binary_ops_match_exact_rounding(op, ref):
    rng = np.random.default_rng(3)
    a, b = _rand32(rng, 2000, -30, 30), _rand32(rng, 2000, -30, 30)
    got = op(a, b)
    for k in range(len(a)):
        assert got[k] == round_to_f32(ref(Fraction(float(a[k])), Fraction(float(b[k]))))
