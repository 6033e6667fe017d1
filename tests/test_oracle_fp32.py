"""Pins for the binary32 emulation (oracle.fp32) against exact rationals."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import fp32


def round_to_f32(x: Fraction) -> np.float32:
    """Correct round-to-nearest-even of an exact rational to binary32,
    chosen among the three binary32 values nearest to float(x)."""
    r0 = np.float32(float(x))
    with np.errstate(over="ignore"):
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


# Property-based pins over the whole finite binary32 range: subnormals,
# zeros, extreme exponents and near-total cancellation, which the random
# draws above (exponents within +-30) do not reach.  Deterministic
# (derandomized, no example database), so a failure reproduces.  An
# unfused multiply-add (product rounded before the sum) fails both fma
# properties; the binary64 double rounding onto a binary32 midpoint is
# too rare for random draws and is pinned by the constructed cases above.
hypothesis = pytest.importorskip("hypothesis")
from hypothesis import assume, given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

F32_MAX = Fraction(float(np.finfo(np.float32).max))
_floats32 = st.floats(width=32, allow_nan=False, allow_infinity=False)
_settings = settings(max_examples=2500, deadline=None, derandomize=True, database=None)


@_settings
@given(_floats32, _floats32, _floats32)
def test_fma32_property_whole_range(a, b, c):
    x = Fraction(a) * Fraction(b) + Fraction(c)
    assume(abs(x) < F32_MAX)
    got = fp32.fma32(np.float32(a), np.float32(b), np.float32(c))
    assert got == round_to_f32(x)


@st.composite
def _cancelling(draw):
    # c within a few binary32 ulps of -a*b: the sum keeps only the low bits
    # of the exact product
    a = draw(st.floats(width=32, min_value=2.0 ** -60, max_value=2.0 ** 60))
    b = draw(st.floats(width=32, min_value=2.0 ** -60, max_value=2.0 ** 60))
    a = a * draw(st.sampled_from([-1.0, 1.0]))
    c = -np.float32(np.float64(a) * np.float64(b))
    for _ in range(draw(st.integers(0, 3))):
        c = np.nextafter(c, np.float32(draw(st.sampled_from([-np.inf, np.inf]))))
    return np.float32(a), np.float32(b), np.float32(c)


@_settings
@given(_cancelling())
def test_fma32_property_cancellation(abc):
    a, b, c = abc
    x = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    assert fp32.fma32(a, b, c) == round_to_f32(x)


@_settings
@given(_floats32, _floats32)
def test_binary_ops_property_whole_range(a, b):
    fa, fb = Fraction(a), Fraction(b)
    for op, exact in ((fp32.add32, fa + fb), (fp32.sub32, fa - fb), (fp32.mul32, fa * fb)):
        if abs(exact) < F32_MAX:
            assert op(np.float32(a), np.float32(b)) == round_to_f32(exact)
