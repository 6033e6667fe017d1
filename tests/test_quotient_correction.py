"""The binning kernel's binary64 quotient for cell spacings h that are not
powers of two: Markstein's fused multiply-add correction from y = RN(1/h),

    q0 = x y,  q1 = fma(fma(-q0, h, x), y, q0),  t = fma(fma(-q1, h, x), y, q1),

emulated here in exact rationals (each fused multiply-add rounds the exact
value once), must equal the IEEE binary64 division x / h.  The theorem's
premises are checked as well: q1 within one ulp of x / h and the last
residual exact.  Inputs cover random positions, quotients below 1 and
positions a few ulps either side of the faces k h, where a wrong rounding
would change the fine cell.  The chunk kernel's form, the product and one
step to a neighbour decided on exact integer midpoints, is checked on the
same inputs and next to powers of two."""
import math
from fractions import Fraction as Fr

import numpy as np


def _fma(a, b, c):
    return float(Fr(a) * Fr(b) + Fr(c))      # float(Fraction) rounds to nearest even


def _cases(rng, box, M):
    h = box / M
    xs = list(rng.uniform(0, box, 400)) + list(rng.uniform(0, h, 40))
    for k in rng.integers(0, M, 150):
        x = float(k) * h
        for d in (-2, -1, 1, 2):
            y = x
            for _ in range(abs(d)):
                y = float(np.nextafter(y, np.inf if d > 0 else -np.inf))
            if 0 < y < box:
                xs.append(y)
    return h, [float(x) for x in xs if x >= 2.0 ** -900]


def test_corrected_quotient_equals_ieee_division():
    rng = np.random.default_rng(2024)
    boxes = [23.0, 98.0, 17.0, 30.0, 1000.0 / 3.0, 0.7, 3.3e5] + list(rng.uniform(6.0, 600.0, 5))
    n = 0
    for box in boxes:
        for M in (max(1, int(box // 4)) << 6, 13, 1000):
            h, xs = _cases(rng, box, M)
            y = float(1 / Fr(h))
            for x in xs:
                q = Fr(x) / Fr(h)
                q0 = x * y
                q1 = _fma(_fma(-q0, h, x), y, q0)
                assert abs(Fr(q1) - q) < Fr(math.ulp(float(q))) or q == 0
                r = Fr(x) - Fr(q1) * Fr(h)
                assert Fr(float(r)) == r, "last residual not exact"
                assert _fma(float(r), y, q1) == x / h, (box, M, x)
                n += 1
    assert n > 20000


def test_single_correction_is_not_enough():
    # the product x y alone can miss the one-ulp premise, so the first
    # correction step is needed: box 23 in 13 cells (r_c = 1.5, no sub-cell
    # bits), where RN(1/h) is 0.41 ulp from 1/h (rounding allows 0.5)
    rng = np.random.default_rng(5)
    h = 23.0 / 13
    y = float(1 / Fr(h))
    far = 0
    for x in rng.uniform(0, 23.0, 4000):
        x = float(x)
        q = Fr(x) / Fr(h)
        if abs(Fr(x * y) - q) >= Fr(math.ulp(float(q))):
            far += 1
    assert far > 0


def _floor_from_product(x, y):
    """The keys kernel's shortcut: floor(x / h) from the one product t' = x y,
    or None where t' lies within 16 ulps of an integer (the kernel then takes
    the corrected quotient)."""
    t = x * y
    if t < 1.0:
        return None if t >= 1.0 - 16 * 2.0 ** -53 else 0
    q = math.floor(t)
    u = math.ulp(t)
    if t - q < 16 * u or (q + 1) - t <= 16 * u:
        return None
    return q


def test_floor_from_one_product_matches_the_division():
    # the shortcut's premise: t' = RN(x RN(1/h)) lies within 2.5 ulp of
    # RN(x / h), so away from integers (16 ulps) floor(t') = floor(x / h);
    # checked on random positions and on positions a few ulps either side of
    # the faces k h, where the shortcut must decline
    rng = np.random.default_rng(77)
    boxes = [23.0, 98.0, 17.0, 30.0, 1000.0 / 3.0, 0.7, 3.3e5] + list(rng.uniform(6.0, 600.0, 5))
    taken = declined = 0
    for box in boxes:
        for M in (max(1, int(box // 4)) << 6, 13, 1000):
            h, xs = _cases(rng, box, M)
            y = float(1 / Fr(h))
            for x in xs:
                exact = Fr(x) / Fr(h)
                t_rn = float(exact)                               # RN(x / h)
                assert abs(Fr(x * y) - Fr(t_rn)) <= Fr(5, 2) * Fr(math.ulp(t_rn))
                q = _floor_from_product(x, y)
                if q is None:
                    declined += 1
                    continue
                taken += 1
                assert q == math.floor(t_rn), (box, M, x)
    assert taken > 15000 and declined > 500


def _bits(v):
    return int(np.float64(v).view(np.uint64))


def _from_bits(u):
    return float(np.uint64(u).view(np.float64))


def _quotient_one_step(x, h, y):
    """The chunk kernel's quotient: q0 = RN(x y), then one step to a
    neighbour decided in integers, comparing x / h with the midpoints next
    to q0 (x = Mx 2^Ex, m h = (2 Mq +- 1) Mh 2^(Eq - 1 + Eh), below a power
    of two (4 Mq - 1) Mh 2^(Eq - 2)), as the kernel does in 128 bits."""
    mant, hidden = (1 << 52) - 1, 1 << 52
    q0 = x * y
    ux, uq, uh = _bits(x), _bits(q0), _bits(h)
    mx, mq, mh = (ux & mant) | hidden, (uq & mant) | hidden, (uh & mant) | hidden
    s = (ux >> 52) - (uq >> 52) - (uh >> 52) + 1076
    assert 52 <= s <= 55
    big = mx << s                                   # x in units of 2^(Eq - 1 + Eh)
    up = big > (2 * mq + 1) * mh
    if mq != hidden:
        down = big < (2 * mq - 1) * mh
    else:
        down = (big << 1) < (4 * mq - 1) * mh
    assert (big << 1) != (4 * mq - 1) * mh and big != (2 * mq + 1) * mh and big != (2 * mq - 1) * mh
    return _from_bits(uq + int(up) - int(down))


def test_one_integer_step_quotient_equals_ieee_division():
    # RN(x / h) from the product and one step decided on exact integer
    # midpoints; the same inputs as the corrected quotient above, plus
    # quotients next to powers of two (where the lower neighbour is half an
    # ulp away) and every position within two ulps of them
    rng = np.random.default_rng(31)
    boxes = [23.0, 98.0, 17.0, 30.0, 1000.0 / 3.0, 0.7, 3.3e5] + list(rng.uniform(6.0, 600.0, 5))
    n = moved = 0
    for box in boxes:
        for M in (max(1, int(box // 4)) << 6, 13, 1000):
            h, xs = _cases(rng, box, M)
            if h == 2.0 ** math.floor(math.log2(h)):
                continue                               # powers of two take the exact scaling
            y = float(1 / Fr(h))
            for k in range(-8, 24):                    # x / h near 2^k
                x0 = float(Fr(2) ** k * Fr(h))
                for d in range(-2, 3):
                    x = x0
                    for _ in range(abs(d)):
                        x = float(np.nextafter(x, np.inf if d > 0 else -np.inf))
                    if 2.0 ** -900 <= x < box:
                        xs.append(x)
            for x in xs:
                t = _quotient_one_step(x, h, y)
                assert t == x / h, (box, M, x)
                moved += t != x * y
                n += 1
    assert n > 20000 and moved > 1000
