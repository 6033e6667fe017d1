"""The invariant sums' arithmetic (sr_invariants, one thread's rows): each
sum is held as an unevaluated pair of binary32 numbers (hi, lo), every
term added by TwoSum with the error put into lo and the pair renormalised,
and the squares of the kinetic energy split exactly (TwoProduct by a fused
multiply-add) before they are added.  Emulated here in IEEE binary32 (numpy
float32 rounds to nearest even), against the exact sums of the same binary32
terms in rational arithmetic: the error stays a small multiple of 2^-47 of
the sum of magnitudes per term added, whatever the count of terms, where a
plain binary32 sum loses 2^-24 per term."""
from fractions import Fraction as Fr

import numpy as np

f32 = np.float32


def _two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    e = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, e


def _df_add(hi, lo, x):
    s, e = _two_sum(hi, x)
    e = f32(e + lo)
    hi = f32(s + e)
    lo = f32(e - f32(hi - s))
    return hi, lo


def _square_error(x):
    p = f32(x * x)
    return p, f32(np.float64(x) * np.float64(x) - np.float64(p))   # exact: x^2 - p fits binary32


def _thread_sums(v):
    """One thread's Σ v_x and ½ Σ |v|^2 over rows v (n, 3) float32, in the
    kernel's order of operations; returned as binary64 (hi + lo)."""
    hx = lx = h6 = l6 = f32(0.0)
    for row in v:
        hx, lx = _df_add(hx, lx, row[0])
        ps, es = zip(*(_square_error(c) for c in row))
        for p in ps:
            h6, l6 = _df_add(h6, l6, p)
        l6 = f32(l6 + f32(es[0] + f32(es[1] + es[2])))
    return float(np.float64(hx) + np.float64(lx)), 0.5 * float(np.float64(h6) + np.float64(l6))


def test_pair_sums_stay_within_a_few_ulps_of_48_bits():
    rng = np.random.default_rng(11)
    worst = 0.0
    for trial in range(120):
        m = int(rng.integers(20, 400))
        mag = 10.0 ** rng.uniform(-6, 3, (m, 3))
        v = (mag * rng.choice([-1.0, 1.0], (m, 3))).astype(np.float32)
        if trial % 4 == 0:                                  # cancelling sums (momentum near zero)
            v[m // 2:2 * (m // 2)] = -v[:m // 2]
        sx, ke = _thread_sums(v)
        exact_x = sum(Fr(float(x)) for x in v[:, 0])
        exact_ke = sum(Fr(float(x)) ** 2 for x in v.ravel()) / 2
        scale_x = sum(abs(Fr(float(x))) for x in v[:, 0])
        for got, exact, scale in ((sx, exact_x, scale_x), (ke, exact_ke, exact_ke)):
            err = abs(Fr(got) - exact) / scale
            bound = Fr(3 * m, 2 ** 47)
            assert err <= bound, (trial, m, float(err), float(bound))
            worst = max(worst, float(err / bound))
    assert worst > 0.0                                     # the bound is met, not trivially zero


def test_pair_sums_beat_plain_binary32():
    # a long run of small terms onto a large one: binary32 alone drops them,
    # the pair keeps them
    v = np.zeros((2000, 3), np.float32)
    v[0, 0] = 1.0e4
    v[1:, 0] = 1.0e-4
    sx, _ = _thread_sums(v)
    exact = float(sum(Fr(float(x)) for x in v[:, 0]))
    plain = f32(0.0)
    for x in v[:, 0]:
        plain = f32(plain + x)
    assert abs(sx - exact) < 1e-10 * exact
    assert abs(float(plain) - exact) > 1e-8 * exact
