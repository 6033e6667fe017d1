"""Exact emulation of IEEE-754 binary32 operations in NumPy.

The in-range pair predicate is defined on binary32 operations (round to
nearest, ties to even), so that pair counts can be compared bit for bit.
Single additions, subtractions and multiplications of binary32 operands are
evaluated in binary64 and rounded once to binary32; because binary64 carries
more than 2*24+2 significand bits, that double rounding is innocuous and the
result equals the correctly rounded binary32 operation.

A fused multiply-add a*b + c is not covered by that argument (three
operands), so ``fma32`` forms the exact product in binary64 (24+24 bits fit),
adds c with an error-free two-sum (s + e equals a*b + c exactly), rounds s
to binary32, and corrects the one case where that rounding differs from the
correct rounding of s + e: s lying exactly halfway between two binary32
neighbours while e is non-zero.  (If s is not a midpoint, |e| <= ulp64(s)/2
cannot move s + e across the binary32 midpoint, which is itself a binary64
number.)
"""
from __future__ import annotations

import numpy as np

F32 = np.float32
F64 = np.float64


def f32(x):
    """Round binary64 values to binary32 (ties to even)."""
    return np.asarray(x, dtype=F64).astype(F32)


def add32(a, b):
    return (np.asarray(a, F32).astype(F64) + np.asarray(b, F32).astype(F64)).astype(F32)


def sub32(a, b):
    return (np.asarray(a, F32).astype(F64) - np.asarray(b, F32).astype(F64)).astype(F32)


def mul32(a, b):
    return (np.asarray(a, F32).astype(F64) * np.asarray(b, F32).astype(F64)).astype(F32)


def fma32(a, b, c):
    """Correctly rounded binary32 fused multiply-add a*b + c."""
    a64 = np.asarray(a, F32).astype(F64)
    b64 = np.asarray(b, F32).astype(F64)
    c64 = np.asarray(c, F32).astype(F64)
    p = a64 * b64                       # exact
    with np.errstate(invalid="ignore", over="ignore"):
        s = p + c64
        bb = s - p
        e = (p - (s - bb)) + (c64 - bb)     # two-sum error: s + e == p + c
        r = s.astype(F32)
        r64 = r.astype(F64)
        up = s > r64
        nb = np.where(up, np.nextafter(r, F32(np.inf)), np.nextafter(r, F32(-np.inf)))
        nb64 = nb.astype(F64)
        mid = 0.5 * (r64 + nb64)            # exact in binary64
        is_mid = (s != r64) & (s == mid) & np.isfinite(s)
        toward = is_mid & (e != 0.0) & (np.sign(e) == np.sign(nb64 - r64))
    return np.where(toward, nb, r).astype(F32)
