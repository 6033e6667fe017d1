"""Long/short force split and the polynomial fit of the long-range part.

The paper (Sec. 2) splits the force into a spectrally filtered PM long-range
part and a short-range part computed by direct particle-particle sums; it
does not print the filter.  The split used here is the Gaussian one: the
long-range force of a unit point mass is

    F_long(r) = (1/r^2) [ erf(r / 2 sigma) - (r / (sigma sqrt(pi))) exp(-r^2 / 4 sigma^2) ],

which is the enclosed-mass law of a 3-D Gaussian of per-axis variance
2 sigma^2.  The short-range kernel replaces F_long(r)/r by a degree-5
polynomial p(s) in s = r^2, fitted by least squares on [0, r_c^2]:

    f_SR(s) = (s + eps^2)^(-3/2) - p(s),      a_i = sum_j (x_j - x_i) f_SR(s_ij).

Fit reading (the paper is silent): M = 4096 midpoint samples
s_k = r_c^2 (k + 1/2) / M, unweighted; basis t^m with t = s / r_c^2 for
conditioning, converted to monomials in s.  mode "constrained" (default)
adds the equality p(r_c^2) = (r_c^2 + eps^2)^(-3/2), so that f_SR(r_c^2) = 0
and the force is continuous at the cutoff; mode "unconstrained" is plain
least squares.  The constraint is eliminated by substitution and the
reduced problem solved with an SVD least-squares routine.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

N_SAMPLES = 4096
DEGREE = 5


def force_long(r, sigma):
    """F_long(r) for r > 0 (Gaussian-split long-range force, unit masses)."""
    r = np.asarray(r, dtype=np.float64)
    u = r / (2.0 * sigma)
    return (erf(u) - (r / (sigma * math.sqrt(math.pi))) * np.exp(-u * u)) / (r * r)


def g_long(s, sigma):
    """F_long(sqrt(s)) / sqrt(s), finite at s = 0.

    For u = sqrt(s)/(2 sigma) < 0.25 the series
    g = (2/sqrt(pi)) / (8 sigma^3) * sum_{n>=1} (-1)^(n+1) 2n u^(2n-2) / (n! (2n+1))
    is used (term-by-term difference of the erf and Gaussian series), giving
    g(0) = 1 / (6 sqrt(pi) sigma^3); otherwise the closed form.
    """
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    out = np.empty_like(s)
    u = np.sqrt(s) / (2.0 * sigma)
    small = u < 0.25
    if np.any(small):
        us = u[small] ** 2
        acc = np.zeros_like(us)
        term_pow = np.ones_like(us)
        fact = 1.0
        for n in range(1, 16):
            fact *= n
            acc += ((-1) ** (n + 1)) * (2.0 * n) * term_pow / (fact * (2 * n + 1))
            term_pow = term_pow * us
        out[small] = (2.0 / math.sqrt(math.pi)) / (8.0 * sigma ** 3) * acc
    big = ~small
    if np.any(big):
        r = np.sqrt(s[big])
        out[big] = force_long(r, sigma) / r
    return out


def fit_poly_to(target_fn, rc: float, eps: float, mode: str = "constrained",
                n_samples: int = N_SAMPLES) -> np.ndarray:
    """Least-squares degree-5 fit of target_fn(s) on [0, rc^2] (see module doc).

    Returns monomial coefficients c[0..5] in s (FP64).
    """
    if mode not in ("constrained", "unconstrained"):
        raise ValueError(mode)
    k = np.arange(n_samples, dtype=np.float64)
    t = (k + 0.5) / n_samples
    s = rc * rc * t
    g = target_fn(s)
    V = np.vander(t, DEGREE + 1, increasing=True)      # columns t^0 .. t^5
    if mode == "unconstrained":
        a, *_ = np.linalg.lstsq(V, g, rcond=None)
    else:
        target = (rc * rc + eps * eps) ** -1.5          # p(rc^2) = sum_m a_m
        # a_0 = target - sum_{m>=1} a_m  =>  V a = target + sum_{m>=1} a_m (t^m - 1)
        R = V[:, 1:] - 1.0
        a_rest, *_ = np.linalg.lstsq(R, g - target, rcond=None)
        a = np.concatenate([[target - a_rest.sum()], a_rest])
    return a / (rc * rc) ** np.arange(DEGREE + 1)


def fit_poly(rc: float, sigma: float, eps: float, mode: str = "constrained",
             n_samples: int = N_SAMPLES) -> np.ndarray:
    """Coefficients c[0..5] of p(s) fitted to g(s) = F_long(sqrt s)/sqrt s."""
    return fit_poly_to(lambda s: g_long(s, sigma), rc, eps, mode, n_samples)


def p_eval(s, c):
    """p(s) by Horner's rule in FP64."""
    s = np.asarray(s, dtype=np.float64)
    acc = np.zeros_like(s) + c[-1]
    for ck in c[-2::-1]:
        acc = acc * s + ck
    return acc


def dp_eval(s, c):
    """p'(s)."""
    s = np.asarray(s, dtype=np.float64)
    d = np.array([k * c[k] for k in range(1, len(c))])
    return p_eval(s, d)


def f_sr(s, eps, c):
    """Short-range pair factor f_SR(s) = (s + eps^2)^(-3/2) - p(s)."""
    s = np.asarray(s, dtype=np.float64)
    return (s + eps * eps) ** -1.5 - p_eval(s, c)


def df_sr(s, eps, c):
    """d f_SR / ds = -3/2 (s + eps^2)^(-5/2) - p'(s)."""
    s = np.asarray(s, dtype=np.float64)
    return -1.5 * (s + eps * eps) ** -2.5 - dp_eval(s, c)
