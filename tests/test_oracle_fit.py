"""Pins for the force split and the polynomial fit (oracle.fit).

Each check compares the oracle with something other than itself: numerical
quadrature of the Gaussian density behind F_long, the Newtonian limit, the
KKT optimality conditions of the least-squares problem, exact recovery of a
polynomial target, and the continuity condition at the cutoff.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import fit

SIGMA = 0.8
RC = 3.0


def gaussian_enclosed(r, sigma):
    """M(<r) of a unit-mass 3-D Gaussian with per-axis variance 2 sigma^2,
    by numerical radial quadrature of its density."""
    norm = (4.0 * math.pi * sigma * sigma) ** -1.5
    val, _ = quad(lambda t: 4.0 * math.pi * t * t * norm * math.exp(-t * t / (4 * sigma * sigma)),
                  0.0, r, epsabs=0, epsrel=1e-13, limit=200)
    return val


@pytest.mark.parametrize("r", [0.05, 0.3, 1.0, 1.7, 3.0, 5.0])
def test_force_long_is_gaussian_enclosed_mass(r):
    expect = gaussian_enclosed(r, SIGMA) / (r * r)
    assert fit.force_long(r, SIGMA) == pytest.approx(expect, rel=1e-11)


def test_g_at_zero_is_central_density_limit():
    # M(<r)/r^3 -> (4 pi / 3) rho(0) as r -> 0
    rho0 = (4.0 * math.pi * SIGMA * SIGMA) ** -1.5
    assert fit.g_long(0.0, SIGMA)[0] == pytest.approx(4.0 * math.pi / 3.0 * rho0, rel=1e-14)


def test_g_series_and_closed_form_agree_near_switch():
    # both branches of g_long evaluated at the same points around u = 0.25
    s = (2 * SIGMA * np.array([0.2, 0.24, 0.26, 0.3])) ** 2
    series_pts = fit.g_long(s * 0 + s, SIGMA)
    closed = fit.force_long(np.sqrt(s), SIGMA) / np.sqrt(s)
    np.testing.assert_allclose(series_pts, closed, rtol=1e-10)


def test_force_long_newtonian_far_field():
    r = np.array([10.0, 20.0])
    np.testing.assert_allclose(fit.force_long(r, SIGMA) * r * r, 1.0, rtol=1e-12)


@pytest.mark.parametrize("eps", [0.1, 0.05, 0.0])
def test_constrained_fit_zero_at_cutoff(eps):
    c = fit.fit_poly(RC, SIGMA, eps)
    assert fit.p_eval(RC * RC, c) == pytest.approx((RC * RC + eps * eps) ** -1.5, rel=1e-14)
    assert abs(fit.f_sr(RC * RC, eps, c)) < 1e-15


def _design(n=fit.N_SAMPLES):
    t = (np.arange(n) + 0.5) / n
    return t, np.vander(t, 6, increasing=True)


@pytest.mark.parametrize("mode", ["constrained", "unconstrained"])
def test_fit_kkt_conditions(mode):
    eps = 0.1
    c = fit.fit_poly(RC, SIGMA, eps, mode)
    t, V = _design()
    a = c * (RC * RC) ** np.arange(6)              # back to the t basis
    r = V @ a - fit.g_long(RC * RC * t, SIGMA)
    grad = V.T @ r
    scale = np.abs(V.T).sum(axis=1) * np.max(np.abs(r)) + 1e-300
    if mode == "unconstrained":
        assert np.all(np.abs(grad) / scale < 1e-11)
    else:
        # gradient parallel to the constraint normal (1, 1, ..., 1)
        lam = grad.mean()
        assert np.all(np.abs(grad - lam) / scale < 1e-11)


@pytest.mark.parametrize("mode", ["constrained", "unconstrained"])
def test_fit_recovers_polynomial_target(mode):
    eps = 0.1
    # a degree-5 target that also satisfies the cutoff equality
    base = np.array([0.2, -0.03, 2e-3, 1e-4, -2e-5, 1e-6])
    P = lambda s: fit.p_eval(s, base)
    tgt = (RC * RC + eps * eps) ** -1.5
    base[0] += tgt - P(RC * RC)
    c = fit.fit_poly_to(lambda s: fit.p_eval(s, base), RC, eps, mode)
    np.testing.assert_allclose(c * (RC * RC) ** np.arange(6),
                               base * (RC * RC) ** np.arange(6), rtol=0, atol=1e-12)


def test_unconstrained_fit_residual_and_value_at_zero():
    c = fit.fit_poly(RC, SIGMA, 0.1, "unconstrained")
    s = np.linspace(0.0, RC * RC, 20001)
    res = np.max(np.abs(fit.p_eval(s, c) - fit.g_long(s, SIGMA)))
    assert res < 5e-5
    assert abs(c[0] - 1.0 / (6 * math.sqrt(math.pi) * SIGMA ** 3)) <= res * (1 + 1e-9)


def test_split_sums_to_softened_newton():
    # short + long range = (s + eps^2)^(-3/2) up to the fit residual
    eps = 0.1
    c = fit.fit_poly(RC, SIGMA, eps)
    s = np.linspace(0.01, 0.8 * RC * RC, 500)
    total = fit.f_sr(s, eps, c) + fit.g_long(s, SIGMA)
    np.testing.assert_allclose(total, (s + eps * eps) ** -1.5, atol=2e-3)


def test_derivative_matches_finite_difference():
    eps = 0.1
    c = fit.fit_poly(RC, SIGMA, eps)
    s = np.linspace(0.05, 8.9, 50)
    h = 1e-6
    fd = (fit.f_sr(s + h, eps, c) - fit.f_sr(s - h, eps, c)) / (2 * h)
    np.testing.assert_allclose(fit.df_sr(s, eps, c), fd, rtol=1e-6, atol=1e-9)
