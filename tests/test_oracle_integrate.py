"""Pins for kick/drift, the force VJP and the trajectory reverse mode
(oracle.integrate) against finite differences and conservation laws."""
import numpy as np
import pytest

from oracle import fit, force, integrate
from workloads import generators as gen

RC, SIG, EPS = 3.0, 0.8, 0.1


@pytest.fixture(scope="module")
def coef():
    return fit.fit_poly(RC, SIG, EPS)


def test_force_vjp_matches_finite_differences(coef):
    L = 10.0
    pos = gen.uniform_box(300, L, 11)
    gbar = np.random.default_rng(2).standard_normal((300, 3))
    xbar = integrate.force_vjp(pos, L, RC, EPS, coef, gbar)
    dirs = gen.random_directions(6, 900, 5).reshape(6, 300, 3)
    h = 1e-6
    for e in dirs:
        ap, _ = force.accel_kdtree(pos + h * e, L, RC, EPS, coef)
        am, _ = force.accel_kdtree(pos - h * e, L, RC, EPS, coef)
        fd = np.sum(gbar * (ap - am)) / (2 * h)
        assert np.sum(xbar * e) == pytest.approx(fd, rel=2e-6, abs=1e-7)


def test_trajectory_gradient_matches_finite_differences(coef):
    L, n_side = 8.0, 8
    x0, psi = gen.zeldovich(n_side, L, 0.5, 1004)
    v0 = 0.1 * psi
    xt, _ = gen.zeldovich(n_side, L, 0.5, 1005)
    dt, K = 0.02, 10
    Lval, gx, gv = integrate.loss_and_grad(x0, v0, xt, L, RC, EPS, coef, dt, K)
    n = len(x0)
    rng = np.random.default_rng(0)
    h = 1e-6

    def lossf(x, v):
        xs, _ = integrate.trajectory(x, v, L, RC, EPS, coef, dt, K)
        return integrate.loss(xs[-1], xt, L)

    for k in range(4):
        ex = rng.standard_normal((n, 3)); ex /= np.linalg.norm(ex)
        ev = rng.standard_normal((n, 3)); ev /= np.linalg.norm(ev)
        fd = (lossf(x0 + h * ex, v0 + h * ev) - lossf(x0 - h * ex, v0 - h * ev)) / (2 * h)
        an = np.sum(gx * ex) + np.sum(gv * ev)
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-8)
    for k in range(4):
        i, ax = rng.integers(n), rng.integers(3)
        e = np.zeros((n, 3)); e[i, ax] = 1.0
        fd = (lossf(x0 + h * e, v0) - lossf(x0 - h * e, v0)) / (2 * h)
        assert gx[i, ax] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_trajectory_conserves_momentum(coef):
    L = 8.0
    x0, psi = gen.zeldovich(8, L, 0.5, 7)
    xs, vs = integrate.trajectory(x0, 0.1 * psi, L, RC, EPS, coef, 0.02, 5)
    p0 = vs[0].sum(axis=0)
    for v in vs[1:]:
        assert np.all(np.abs(v.sum(axis=0) - p0) < 1e-12 * (1 + np.abs(v).sum()))


def test_force_vjp_term_magnitudes(coef):
    # the per-row magnitude sums bound the sum (triangle inequality), equal
    # it for a row with one term (an isolated pair: each row holds the same
    # single term), and the value returned with them is the plain VJP's
    L = 10.0
    pos = gen.uniform_box(200, L, 13)
    gbar = np.random.default_rng(4).standard_normal((200, 3))
    out, mag = integrate.force_vjp(pos, L, RC, EPS, coef, gbar, absolute=True)
    np.testing.assert_array_equal(out, integrate.force_vjp(pos, L, RC, EPS, coef, gbar))
    assert np.all(np.abs(out) <= mag * (1 + 1e-12) + 1e-300)
    two = gen.two_body(1.7, 20.0, axis=0)
    g2 = np.array([[0.3, -0.2, 0.5], [-0.1, 0.4, 0.2]])
    o2, m2 = integrate.force_vjp(two, 20.0, RC, EPS, coef, g2, absolute=True)
    np.testing.assert_allclose(np.abs(o2), m2, rtol=1e-14)
    assert np.all(m2 > 0)


def test_kick_drift_basic():
    v = integrate.kick(np.ones((2, 3)), np.full((2, 3), 2.0), 0.5)
    np.testing.assert_array_equal(v, 2.0)
    x = integrate.drift(np.array([[7.9, 0.0, 1.0]]), np.array([[1.0, -1.0, 0.0]]), 0.2, 8.0)
    np.testing.assert_allclose(x, [[0.1, 7.8, 1.0]], atol=1e-12)
    inv = integrate.invariants(np.ones((4, 3)), np.zeros((4, 3)))
    assert inv["kinetic"] == 6.0 and np.all(inv["momentum"] == 4.0)


def test_leapfrog_reversible_and_second_order(coef):
    # leapfrog is time-reversible (run back with -dt) and its error shrinks
    # by ~4x when dt halves (second order), against a fine-step reference
    L = 8.0
    x0, psi = gen.zeldovich(8, L, 0.5, 7)
    v0 = 0.1 * psi
    x1, v1, a1 = integrate.leapfrog(x0, v0, L, RC, EPS, coef, 0.01, 20)
    xb, vb, _ = integrate.leapfrog(x1, -v1, L, RC, EPS, coef, 0.01, 20, a0=a1)
    assert np.max(np.abs(force.min_image(xb - x0, L))) < 1e-10
    assert np.max(np.abs(vb + v0)) < 1e-9
    # order of accuracy in a smooth regime: a lattice with small displacements
    xs, psis = gen.zeldovich(8, L, 0.05, 8)
    T = 0.4
    ref, _, _ = integrate.leapfrog(xs, 0.5 * psis, L, RC, EPS, coef, T / 256, 256)
    errs = []
    for k in (16, 32):
        xk, _, _ = integrate.leapfrog(xs, 0.5 * psis, L, RC, EPS, coef, T / k, k)
        errs.append(np.max(np.abs(force.min_image(xk - ref, L))))
    assert 3.0 < errs[0] / errs[1] < 5.0
