"""Pins for the most-bound-particle center finder oracle (oracle.centers)
against closed forms, a continuum limit and symmetries of the potential."""
import math

import numpy as np
import pytest

from oracle import centers
from workloads import generators as gen


def test_two_body_closed_form():
    L, eps, r = 50.0, 0.1, 1.7
    pos = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
    c, cphi, phi = centers.halo_centers(pos, np.array([0, 0]), L, eps, 1)
    want = -1.0 / math.sqrt(r * r + eps * eps)
    np.testing.assert_allclose(phi, [want, want], rtol=1e-15)
    assert c[0] == 0 and cphi[0] == phi[0]              # tie -> smaller index


def test_octahedron_with_center_closed_form():
    # six vertices at distance R on the axes plus one particle at the centre
    L, eps, R = 40.0, 0.05, 2.0
    ctr = np.array([20.0, 20.0, 20.0])
    verts = np.array([[R, 0, 0], [-R, 0, 0], [0, R, 0], [0, -R, 0], [0, 0, R], [0, 0, -R]])
    pos = np.vstack([ctr + verts, ctr])
    c, cphi, phi = centers.halo_centers(pos, np.zeros(7, int), L, eps, 1)
    inv = lambda d: 1.0 / math.sqrt(d * d + eps * eps)
    vert = -(inv(R) + 4 * inv(R * math.sqrt(2)) + inv(2 * R))
    np.testing.assert_allclose(phi[:6], vert, rtol=1e-14)
    np.testing.assert_allclose(phi[6], -6 * inv(R), rtol=1e-14)
    assert c[0] == 6


def test_coincident_particles_softened_limit():
    # all members at one point: every phi is -(n-1)/eps, the first index wins
    n, eps = 37, 0.25
    pos = np.full((n, 3), 3.0)
    c, cphi, phi = centers.halo_centers(pos, np.zeros(n, int), 8.0, eps, 1)
    np.testing.assert_allclose(phi, -(n - 1) / eps, rtol=1e-14)
    assert c[0] == 0


def test_uniform_sphere_central_potential():
    # continuum limit: the potential at the centre of a uniform sphere of
    # n unit masses and radius R is -3n/(2R); the most bound particle sits
    # near the centre (shot noise moves it off the exact middle)
    n, R, L = 12000, 10.0, 100.0
    rng = np.random.default_rng(5)
    d = gen.random_directions(n, 3, 6)
    r = R * rng.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    pos = 50.0 + d * r[:, None]
    pos[0] = 50.0
    c, cphi, phi = centers.halo_centers(pos, np.zeros(n, int), L, 0.01, 1)
    assert phi[0] == pytest.approx(-1.5 * n / R, rel=0.02)
    assert cphi[0] <= phi[0] and cphi[0] == pytest.approx(-1.5 * n / R, rel=0.03)
    assert np.linalg.norm(pos[c[0]] - 50.0) < 0.3 * R
    # and at radius r the continuum value is -(n/(2R^3))(3R^2 - r^2)
    far = r > 0.5 * R
    want = -(n / (2 * R ** 3)) * (3 * R * R - r[far] ** 2)
    assert np.median(np.abs(phi[far] / want - 1.0)) < 0.01


def test_periodic_wrap_invariance_and_halo_independence():
    # a halo straddling the box corner has the same potentials as the same
    # halo moved to the interior; a second halo and unlabelled particles
    # change nothing
    L, eps = 32.0, 0.05
    rng = np.random.default_rng(9)
    blob = rng.normal(0.0, 1.5, size=(600, 3))
    inside = blob + 16.0
    wrapped = np.mod(blob + 0.3, L)                     # straddles 0 / L
    phi_in = centers.halo_potentials(inside, np.zeros(600, int), L, eps, block=128)
    phi_w = centers.halo_potentials(wrapped, np.zeros(600, int), L, eps, block=128)
    np.testing.assert_allclose(phi_w, phi_in, rtol=1e-12)
    other = rng.uniform(0.0, L, size=(300, 3))
    pos = np.vstack([wrapped, other, other + 0.01])
    lab = np.concatenate([np.zeros(600, int), np.ones(300, int), -np.ones(300, int)])
    c, cphi, phi = centers.halo_centers(pos, lab, L, eps, 3)
    np.testing.assert_allclose(phi[:600], phi_in, rtol=1e-12)
    assert np.all(phi[900:] == 0.0)
    assert c[2] == -1 and cphi[2] == np.inf              # empty halo
    assert c[0] == int(np.argmin(phi_in))


def test_block_size_and_member_order_do_not_matter():
    pos, lab, sizes = gen.nfw_clustered(3000, 20.0, 17, m_lo=40.0, m_hi=800.0)
    nh = len(sizes)
    c1, _, phi1 = centers.halo_centers(pos, lab, 20.0, 0.05, nh)
    perm = np.random.default_rng(3).permutation(len(pos))
    c2, _, phi2 = centers.halo_centers(pos[perm], lab[perm], 20.0, 0.05, nh)
    np.testing.assert_allclose(phi2, phi1[perm], rtol=1e-12)
    ok = c1 >= 0
    np.testing.assert_array_equal(perm[c2[ok]], c1[ok])
    phi3 = centers.halo_potentials(pos, lab, 20.0, 0.05, block=7)
    np.testing.assert_allclose(phi3, phi1, rtol=1e-12)


def test_member_potentials_agree_with_full_sum():
    pos, lab, sizes = gen.nfw_clustered(2000, 16.0, 21, m_lo=40.0, m_hi=500.0)
    phi = centers.halo_potentials(pos, lab, 16.0, 0.05)
    idx = np.random.default_rng(1).choice(len(pos), 50, replace=False)
    np.testing.assert_allclose(centers.member_potentials(pos, lab, 16.0, 0.05, idx), phi[idx],
                               rtol=1e-12)
