"""Pins for the short-range force and the binary32 pair predicate
(oracle.force): independent enumerations, textbook two-body limits,
Newton's third law, lattice symmetry, continuity at the cutoff."""
import numpy as np
import pytest

from oracle import binning, fit, force
from workloads import generators as gen

RC, SIG = 3.0, 0.8


@pytest.fixture(scope="module")
def coef():
    return fit.fit_poly(RC, SIG, 0.1)


@pytest.mark.parametrize("L,n,seed", [(7.0, 300, 1), (8.0, 512, 2), (10.0, 400, 3)])
def test_three_enumerations_agree(L, n, seed, coef):
    pos = gen.uniform_box(n, L, seed)
    a1, c1 = force.accel_brute(pos, L, RC, 0.1, coef)
    a2, c2 = force.accel_celllist(pos, L, RC, 0.1, coef)
    a3, c3 = force.accel_kdtree(pos, L, RC, 0.1, coef)
    scale = np.max(np.abs(a1)) + 1e-300
    np.testing.assert_allclose(a2, a1, rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(a3, a1, rtol=0, atol=1e-13 * scale)
    np.testing.assert_array_equal(c1, c2)
    np.testing.assert_array_equal(c1, c3)
    rows = np.array([0, 5, n - 1])
    a4, c4 = force.accel_rows(pos, L, RC, 0.1, coef, rows)
    np.testing.assert_allclose(a4, a1[rows], rtol=0, atol=1e-13 * scale)


@pytest.mark.parametrize("r", [0.3, 1.0, 2.2])
def test_two_body_newton_and_plummer(r):
    L = 20.0
    zero = np.zeros(6)
    pos = gen.two_body(r, L, axis=1)
    a, _ = force.accel_brute(pos, L, RC, 0.0, zero)
    # particle 0 sits below particle 1 on y: pulled towards +y with 1/r^2
    assert a[0, 1] == pytest.approx(1.0 / r ** 2, rel=1e-13)
    assert a[1, 1] == pytest.approx(-1.0 / r ** 2, rel=1e-13)
    assert np.all(a[:, [0, 2]] == 0)
    eps = 0.1
    a, _ = force.accel_brute(pos, L, RC, eps, zero)
    assert a[0, 1] == pytest.approx(r / (r * r + eps * eps) ** 1.5, rel=1e-13)


def test_minimum_image_across_boundary():
    L = 20.0
    zero = np.zeros(6)
    pos = np.array([[0.5, 10.0, 10.0], [19.5, 10.0, 10.0]])
    a, _ = force.accel_brute(pos, L, RC, 0.0, zero)
    assert a[0, 0] == pytest.approx(-1.0, rel=1e-13)      # neighbour lies at -1
    assert a[1, 0] == pytest.approx(1.0, rel=1e-13)


def test_newton_third_law(coef):
    pos, _, _ = gen.nfw_clustered(3000, 16.0, 4, m_hi=800.0)
    a, _ = force.accel_kdtree(pos, 16.0, RC, 0.1, coef)
    assert np.all(np.abs(a.sum(axis=0)) < 1e-12 * np.abs(a).sum())


def test_perfect_lattice_zero_force(coef):
    pos = gen.lattice(12, 12.0)
    a, cnt = force.accel_celllist(pos, 12.0, RC, 0.1, coef)
    assert np.max(np.abs(a)) < 1e-13
    assert np.all(cnt == cnt[0]) and cnt[0] > 0


def test_continuity_at_cutoff(coef):
    L = 20.0
    mags = []
    deltas = np.array([1e-2, 5e-3, 2.5e-3])
    for d in deltas:
        a, _ = force.accel_brute(gen.two_body(RC - d, L), L, RC, 0.1, coef)
        mags.append(abs(a[0, 0]))
    mags = np.array(mags)
    assert mags[0] < 0.02 / RC ** 2          # tiny against the Newtonian 1/r_c^2
    # linear approach to zero: halving delta halves |a|
    np.testing.assert_allclose(mags[1:] / mags[:-1], 0.5, rtol=0.02)


def test_fp32_predicate_agrees_with_fp64_away_from_cutoff(coef):
    L = 16.0
    pos = gen.uniform_box(4096, L, 1000)
    B = binning.bin_particles([(pos, L)], [4], 5)
    cnt32 = force.pair_counts_fp32(B, [(pos, L)], RC, 0.1)
    _, cnt64 = force.accel_kdtree(pos, L, RC, 0.1, coef)
    # any disagreement must come from pairs within 1e-5 of the cutoff
    i, j, m = force.candidate_pairs(pos, L, RC * 1.001)
    d = force.min_image(pos[j] - pos[i], L)
    s = np.sum(d * d, axis=1)
    near = np.abs(s - RC * RC) < 1e-5 * RC * RC
    near_per_i = np.bincount(i[near], minlength=len(pos))
    assert np.all(np.abs(cnt32 - cnt64) <= near_per_i)
    assert cnt32.sum() > 0
    rows = np.array([3, 77, 4000])
    np.testing.assert_array_equal(force.pair_counts_fp32(B, [(pos, L)], RC, 0.1, rows=rows), cnt32[rows])


def test_fp32_predicate_single_pair_by_hand():
    # one pair in the same chunk: offsets exact, predicate decided by s'
    L, n_c, b = 16.0, 4, 5
    h, e2, r2 = force.unit_constants(L, n_c, b, RC, 0.1)
    assert h == 0.125 and e2 == np.float32(0.64) and r2 == np.float32((9.0 + 0.01) / h / h)
    off_i = np.array([[1.0, 2.0, 3.0]], np.float32)
    inside = np.array([[1.0 + 23.0, 2.0, 3.0]], np.float32)     # 23 h = 2.875 < 3
    outside = np.array([[1.0 + 24.0, 2.0, 3.0]], np.float32)    # 24 h = 3.0, s' = 576.64 >= rc2p
    z = np.zeros((1, 3))
    assert force.pair_predicate(off_i, inside, z, e2, r2)[0]
    assert not force.pair_predicate(off_i, outside, z, e2, r2)[0]
