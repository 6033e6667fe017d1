"""Pins for the long-range PM and power-spectrum oracle (oracle.pm): CIC
invariants, the Poisson shot-noise spectrum in closed form, Parseval, the
PM force against a direct Fourier sum of the filtered periodic force, and
the split summing back to Newton."""
import numpy as np
import pytest

from oracle import fit, force, pm
from workloads import generators as gen


def test_cic_conserves_mass_and_hits_grid_points():
    L, ng = 10.0, 10
    pos = gen.uniform_box(500, L, 1)
    g = pm.cic_deposit(pos, L, ng)
    assert g.sum() == pytest.approx(500.0, rel=1e-13)
    assert g.min() >= 0.0
    one = pm.cic_deposit(np.array([[3.0, 4.0, 9.0]]), L, ng)
    assert one[3, 4, 9] == 1.0 and one.sum() == 1.0
    mid = pm.cic_deposit(np.array([[3.5, 9.5, 0.5]]), L, ng)
    for ix in (3, 4):
        for iy in (9, 0):                                   # wraps at the box edge
            for iz in (0, 1):
                assert mid[ix, iy, iz] == 0.125


def test_cic_translation_and_adjointness():
    L, ng = 16.0, 16
    pos = gen.uniform_box(300, L, 2)
    g = pm.cic_deposit(pos, L, ng)
    shifted = pm.cic_deposit(pos + np.array([1.0, 0.0, 2.0]), L, ng)
    np.testing.assert_allclose(shifted, np.roll(np.roll(g, 1, axis=0), 2, axis=2), atol=1e-12)
    # interpolation is the transpose of the deposit: sum_p F(x_p) = sum_x F(x) counts(x)
    field = np.random.default_rng(3).standard_normal((ng, ng, ng))
    assert pm.cic_interpolate(field, pos, L).sum() == pytest.approx((field * g).sum(), rel=1e-12)
    assert np.allclose(pm.cic_interpolate(np.full((ng, ng, ng), 2.5), pos, L), 2.5)


def test_cic_window_values():
    w = pm.cic_window(8, 8.0)
    assert w[0, 0, 0] == 1.0
    assert w[4, 0, 0] == pytest.approx((2.0 / np.pi) ** 2, rel=1e-14)   # Nyquist: sinc^2(pi/2)
    assert w[4, 4, 4] == pytest.approx((2.0 / np.pi) ** 6, rel=1e-14)


def test_lattice_on_the_grid_has_no_power():
    L, ng = 16.0, 16
    pos = gen.lattice(16, L, offset=0.0)
    k, p, modes = pm.power_spectrum(pos, L, ng)
    assert np.all(modes > 0) and np.max(np.abs(p)) < 1e-20


def test_power_normalisation_parseval():
    # sum over all modes of P W^2 equals V / n_g^3 * sum_x delta^2
    L, ng = 12.0, 12
    pos = gen.uniform_box(3000, L, 4)
    counts = pm.cic_deposit(pos, L, ng)
    delta = counts / (len(pos) / ng ** 3) - 1.0
    dk = np.fft.fftn(delta)
    p3 = (L ** 3 / ng ** 6) * np.abs(dk) ** 2
    assert p3.sum() == pytest.approx(L ** 3 / ng ** 3 * (delta ** 2).sum(), rel=1e-12)


def test_poisson_shot_noise_closed_form():
    # uniform random points: after the CIC compensation the expected power
    # of mode k is (1/nbar) prod_a [1 - (2/3) sin^2(k_a D / 2)] / W(k)^2
    L, ng, n = 32.0, 32, 200000
    pos = gen.uniform_box(n, L, 5)
    k, p, modes = pm.power_spectrum(pos, L, ng)
    m, k1 = pm.wavenumbers(ng, L)
    s2 = np.sin(0.5 * k1 * (L / ng)) ** 2
    alias = (1 - 2 / 3 * s2)[:, None, None] * (1 - 2 / 3 * s2)[None, :, None] * (1 - 2 / 3 * s2)[None, None, :]
    expect3 = (L ** 3 / n) * alias / pm.cic_window(ng, L) ** 2
    mm = np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2)
    b = np.rint(mm).astype(int)
    for bin_ in range(2, ng // 2 + 1):
        want = expect3[b == bin_].mean()
        # per bin: mean of ~modes/2 independent exponential variables
        sig = want / np.sqrt(modes[bin_ - 1] / 2)
        assert abs(p[bin_ - 1] - want) < 5 * sig + 1e-3 * want, bin_


def _direct_long_range(d, L, sigma, mmax):
    """Exact periodic filtered force on a particle at separation d from one
    unit source (Fourier series, no grid):
    a = (1/V) sum_{k != 0} i k (4 pi / k^2) exp(-k^2 sigma^2) exp(i k . d)."""
    m = np.arange(-mmax, mmax + 1)
    kx, ky, kz = np.meshgrid(*(2 * np.pi * m / L,) * 3, indexing="ij")
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    k2[mmax, mmax, mmax] = 1.0
    amp = 4 * np.pi * np.exp(-k2 * sigma ** 2) / k2
    amp[mmax, mmax, mmax] = 0.0
    phase = kx * d[0] + ky * d[1] + kz * d[2]
    # i k e^{i phase}: real part -k sin(phase)
    s = np.sin(phase)
    return np.array([-(kx * amp * s).sum(), -(ky * amp * s).sum(), -(kz * amp * s).sum()]) / L ** 3


def test_pm_force_matches_direct_fourier_sum():
    L, ng, sigma = 32.0, 32, 0.8
    src = np.array([10.3, 12.6, 15.2])
    for r in (2.0, 3.5, 6.0, 9.0):
        d = np.array([r * 0.8, r * 0.6, 0.0])
        pos = np.vstack([src, src + d])
        a = pm.pm_accel(pos, L, ng, sigma)[1]
        ref = _direct_long_range(d, L, sigma, 24)
        assert np.linalg.norm(a - ref) <= 0.03 * np.linalg.norm(ref), r
    # far from the source the periodic sum approaches the isolated F_long
    d = np.array([4.0, 0.0, 0.0])
    ref = _direct_long_range(d, L, sigma, 24)
    iso = -fit.force_long(4.0, sigma)
    assert ref[0] == pytest.approx(iso, rel=0.03)


def test_pm_momentum_conservation():
    L, ng = 16.0, 16
    pos, _, _ = gen.nfw_clustered(2000, L, 8, m_lo=50.0, m_hi=600.0)
    a = pm.pm_accel(pos, L, ng, 0.8)
    scale = np.abs(a).sum()
    assert np.all(np.abs(a.sum(axis=0)) < 1e-12 * scale)


def test_split_sums_back_to_newton():
    # an isolated pair: PM long range + fitted short range ~ softened Newton
    L, ng, rc, sigma, eps = 64.0, 64, 3.0, 0.8, 0.05
    c = fit.fit_poly(rc, sigma, eps)
    src = np.array([20.2, 30.1, 25.7])
    for r in (1.0, 1.8, 2.6, 4.0):
        pos = np.vstack([src, src + np.array([r, 0.0, 0.0])])
        a_l = pm.pm_accel(pos, L, ng, sigma)[1, 0]
        a_s = force.accel_brute(pos, L, rc, eps, c)[0][1, 0]
        newton = -r / (r * r + eps * eps) ** 1.5
        assert a_l + a_s == pytest.approx(newton, rel=0.03), r


def test_shell_binning_brute_force():
    # modes per shell and their mean |k|, counted by a plain triple loop over
    # signed integer frequencies: shell b holds the modes with round(|m|) = b
    L, ng = 8.0, 8
    pos = gen.uniform_box(100, L, 9)
    k, p, modes = pm.power_spectrum(pos, L, ng)
    cnt = [0] * (ng // 2 + 1)
    ksum = [0.0] * (ng // 2 + 1)
    for a in range(ng):
        for b in range(ng):
            for c in range(ng):
                m = [v if v < ng // 2 else v - ng for v in (a, b, c)]
                r = (m[0] ** 2 + m[1] ** 2 + m[2] ** 2) ** 0.5
                sh = int(r + 0.5) if r % 1 != 0.5 else int(round(r))
                if 1 <= sh <= ng // 2:
                    cnt[sh] += 1
                    ksum[sh] += 2 * np.pi * r / L
    np.testing.assert_array_equal(modes, cnt[1:])
    np.testing.assert_allclose(k, np.array(ksum[1:]) / np.array(cnt[1:]), rtol=1e-13)
