"""The seeded input generators against the recipe they state: determinism
per seed; Zel'dovich displacements with the requested rms, zero mean, a
potential (curl-free) field and a power spectrum falling as k^-4 (|delta|^2
~ k^-2 times 1/k^2); NFW halo sets with the exact halo budget, sizes on
[m_lo, m_hi] following dN/dM ~ M^-1.9, radii following the NFW enclosed
mass; batch volumes that are cubes at one particle per cell with
10^4 <= N <= 10^6."""
import numpy as np
import pytest
from scipy import stats

from workloads import configs as wc
from workloads import generators as gen


def test_generators_are_deterministic_per_seed():
    a, _ = gen.zeldovich(16, 16.0, 0.5, 7)
    b, _ = gen.zeldovich(16, 16.0, 0.5, 7)
    c, _ = gen.zeldovich(16, 16.0, 0.5, 8)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    p1 = gen.nfw_clustered(5000, 24.0, 3, m_lo=40.0, m_hi=600.0)
    p2 = gen.nfw_clustered(5000, 24.0, 3, m_lo=40.0, m_hi=600.0)
    assert all(np.array_equal(x, y) for x, y in zip(p1, p2))
    w1 = wc.make_workload(wc.small_variant("clustered256"))
    w2 = wc.make_workload(wc.small_variant("clustered256"))
    assert np.array_equal(w1["volumes"][0][0], w2["volumes"][0][0])


def test_zeldovich_field():
    n, box, rms = 32, 32.0, 0.5
    pos, psi = gen.zeldovich(n, box, rms, 11)
    assert np.sqrt(np.mean(np.sum(psi * psi, axis=1))) == pytest.approx(rms, rel=1e-12)
    assert np.all(np.abs(psi.mean(axis=0)) < 1e-12)
    assert np.all((pos >= 0) & (pos < box))
    d = pos - gen.lattice(n, box)
    d -= box * np.round(d / box)
    assert np.allclose(d, psi, atol=1e-9)
    # a gradient field: k_y psi_x(k) = k_x psi_y(k) (and cyclic)
    P = [np.fft.fftn(psi[:, a].reshape(n, n, n)) for a in range(3)]
    k = 2 * np.pi * np.fft.fftfreq(n, d=box / n)
    kx, ky, kz = np.meshgrid(k, k, k, indexing="ij")
    K = (kx, ky, kz)
    scale = np.max(np.abs(P[0]))
    for a, b in ((0, 1), (1, 2), (0, 2)):
        assert np.max(np.abs(K[b] * P[a] - K[a] * P[b])) < 1e-9 * scale * np.max(np.abs(k))
    # |psi(k)|^2 falls as k^-4: k^4 |psi(k)|^2 is white noise, so its means
    # over shells of 2,000 modes are flat in k
    k2 = kx * kx + ky * ky + kz * kz
    white = (sum(np.abs(p) ** 2 for p in P) * k2 * k2).ravel()
    kk = np.sqrt(k2).ravel()
    sel = (kk > 0) & (kk < 0.9 * np.max(np.abs(k)))
    order = np.argsort(kk[sel])
    groups = np.array_split(order, len(order) // 2000)
    ks = [kk[sel][g].mean() for g in groups]
    ws = [white[sel][g].mean() for g in groups]
    slope = np.polyfit(np.log(ks), np.log(ws), 1)[0]
    assert abs(slope) < 0.1, slope


def test_nfw_halo_budget_and_mass_function():
    n, box = 400_000, 200.0
    pos, labels, sizes = gen.nfw_clustered(n, box, 5)
    assert np.all((pos >= 0) & (pos < box))
    assert int(sizes.sum()) == n // 2 and np.count_nonzero(labels >= 0) == n // 2
    assert np.array_equal(np.bincount(labels[labels >= 0]), sizes)
    full = sizes[:-1]                                 # the last halo is cut to the budget
    assert full.min() >= 100 and full.max() <= 200_000
    # maximum-likelihood exponent of a power law on [100, 200000] (continuous
    # approximation) for the drawn sizes
    alphas = np.linspace(1.5, 2.3, 801)
    lo, hi = 100.0, 200_000.0
    ll = [len(full) * np.log((a - 1) / (lo ** (1 - a) - hi ** (1 - a))) - a * np.log(full).sum() for a in alphas]
    assert alphas[int(np.argmax(ll))] == pytest.approx(1.9, abs=0.08)


def test_nfw_radii_follow_the_enclosed_mass():
    # one halo of 20,000 particles with concentration 8 (halo_frac 1): the
    # distances from its centre follow mu(r / r_s) / mu(c) on [0, r_200]
    n, box, c = 20_000, 1000.0, 8.0
    pos, labels, sizes = gen.nfw_clustered(n, box, 9, halo_frac=1.0, m_lo=n, m_hi=n, c_lo=c, c_hi=c)
    assert sizes.tolist() == [n]
    d = pos - pos[0]
    d -= box * np.round(d / box)                      # one halo, far smaller than the box
    ctr = np.median(d, axis=0)
    r = np.linalg.norm(d - ctr, axis=1)
    r200 = (3.0 * n / (4.0 * np.pi * 200.0 * (n / box ** 3))) ** (1.0 / 3.0)
    rs = r200 / c
    mu = lambda x: np.log1p(x) - x / (1.0 + x)        # noqa: E731
    assert r.max() <= r200 * 1.02
    ks = stats.kstest(r, lambda rr: mu(np.minimum(rr / rs, c)) / mu(c))
    assert ks.statistic < 0.02, ks


def test_batch_volumes_recipe():
    vols = gen.batch_volumes(8, 3)
    for p, L in vols:
        n_side = int(L)
        assert L == float(n_side) and len(p) == n_side ** 3
        assert 10 ** 4 * 0.8 <= len(p) <= 10 ** 6 * 1.05
        assert np.all((p >= 0) & (p < L))
    assert len({len(p) for p, _ in vols}) > 1
