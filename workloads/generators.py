"""Seeded particle-set generators (NumPy, FP64, CPU only).

Every generator takes an explicit integer seed and draws from NumPy's PCG64
bit generator, so the oracle and the GPU tests see identical inputs.  Box
lengths are in units of the mean inter-particle spacing ("cells"), as in the
simulation the paper describes, whose particle count equals its PM grid size
(Sec. 3.1: 8192^3 particles; Sec. 4.1: 8192^3 PM grid), i.e. a mean density
of one particle per cell.

None of these functions implement the short-range force method; they only
stand in for the paper's particle data (Sec. 3.1 initial conditions from the
Zel'dovich approximation; Sec. 3.3/4.3 NFW halos), which is not available.
"""
from __future__ import annotations

import numpy as np
from scipy.special import lambertw


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _wrap(pos: np.ndarray, box: float) -> np.ndarray:
    """Fold positions into [0, box); values that round to box become 0."""
    pos = np.mod(pos, box)
    pos[pos >= box] = 0.0
    return pos


def uniform_box(n: int, box: float, seed: int) -> np.ndarray:
    """n points uniform in the periodic cube [0, box)^3, shape (n, 3) float64."""
    return _rng(seed).uniform(0.0, box, size=(int(n), 3))


def lattice(n_side: int, box: float, offset: float = 0.5) -> np.ndarray:
    """Simple cubic lattice of n_side^3 points at (i + offset) * box / n_side.

    Order: C order over (ix, iy, iz) with iz fastest.
    """
    a = box / n_side
    i = (np.arange(n_side, dtype=np.float64) + offset) * a
    gx, gy, gz = np.meshgrid(i, i, i, indexing="ij")
    return np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)


def zeldovich_displacement(n_side: int, box: float, rms: float, seed: int) -> np.ndarray:
    """Zel'dovich displacement field psi on the n_side^3 lattice (Sec. 3.1).

    A real Gaussian white-noise field is Fourier transformed and shaped so
    that <|delta(k)|^2> is proportional to k^-2; the displacement is
    psi(k) = i k delta(k) / k^2 (zero mean mode, Nyquist planes zeroed), and
    psi is rescaled so that sqrt(<|psi|^2>) = rms (rms of the displacement
    magnitude, in cells).  Returns shape (n_side^3, 3), lattice order.
    """
    n = int(n_side)
    w = _rng(seed).standard_normal((n, n, n))
    W = np.fft.rfftn(w)
    kf = 2.0 * np.pi * np.fft.fftfreq(n, d=box / n)
    kr = 2.0 * np.pi * np.fft.rfftfreq(n, d=box / n)
    kx, ky, kz = np.meshgrid(kf, kf, kr, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    amp = W / (k2 * np.sqrt(k2))          # delta(k)/k^2 with |delta| ~ k^-1
    amp[0, 0, 0] = 0.0
    if n % 2 == 0:
        amp[n // 2, :, :] = 0.0
        amp[:, n // 2, :] = 0.0
        amp[:, :, -1] = 0.0
    psi = np.empty((n, n, n, 3))
    for axis, kk in enumerate((kx, ky, kz)):
        psi[..., axis] = np.fft.irfftn(1j * kk * amp, s=(n, n, n), axes=(0, 1, 2))
    psi = psi.reshape(-1, 3)
    scale = rms / np.sqrt(np.mean(np.sum(psi * psi, axis=1)))
    return psi * scale


def zeldovich(n_side: int, box: float, rms: float, seed: int):
    """Zel'dovich-displaced lattice: returns (positions, psi), both (n^3, 3)."""
    psi = zeldovich_displacement(n_side, box, rms, seed)
    pos = _wrap(lattice(n_side, box) + psi, box)
    return pos, psi


def _nfw_mu(x):
    return np.log1p(x) - x / (1.0 + x)


def nfw_clustered(n_total: int, box: float, seed: int, halo_frac: float = 0.5,
                  m_lo: float = 100.0, m_hi: float = 200000.0, slope: float = 1.9,
                  c_lo: float = 5.0, c_hi: float = 15.0):
    """Halo-clustered set: NFW halos plus a uniform background.

    - halo particle budget round(halo_frac * n_total); halo sizes N_h drawn
      from dN/dM ~ M^-slope on [m_lo, m_hi] by inverse CDF (floor to an
      integer), drawn until the budget is reached; the last halo is cut to
      fit the budget exactly;
    - concentration c ~ U[c_lo, c_hi]; r_200 such that the mean density
      inside it is 200 times the box mean density; r_s = r_200 / c;
    - radii by inverse CDF of the NFW enclosed mass mu(x) = ln(1+x) - x/(1+x)
      on [0, c] (closed form through the principal Lambert W branch);
      isotropic directions; centres uniform; positions wrapped;
    - the particle order is a seeded random permutation.

    Returns (positions (n_total, 3), labels (n_total,) int64 with -1 for
    background, halo_sizes (n_halo,) int64).
    """
    rng = _rng(seed)
    n_total = int(n_total)
    budget = int(round(halo_frac * n_total))
    e = 1.0 - slope
    lo_e, hi_e = m_lo ** e, m_hi ** e
    sizes = []
    have = 0
    while have < budget:
        u = rng.uniform(0.0, 1.0, size=4096)
        m = np.floor((lo_e + u * (hi_e - lo_e)) ** (1.0 / e)).astype(np.int64)
        m = np.clip(m, int(m_lo), int(m_hi))
        for mh in m:
            take = min(int(mh), budget - have)
            sizes.append(take)
            have += take
            if have >= budget:
                break
    sizes = np.asarray(sizes, dtype=np.int64)
    n_h = sizes.size
    conc = rng.uniform(c_lo, c_hi, size=n_h)
    rho_mean = n_total / box ** 3
    r200 = (3.0 * sizes / (4.0 * np.pi * 200.0 * rho_mean)) ** (1.0 / 3.0)
    rs = r200 / conc
    centres = rng.uniform(0.0, box, size=(n_h, 3))

    rep_c = np.repeat(conc, sizes)
    rep_rs = np.repeat(rs, sizes)
    rep_ctr = np.repeat(centres, sizes, axis=0)
    u = rng.uniform(0.0, 1.0, size=budget)
    m = u * _nfw_mu(rep_c)
    w0 = lambertw(-np.exp(-1.0 - m), 0).real
    x = -1.0 / w0 - 1.0
    r = x * rep_rs
    cth = rng.uniform(-1.0, 1.0, size=budget)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=budget)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    dirs = np.stack([sth * np.cos(phi), sth * np.sin(phi), cth], axis=1)
    halo_pos = rep_ctr + r[:, None] * dirs
    bg = rng.uniform(0.0, box, size=(n_total - budget, 3))
    pos = np.concatenate([halo_pos, bg], axis=0)
    labels = np.concatenate([np.repeat(np.arange(n_h, dtype=np.int64), sizes),
                             np.full(n_total - budget, -1, dtype=np.int64)])
    order = rng.permutation(n_total)
    return _wrap(pos[order], box), labels[order], sizes


def batch_volumes(n_vol: int, seed: int, log_lo: float = 4.0, log_hi: float = 6.0,
                  rms: float = 0.5):
    """Independent periodic Zel'dovich sub-volumes for the batched workload.

    Volume sizes: N = 10^U(log_lo, log_hi), n_side = round(N^(1/3)),
    N_v = n_side^3, box side L_v = n_side (mean density one per cell).
    Volume v uses seed * 1000 + v for its displacement field.
    Returns a list of (positions (N_v, 3), L_v).
    """
    rng = _rng(seed)
    u = rng.uniform(log_lo, log_hi, size=int(n_vol))
    out = []
    for v, uu in enumerate(u):
        n_side = int(round((10.0 ** uu) ** (1.0 / 3.0)))
        pos, _ = zeldovich(n_side, float(n_side), rms, seed * 1000 + v)
        out.append((pos, float(n_side)))
    return out


def two_body(r: float, box: float, axis: int = 0, centre=None) -> np.ndarray:
    """Two particles separated by r along one axis, centred in the box."""
    c = np.full(3, box / 2.0) if centre is None else np.asarray(centre, float)
    d = np.zeros(3)
    d[axis] = r / 2.0
    return np.stack([c - d, c + d])


def random_directions(n: int, dim: int, seed: int) -> np.ndarray:
    """n unit vectors in R^dim (for directional finite differences)."""
    v = _rng(seed).standard_normal((int(n), int(dim)))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def velocities(n: int, seed: int, scale: float = 0.1) -> np.ndarray:
    """Gaussian initial velocities (n, 3), per-component std `scale`."""
    return scale * _rng(seed).standard_normal((int(n), 3))
