"""Long-range side of the force split and the on-the-fly power spectrum
(FP64 oracle).

Sec. 2: the long-range force comes from a spectrally filtered
particle-mesh (PM) solver on a uniform grid; Sec. 4.1: the matter power
spectrum is measured on the fly by a cloud-in-cell (CIC) deposit onto the
PM grid, a discrete Fourier transform, |delta(k)|^2 binned in |k|, and a
division by the CIC window.  The paper prints no formulas; the readings
(all in this module):

Grid.  n_g^3 points at x = (i, j, k) * D, D = L / n_g, periodic.
CIC.   A particle at x has u = x / D (after folding into [0, L)), cell
       i0 = floor(u), f = u - i0; weight (1 - f) to i0 and f to i0 + 1 per
       axis, the product over axes to the 8 corners (mod n_g).
Delta. counts / nbar - 1, nbar = N / n_g^3.
FFT.   delta_k = sum_x delta(x) exp(-i k . x) (numpy's forward convention),
       k = 2 pi m / L with m the signed integer frequency.
P(k).  P(k_vec) = (L^3 / n_g^6) |delta_k|^2 / W(k)^2,
       W(k) = prod_a sinc^2(k_a D / 2) (the CIC assignment window; the
       measured power carries it squared); modes binned by
       b = round(|m|), b = 1 .. n_g/2; per bin the mean |k|, the mean P
       and the number of modes (both k and -k count).
Force. Poisson with G = 1, unit masses, the mean density removed; the
       long-range part keeps exp(-k^2 sigma^2) of the spectrum, the
       Fourier transform of the Gaussian behind F_long(r) of the split:
         a(k) = i k (4 pi / k^2) exp(-k^2 sigma^2) C(k) / W(k)^2,
       C(k) the DFT of the CIC counts (k = 0 and, per axis, the Nyquist
       component of the gradient set to 0), a(x) = ifft(a(k)) / D^3,
       interpolated back to the particles with the CIC weights.  One W
       compensates the deposit, the other the interpolation.
"""
from __future__ import annotations

import numpy as np

from .force import _wrap_for_tree


def cic_weights(pos, box, n_g):
    """Per particle: base cell (n, 3) int and fractional offsets (n, 3)."""
    x = _wrap_for_tree(pos, box)
    u = np.asarray(x, np.float64) * (n_g / box)
    i0 = np.floor(u)
    f = u - i0
    i0 = i0.astype(np.int64) % n_g
    return i0, f


def cic_deposit(pos, box, n_g):
    """CIC particle counts on the grid, array (n_g, n_g, n_g) indexed [x, y, z]."""
    i0, f = cic_weights(pos, box, n_g)
    grid = np.zeros((n_g, n_g, n_g))
    for dx in (0, 1):
        wx = f[:, 0] if dx else 1.0 - f[:, 0]
        for dy in (0, 1):
            wy = f[:, 1] if dy else 1.0 - f[:, 1]
            for dz in (0, 1):
                wz = f[:, 2] if dz else 1.0 - f[:, 2]
                np.add.at(grid, ((i0[:, 0] + dx) % n_g, (i0[:, 1] + dy) % n_g, (i0[:, 2] + dz) % n_g),
                          wx * wy * wz)
    return grid


def cic_interpolate(field, pos, box):
    """Values of a grid field (n_g, n_g, n_g[, c]) at the particles, CIC weights."""
    n_g = field.shape[0]
    i0, f = cic_weights(pos, box, n_g)
    out = 0.0
    for dx in (0, 1):
        wx = f[:, 0] if dx else 1.0 - f[:, 0]
        for dy in (0, 1):
            wy = f[:, 1] if dy else 1.0 - f[:, 1]
            for dz in (0, 1):
                wz = f[:, 2] if dz else 1.0 - f[:, 2]
                w = wx * wy * wz
                v = field[(i0[:, 0] + dx) % n_g, (i0[:, 1] + dy) % n_g, (i0[:, 2] + dz) % n_g]
                out = out + (w[:, None] * v if v.ndim == 2 else w * v)
    return out


def wavenumbers(n_g, box):
    """Signed integer frequencies m (n_g,) and k = 2 pi m / L along one axis."""
    m = np.fft.fftfreq(n_g, d=1.0 / n_g)
    return m, 2.0 * np.pi * m / box


def cic_window(n_g, box):
    """W(k) = prod_a sinc^2(k_a D / 2) on the full grid [x, y, z]."""
    _, k = wavenumbers(n_g, box)
    h = 0.5 * k * (box / n_g)
    s = np.ones_like(h)
    nz = h != 0.0
    s[nz] = np.sin(h[nz]) / h[nz]
    w1 = s * s
    return w1[:, None, None] * w1[None, :, None] * w1[None, None, :]


def power_spectrum(pos, box, n_g):
    """(k_mean, P, modes) per shell b = 1 .. n_g/2 of the CIC-compensated
    power spectrum of the particle set."""
    counts = cic_deposit(pos, box, n_g)
    nbar = len(pos) / n_g ** 3
    delta = counts / nbar - 1.0
    dk = np.fft.fftn(delta)
    p3 = (box ** 3 / n_g ** 6) * np.abs(dk) ** 2 / cic_window(n_g, box) ** 2
    m, k1 = wavenumbers(n_g, box)
    mm = np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2)
    kk = np.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + k1[None, None, :] ** 2)
    b = np.rint(mm).astype(np.int64)
    nb = n_g // 2
    sel = (b >= 1) & (b <= nb)
    modes = np.bincount(b[sel], minlength=nb + 1)[1:]
    psum = np.bincount(b[sel], weights=p3[sel], minlength=nb + 1)[1:]
    ksum = np.bincount(b[sel], weights=kk[sel], minlength=nb + 1)[1:]
    with np.errstate(invalid="ignore", divide="ignore"):
        return ksum / modes, psum / modes, modes


def pm_accel_grid(counts, box, sigma):
    """Long-range acceleration on the grid, array (n_g, n_g, n_g, 3)."""
    n_g = counts.shape[0]
    c_k = np.fft.fftn(counts)
    m, k1 = wavenumbers(n_g, box)
    k2 = k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + k1[None, None, :] ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        g = 4.0 * np.pi * np.exp(-k2 * sigma * sigma) / k2 / cic_window(n_g, box) ** 2
    g[0, 0, 0] = 0.0
    kg = k1.copy()
    kg[np.abs(m) == n_g // 2] = 0.0                     # no gradient at the Nyquist plane
    dvol = (box / n_g) ** 3
    out = np.empty((n_g, n_g, n_g, 3))
    shapes = [(n_g, 1, 1), (1, n_g, 1), (1, 1, n_g)]
    for a in range(3):
        ak = 1j * kg.reshape(shapes[a]) * g * c_k
        out[..., a] = np.real(np.fft.ifftn(ak)) / dvol
    return out


def pm_accel(pos, box, n_g, sigma):
    """Long-range PM acceleration of every particle (n, 3)."""
    grid = pm_accel_grid(cic_deposit(pos, box, n_g), box, sigma)
    return cic_interpolate(grid, pos, box)
