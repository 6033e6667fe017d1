"""Most-bound-particle halo centers (FP64 oracle).

The paper's in-situ analysis (Sec. 2.2) finds, for every halo, the member
with the lowest potential ("most bound particle"), with a direct pairwise
potential sum over the halo's members computed by data-parallel
primitives on the GPU.  The paper gives no formula; the reading used here
(the halo treated as isolated, unit masses, G = 1, minimum image in the
periodic box, Plummer softening eps):

    phi_i = - sum_{j in halo(i), j != i} (|d_ij|^2 + eps^2)^(-1/2),

center(halo) = argmin_i phi_i over the halo's members, ties broken by the
smaller particle index.  Particles with label -1 belong to no halo.
"""
from __future__ import annotations

import numpy as np

from .force import min_image


def halo_potentials(pos, labels, box, eps, block=2048):
    """phi_i for every particle (0 for label -1), binary64, O(N_h^2) per halo."""
    pos = np.asarray(pos, np.float64)
    labels = np.asarray(labels)
    phi = np.zeros(len(pos))
    order = np.argsort(labels, kind="stable")
    lab_s = labels[order]
    starts = np.searchsorted(lab_s, np.unique(lab_s[lab_s >= 0]))
    ends = np.searchsorted(lab_s, np.unique(lab_s[lab_s >= 0]), side="right")
    e2 = eps * eps
    for s0, s1 in zip(starts, ends):
        idx = order[s0:s1]
        x = pos[idx]
        out = np.zeros(len(idx))
        for b0 in range(0, len(idx), block):
            d = min_image(x[None, :, :] - x[b0:b0 + block, None, :], box)
            r2 = np.sum(d * d, axis=2) + e2
            inv = 1.0 / np.sqrt(r2)
            k = np.arange(b0, min(len(idx), b0 + block))
            inv[np.arange(len(k)), k] = 0.0                 # no self term
            out[b0:b0 + block] = -inv.sum(axis=1)
        phi[idx] = out
    return phi


def halo_centers(pos, labels, box, eps, n_halos):
    """(center index per halo (-1 if empty), its potential, phi per particle)."""
    labels = np.asarray(labels)
    phi = halo_potentials(pos, labels, box, eps)
    center = np.full(n_halos, -1, dtype=np.int64)
    cphi = np.full(n_halos, np.inf)
    for i in np.argsort(labels, kind="stable"):
        h = labels[i]
        if h < 0:
            continue
        if phi[i] < cphi[h] or (phi[i] == cphi[h] and i < center[h]):
            cphi[h] = phi[i]
            center[h] = i
    return center, cphi, phi


def member_potentials(pos, labels, box, eps, idx):
    """phi_i for the particles idx only (each summed over its own halo), for
    checks of single outputs of large inputs."""
    pos = np.asarray(pos, np.float64)
    labels = np.asarray(labels)
    out = np.zeros(len(idx))
    e2 = eps * eps
    for k, i in enumerate(np.asarray(idx)):
        h = labels[i]
        if h < 0:
            continue
        mem = np.flatnonzero(labels == h)
        mem = mem[mem != i]
        d = min_image(pos[mem] - pos[i], box)
        out[k] = -np.sum(1.0 / np.sqrt(np.sum(d * d, axis=1) + e2))
    return out
