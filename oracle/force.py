"""Short-range accelerations and in-range pair counts (FP64 oracle).

Definition (the short-range half of the force split of Sec. 2, evaluated by
direct particle-particle sums): with unit masses and G = 1, for particle i

    a_i = sum_{j != i, s_ij < r_c^2} d_ij f_SR(s_ij),   d_ij = x_j - x_i (minimum image),
    s_ij = |d_ij|^2,  f_SR(s) = (s + eps^2)^(-3/2) - p(s)   (see ``fit``).

The force is attractive: a_i points from i towards j.  r_c < L/2 makes the
minimum image unique.  Three independent enumerations are provided (O(N^2)
brute force, a cell list, and a k-d tree neighbour search) plus a per-row
version for sampled particles; all sum in binary64.

The in-range pair predicate used for pair counts is defined on binary32
operations in units of the fine grid h (see ``binning``):

    eps2_u  = binary32(eps^2 / h^2),  rc2p_u = binary32((r_c^2 + eps^2) / h^2)
    S       = binary32(qA_j - qA_i + m M)       (chunk anchors, image m; exact)
    xj'     = fl32(off_j + S),   dx = fl32(xj' - off_i)      (per axis)
    s'      = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps2_u)))
    in range  <=>  s' < rc2p_u,  j != i.

A pair's count is the number of ordered (i, j) passing it.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from . import fp32
from .fit import f_sr


def min_image(d, box):
    return d - box * np.round(d / box)


def accel_brute(pos, box, rc, eps, c, block=256):
    """O(N^2) minimum-image sum (tiny inputs)."""
    pos = np.asarray(pos, np.float64)
    n = len(pos)
    acc = np.zeros((n, 3))
    cnt = np.zeros(n, dtype=np.int64)
    for i0 in range(0, n, block):
        xi = pos[i0:i0 + block]
        d = min_image(pos[None, :, :] - xi[:, None, :], box)
        s = np.sum(d * d, axis=2)
        m = s < rc * rc
        idx = np.arange(i0, min(n, i0 + block))
        m[np.arange(len(idx)), idx] = False
        f = np.where(m, f_sr(np.where(m, s, 1.0), eps, c), 0.0)
        acc[i0:i0 + block] = np.sum(d * f[:, :, None], axis=1)
        cnt[i0:i0 + block] = m.sum(axis=1)
    return acc, cnt


def accel_celllist(pos, box, rc, eps, c):
    """Cell-list sum: cells of side >= r_c, 27 neighbour cells with images.

    Needs at least 3 cells per axis (distinct neighbours); otherwise falls
    back to brute force.
    """
    pos = _wrap_for_tree(pos, box)
    n = len(pos)
    nc = int(np.floor(box / rc))
    if nc < 3:
        return accel_brute(pos, box, rc, eps, c)
    side = box / nc
    cid3 = np.minimum((pos / side).astype(np.int64), nc - 1)
    cid = (cid3[:, 0] * nc + cid3[:, 1]) * nc + cid3[:, 2]
    order = np.argsort(cid, kind="stable")
    start = np.searchsorted(cid[order], np.arange(nc ** 3 + 1))
    acc = np.zeros((n, 3))
    cnt = np.zeros(n, dtype=np.int64)
    for cx in range(nc):
        for cy in range(nc):
            for cz in range(nc):
                ci = (cx * nc + cy) * nc + cz
                ii = order[start[ci]:start[ci + 1]]
                if ii.size == 0:
                    continue
                xi = pos[ii]
                ai = np.zeros((ii.size, 3))
                ni = np.zeros(ii.size, dtype=np.int64)
                for ox in (-1, 0, 1):
                    for oy in (-1, 0, 1):
                        for oz in (-1, 0, 1):
                            jx, jy, jz = cx + ox, cy + oy, cz + oz
                            shift = np.array([np.floor_divide(jx, nc), np.floor_divide(jy, nc),
                                              np.floor_divide(jz, nc)], dtype=np.float64) * box
                            cj = ((jx % nc) * nc + (jy % nc)) * nc + (jz % nc)
                            jj = order[start[cj]:start[cj + 1]]
                            if jj.size == 0:
                                continue
                            d = (pos[jj] + shift)[None, :, :] - xi[:, None, :]
                            s = np.sum(d * d, axis=2)
                            m = (s < rc * rc) & (jj[None, :] != ii[:, None])
                            f = np.where(m, f_sr(np.where(m, s, 1.0), eps, c), 0.0)
                            ai += np.sum(d * f[:, :, None], axis=1)
                            ni += m.sum(axis=1)
                acc[ii] = ai
                cnt[ii] = ni
    return acc, cnt


def _wrap_for_tree(pos, box):
    p = np.mod(np.asarray(pos, np.float64), box)
    p[p >= box] = 0.0
    return p


def accel_kdtree(pos, box, rc, eps, c):
    """Sum over the unordered pairs a periodic k-d tree finds within r_c."""
    pos = _wrap_for_tree(pos, box)
    n = len(pos)
    tree = cKDTree(pos, boxsize=box)
    pairs = tree.query_pairs(rc, output_type="ndarray")
    i, j = pairs[:, 0], pairs[:, 1]
    d = min_image(pos[j] - pos[i], box)
    s = np.sum(d * d, axis=1)
    keep = s < rc * rc
    i, j, d, s = i[keep], j[keep], d[keep], s[keep]
    w = d * f_sr(s, eps, c)[:, None]
    acc = np.zeros((n, 3))
    for ax in range(3):
        acc[:, ax] = np.bincount(i, weights=w[:, ax], minlength=n) - \
            np.bincount(j, weights=w[:, ax], minlength=n)
    cnt = np.bincount(i, minlength=n) + np.bincount(j, minlength=n)
    return acc, cnt


def accel_rows(pos, box, rc, eps, c, rows, tree=None):
    """a_i for the particle indices in ``rows`` only (sampled comparison)."""
    pos = _wrap_for_tree(pos, box)
    if tree is None:
        tree = cKDTree(pos, boxsize=box)
    rows = np.asarray(rows, dtype=np.int64)
    acc = np.zeros((rows.size, 3))
    cnt = np.zeros(rows.size, dtype=np.int64)
    nbrs = tree.query_ball_point(pos[rows], rc)
    for k, (i, nb) in enumerate(zip(rows, nbrs)):
        nb = np.asarray(nb, dtype=np.int64)
        nb = nb[nb != i]
        d = min_image(pos[nb] - pos[i], box)
        s = np.sum(d * d, axis=1)
        m = s < rc * rc
        acc[k] = np.sum(d[m] * f_sr(s[m], eps, c)[:, None], axis=0)
        cnt[k] = int(m.sum())
    return acc, cnt


# ----------------------------------------------------------------------------
# binary32 in-range predicate (bit-exact pair counts)
# ----------------------------------------------------------------------------

def unit_constants(box, n_c, b, rc, eps):
    """(h, eps2_u, rc2p_u) of the predicate, per the spec in the module doc."""
    M = n_c << b
    h = box / M
    h2 = h * h
    e64 = eps * eps
    return h, fp32.f32(e64 / h2), fp32.f32((rc * rc + e64) / h2)


def pair_predicate(off_i, off_j, shift, eps2_u, rc2p_u):
    """Vectorised binary32 predicate; off_* (k,3) float32, shift (k,3) ints."""
    S = fp32.f32(shift)
    d = []
    for ax in range(3):
        xj = fp32.add32(off_j[:, ax], S[:, ax])
        d.append(fp32.sub32(xj, off_i[:, ax]))
    s = fp32.fma32(d[0], d[0], np.full(len(d[0]), eps2_u, dtype=np.float32))
    s = fp32.fma32(d[1], d[1], s)
    s = fp32.fma32(d[2], d[2], s)
    return s < rc2p_u


def candidate_pairs(pos, box, radius, rows=None, tree=None):
    """Ordered candidate pairs (i, j), i != j, with minimum-image distance
    below ``radius`` and their image vectors m (x_j - x_i + m L is the
    minimum-image displacement)."""
    pos = _wrap_for_tree(pos, box)
    if rows is None:
        tree = cKDTree(pos, boxsize=box) if tree is None else tree
        pr = tree.query_pairs(radius, output_type="ndarray")
        i = np.concatenate([pr[:, 0], pr[:, 1]])
        j = np.concatenate([pr[:, 1], pr[:, 0]])
    else:
        tree = cKDTree(pos, boxsize=box) if tree is None else tree
        rows = np.asarray(rows, dtype=np.int64)
        nbrs = tree.query_ball_point(pos[rows], radius)
        lens = np.array([len(x) for x in nbrs], dtype=np.int64)
        i = np.repeat(rows, lens)
        j = np.concatenate([np.asarray(x, dtype=np.int64) for x in nbrs]) if lens.sum() else \
            np.zeros(0, dtype=np.int64)
        keep = i != j
        i, j = i[keep], j[keep]
    raw = pos[j] - pos[i]
    m = -np.round(raw / box).astype(np.int64)
    return i, j, m


def pair_counts_fp32(binned, volumes, rc, eps, rows=None, margin=1e-3):
    """Per-particle in-range counts under the binary32 predicate.

    ``rows``: optional original indices (global over the batch) to count
    for; default all.  Returns int64 counts aligned with ``rows`` (or all
    particles).
    """
    b = binned["sub_bits"]
    slot = binned["slot_of"]
    chunk = slot // binned["chunk"]
    off = binned["slot_pos"][slot, :3]
    qa = binned["chunk_anchor"][chunk]
    n_tot = binned["n"]
    out_all = np.zeros(n_tot, dtype=np.int64)
    base = 0
    for (pos, box), n_c in zip(volumes, binned["n_cells"]):
        nv = len(pos)
        M = n_c << b
        _, eps2_u, rc2p_u = unit_constants(box, n_c, b, rc, eps)
        loc_rows = None
        if rows is not None:
            rr = np.asarray(rows, dtype=np.int64)
            loc_rows = rr[(rr >= base) & (rr < base + nv)] - base
            if loc_rows.size == 0:
                base += nv
                continue
        i, j, m = candidate_pairs(pos, box, rc * (1.0 + margin), rows=loc_rows)
        gi, gj = i + base, j + base
        for k0 in range(0, len(gi), 1 << 22):
            sl = slice(k0, k0 + (1 << 22))
            shift = qa[gj[sl]] - qa[gi[sl]] + m[sl] * M
            ok = pair_predicate(off[gi[sl]], off[gj[sl]], shift, eps2_u, rc2p_u)
            out_all += np.bincount(gi[sl][ok], minlength=n_tot)
        base += nv
    if rows is None:
        return out_all
    return out_all[np.asarray(rows, dtype=np.int64)]
