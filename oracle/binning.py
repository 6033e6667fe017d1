"""Cell binning, sub-cell order and 32- or 64-particle chunks (bit-exact spec).

This is the partition step of the paper's short-range timestep (Sec. 2.1,
step 1: each node volume is partitioned into overlapping data blocks holding
"active" particles, whose neighbours within the cutoff are read as "passive"
ones).  Here the blocks are chunks of at most C spatially consecutive
particles inside a cell (32 or 64); a chunk's passive set is every particle within r_c
of it, read from the neighbouring cells.

Spec, per volume of side L with n_c cells per axis and b sub-cell bits:

1. wrap:   x < 0 -> x + L; then x >= L -> x - L (inputs must lie in [-L, 2L)).
2. grid:   M = n_c * 2^b fine cells per axis, h = L / M (binary64 division).
           t = x / h (binary64), q = min(floor(t), M - 1) per axis.
3. cells:  cell = q >> b (side 2^b fine cells = L / n_c), sub = q & (2^b - 1).
           global cell id = base_v + (cz * n_c + cy) * n_c + cx, volumes in
           order, base_v = sum of n_c^3 over earlier volumes.
4. key:    (global cell id << 3b) | morton(sub), morton bit 3i = bit i of x,
           3i+1 of y, 3i+2 of z.  Particles are ordered by key, ties by the
           original index (a stable sort).
5. chunks: each cell's run of n particles is cut into ceil(n / C) chunks of
           C consecutive particles (last one ragged; C = 32 or 64); chunk ids
           follow cell order.  Chunk k owns slots [Ck, Ck + C).
6. anchor: the fine-cell coordinates qA of the chunk's first particle; the
           chunk origin is qA * h (binary64).
7. offset: per particle, off = binary32(t - qA) (the binary64 difference is
           exact), i.e. the position relative to the chunk origin in units
           of h.  Slot value (off_x, off_y, off_z, 1); empty slots hold
           (1e30, 1e30, 1e30, 0) and original index -1.
8. bbox:   per chunk, the per-axis min and max of its particles' offsets.
"""
from __future__ import annotations

import numpy as np

from .fp32 import f32

CHUNK = 32
PAD = np.float32(1e30)


def wrap_positions(x, box: float) -> np.ndarray:
    x = np.array(x, dtype=np.float64, copy=True)
    if not np.all(np.isfinite(x)) or np.any(x < -box) or np.any(x >= 2.0 * box):
        raise ValueError("positions must be finite and lie in [-L, 2L)")
    neg = x < 0.0
    x[neg] = x[neg] + box
    big = x >= box
    x[big] = x[big] - box
    return x


def morton3(sx, sy, sz, bits: int) -> np.ndarray:
    code = np.zeros(np.shape(sx), dtype=np.uint64)
    for i in range(bits):
        code |= ((sx >> i) & 1).astype(np.uint64) << np.uint64(3 * i)
        code |= ((sy >> i) & 1).astype(np.uint64) << np.uint64(3 * i + 1)
        code |= ((sz >> i) & 1).astype(np.uint64) << np.uint64(3 * i + 2)
    return code


def fine_coords(x, box: float, n_c: int, b: int):
    """Return (t, q): binary64 positions in fine-cell units and their cells."""
    M = n_c << b
    h = box / M
    xw = wrap_positions(x, box)
    t = xw / h
    q = np.minimum(np.floor(t).astype(np.int64), M - 1)
    return t, q


def bin_particles(volumes, n_cells, sub_bits: int, chunk: int = CHUNK) -> dict:
    """Bin a batch of volumes.

    volumes: list of (positions (n_v, 3) float64, L_v); n_cells: list of n_c
    per volume; chunk: particles per chunk C.  Returns arrays in the sorted /
    chunked layout plus the per-particle fine coordinates.
    """
    b = int(sub_bits)
    C = int(chunk)
    ts, qs, cells, keys, vols = [], [], [], [], []
    base = 0
    for v, ((pos, box), n_c) in enumerate(zip(volumes, n_cells)):
        t, q = fine_coords(pos, box, n_c, b)
        c = q >> b
        sub = q & ((1 << b) - 1)
        cg = base + (c[:, 2] * n_c + c[:, 1]) * n_c + c[:, 0]
        key = (cg.astype(np.uint64) << np.uint64(3 * b)) | morton3(sub[:, 0], sub[:, 1], sub[:, 2], b)
        ts.append(t); qs.append(q); cells.append(cg); keys.append(key)
        vols.append(np.full(len(pos), v, dtype=np.int64))
        base += n_c ** 3
    total_cells = base
    t = np.concatenate(ts); q = np.concatenate(qs)
    cell = np.concatenate(cells); key = np.concatenate(keys); vol = np.concatenate(vols)
    n = len(key)

    perm = np.argsort(key, kind="stable")
    key_s = key[perm]
    cell_s = cell[perm]
    cell_start = np.searchsorted(cell_s, np.arange(total_cells + 1), side="left")
    counts = np.diff(cell_start)
    nch = (counts + C - 1) // C
    cell_chunk_start = np.concatenate([[0], np.cumsum(nch)]).astype(np.int64)
    n_chunks = int(cell_chunk_start[-1])

    rank = np.arange(n) - cell_start[cell_s]
    chunk_of = cell_chunk_start[cell_s] + rank // C
    slot_of = chunk_of * C + rank % C
    first = cell_start[cell_s] + (rank // C) * C
    q_s = q[perm]
    t_s = t[perm]
    qa = q_s[first]
    off = f32(t_s - qa)

    slot_pos = np.zeros((n_chunks * C, 4), dtype=np.float32)
    slot_pos[:, :3] = PAD
    slot_pos[slot_of, :3] = off
    slot_pos[slot_of, 3] = 1.0
    slot_idx = np.full(n_chunks * C, -1, dtype=np.int64)
    slot_idx[slot_of] = perm

    chunk_anchor = np.zeros((n_chunks, 3), dtype=np.int64)
    chunk_anchor[chunk_of] = qa
    chunk_cell = np.zeros(n_chunks, dtype=np.int64)
    chunk_cell[chunk_of] = cell_s
    chunk_vol = np.zeros(n_chunks, dtype=np.int64)
    chunk_vol[chunk_of] = vol[perm]
    chunk_count = np.bincount(chunk_of, minlength=n_chunks).astype(np.int64)
    lo = np.full((n_chunks, 3), np.inf, dtype=np.float32)
    hi = np.full((n_chunks, 3), -np.inf, dtype=np.float32)
    np.minimum.at(lo, chunk_of, off)
    np.maximum.at(hi, chunk_of, off)

    # per original particle: its slot, chunk and offset
    slot_orig = np.empty(n, dtype=np.int64)
    slot_orig[perm] = slot_of
    return dict(
        n=n, sub_bits=b, chunk=C, n_cells=list(n_cells), total_cells=total_cells,
        key_sorted=key_s, perm=perm, cell_start=cell_start,
        cell_chunk_start=cell_chunk_start, n_chunks=n_chunks,
        slot_pos=slot_pos, slot_idx=slot_idx, chunk_anchor=chunk_anchor,
        chunk_cell=chunk_cell, chunk_vol=chunk_vol, chunk_count=chunk_count,
        chunk_lo=lo, chunk_hi=hi, slot_of=slot_orig, t=t, q=q, cell=cell,
    )


def dequantized_positions(binned: dict, volumes) -> np.ndarray:
    """Positions the FP32 offsets represent: (qA + off) * h, in binary64,
    in the original particle order."""
    b = binned["sub_bits"]
    n = binned["n"]
    out = np.empty((n, 3))
    slot = binned["slot_of"]
    chunk = slot // binned["chunk"]
    off = binned["slot_pos"][slot, :3].astype(np.float64)
    qa = binned["chunk_anchor"][chunk].astype(np.float64)
    vol = binned["chunk_vol"][chunk]
    for v, ((pos, box), n_c) in enumerate(zip(volumes, binned["n_cells"])):
        h = box / (n_c << b)
        m = vol == v
        out[m] = (qa[m] + off[m]) * h
    return out
