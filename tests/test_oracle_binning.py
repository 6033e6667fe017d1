"""Pins for the binning spec (oracle.binning): containment, stable order,
chunk structure, offset accuracy and Morton locality."""
import numpy as np
import pytest

from oracle import binning
from workloads import generators as gen


def _bin(pos, box, n_c=4, b=5):
    return binning.bin_particles([(pos, box)], [n_c], b)


def test_wrap_rules():
    L = 16.0
    x = np.array([-16.0, -1e-300, -3.5, 0.0, 15.999, 16.0, 31.9])
    w = binning.wrap_positions(x, L)
    assert np.all((w >= 0) & (w < L))
    np.testing.assert_array_equal(w, [0.0, 0.0, 12.5, 0.0, 15.999, 0.0, 31.9 - 16.0])
    with pytest.raises(ValueError):
        binning.wrap_positions(np.array([32.0]), L)
    with pytest.raises(ValueError):
        binning.wrap_positions(np.array([np.nan]), L)


def test_fine_cells_contain_positions():
    L = 16.0
    pos = gen.uniform_box(5000, L, 5)
    t, q = binning.fine_coords(pos, L, 4, 5)
    h = L / (4 << 5)                      # a power of two: q*h is exact
    assert np.all(q * h <= pos) and np.all(pos < (q + 1) * h)
    # grid points map to themselves
    k = np.arange(0, 4 << 5)
    tg, qg = binning.fine_coords(np.stack([k * h] * 3, axis=1), L, 4, 5)
    np.testing.assert_array_equal(qg[:, 0], k)


def test_sorted_order_is_stable_by_key():
    pos = gen.uniform_box(3000, 16.0, 6)
    # duplicate positions to create equal keys
    pos = np.concatenate([pos, pos[:500]])
    B = _bin(pos, 16.0)
    perm, key = B["perm"], B["key_sorted"]
    assert sorted(perm.tolist()) == list(range(len(pos)))
    assert np.all(np.diff(key.astype(np.float64)) >= 0)
    same = key[1:] == key[:-1]
    assert np.all(perm[1:][same] > perm[:-1][same])


def test_chunks_cover_cells():
    pos, _, _ = gen.nfw_clustered(6000, 16.0, 8, m_hi=1500.0)
    B = _bin(pos, 16.0)
    counts = np.diff(B["cell_start"])
    nch = np.diff(B["cell_chunk_start"])
    np.testing.assert_array_equal(nch, (counts + 31) // 32)
    cc = B["chunk_count"]
    assert cc.min() >= 1 and cc.max() <= 32
    # every chunk but the last of its cell is full
    last = np.zeros(B["n_chunks"], bool)
    last[B["cell_chunk_start"][1:][nch > 0] - 1] = True
    assert np.all(cc[~last] == 32)
    # slots: valid slots hold each particle exactly once, pads are inert
    idx = B["slot_idx"]
    valid = idx >= 0
    assert np.array_equal(np.sort(idx[valid]), np.arange(len(pos)))
    assert np.all(B["slot_pos"][~valid, :3] == binning.PAD)
    assert np.all(B["slot_pos"][valid, 3] == 1.0)


def test_offsets_reconstruct_positions():
    L = 24.0                                # h not a power of two here
    pos = gen.uniform_box(4000, L, 9)
    B = binning.bin_particles([(pos, L)], [5], 6)
    xr = binning.dequantized_positions(B, [(pos, L)])
    h = L / (5 << 6)
    off = B["slot_pos"][B["slot_of"], :3].astype(np.float64)
    # binary32 rounding of the offset (in units of h) bounds the error
    bound = (np.abs(off) * 2.0 ** -24 + 1e-12) * h
    assert np.all(np.abs(xr - pos) <= bound * 1.0001 + 1e-12)
    # bboxes contain their chunk's offsets
    ch = B["slot_of"] // 32
    assert np.all(B["chunk_lo"][ch] <= off) and np.all(off <= B["chunk_hi"][ch])


def test_morton_blocks_are_cubes():
    b = 3
    g = np.arange(1 << b)
    sx, sy, sz = [a.ravel() for a in np.meshgrid(g, g, g, indexing="ij")]
    code = binning.morton3(sx, sy, sz, b)
    assert np.array_equal(np.sort(code), np.arange(1 << (3 * b), dtype=np.uint64))
    order = np.argsort(code)
    for lev in range(1, b + 1):
        blk = 1 << (3 * lev)
        side = 1 << lev
        for k0 in range(0, len(order), blk):
            sel = order[k0:k0 + blk]
            for a in (sx, sy, sz):
                v = a[sel]
                assert v.max() - v.min() == side - 1 and v.min() % side == 0


def test_batch_volumes_are_independent():
    vols = [(gen.uniform_box(700, 12.0, 1), 12.0), (gen.uniform_box(900, 20.0, 2), 20.0)]
    B = binning.bin_particles(vols, [3, 5], 4)
    # cells of volume 1 follow all cells of volume 0
    assert B["total_cells"] == 27 + 125
    v = B["chunk_vol"]
    assert np.all(np.diff(v) >= 0)
    assert np.all(B["chunk_cell"][v == 0] < 27) and np.all(B["chunk_cell"][v == 1] >= 27)
    # binning one volume alone gives the same local layout
    B1 = binning.bin_particles([vols[1]], [5], 4)
    sel = B["slot_idx"] >= 700
    np.testing.assert_array_equal(B["slot_pos"][B["chunk_vol"].repeat(32) == 1], B1["slot_pos"])
    assert sel.sum() == 900
