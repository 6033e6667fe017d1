"""sr_bin on the GPU is bit-exact against the oracle's binning spec."""
from fractions import Fraction

import numpy as np
import pytest

from workloads import configs as wc
from workloads import generators as gen

from helpers import make_plan, oracle_binning, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _run_bin(vols, params, **kw):
    pos = np.concatenate([p for p, _ in vols])
    plan = make_plan(vols, params, **kw)
    plan.bin(torch.from_numpy(pos).cuda())
    torch.cuda.synchronize()
    return plan


def _compare(plan, vols):
    B = oracle_binning(plan, vols)
    info = plan.info()
    assert info["n_chunks"] == B["n_chunks"]
    np.testing.assert_array_equal(to_np(plan.export("perm")), B["perm"])
    np.testing.assert_array_equal(to_np(plan.export("cell_start")), B["cell_start"])
    np.testing.assert_array_equal(to_np(plan.export("cell_chunk_start")), B["cell_chunk_start"])
    sp = to_np(plan.export("slot_pos"))
    assert sp.view(np.uint32).tobytes() == B["slot_pos"].view(np.uint32).tobytes()
    np.testing.assert_array_equal(to_np(plan.export("slot_idx")), B["slot_idx"])
    meta = to_np(plan.export("chunk_meta"))
    np.testing.assert_array_equal(meta[:, :3], B["chunk_anchor"])
    np.testing.assert_array_equal(meta[:, 3], B["chunk_vol"])
    lo = to_np(plan.export("chunk_lo"))
    hi = to_np(plan.export("chunk_hi"))
    np.testing.assert_array_equal(lo[:, :3].view(np.uint32), B["chunk_lo"].view(np.uint32))
    np.testing.assert_array_equal(hi[:, :3].view(np.uint32), B["chunk_hi"].view(np.uint32))
    np.testing.assert_array_equal(lo[:, 3].view(np.int32), B["chunk_count"])


@pytest.mark.parametrize("chunk", [32, 64])
@pytest.mark.parametrize("name", ["uniform4k", "zeldovich128", "clustered256", "batch64"])
def test_bin_bit_exact_small(name, chunk):
    cfg = wc.small_variant(name)
    w = wc.make_workload(cfg)
    plan = _run_bin(w["volumes"], w["params"], chunk_size=chunk)
    assert plan.info()["chunk_size"] == chunk
    _compare(plan, w["volumes"])


@pytest.mark.parametrize("sub_bits,n_cells,chunk", [(1, 0, 32), (4, 3, 64), (8, 5, 32), (6, 4, 64)])
def test_bin_geometry_variants(sub_bits, n_cells, chunk):
    pos = gen.uniform_box(3000, 17.0, 21)            # h not a power of two
    vols = [(pos, 17.0)]
    plan = _run_bin(vols, dict(rc=3.0, eps=0.1, sigma=0.8), sub_bits=sub_bits, n_cells=[n_cells],
                    chunk_size=chunk)
    _compare(plan, vols)


def test_bin_positions_next_to_fine_cell_faces():
    # box 23 with 5 cells of 64 fine cells: h = 23/320 is not a power of two,
    # so the fine cell and the offset come from the corrected binary64
    # quotient x / h.  Positions within three ulps of the faces k h (and a
    # few below 0, folded) are where a quotient off by one ulp would change
    # the cell or the offset.
    L, n_c, b = 23.0, 5, 6
    h = L / (n_c << b)
    rng = np.random.default_rng(31)
    pos = rng.integers(0, n_c << b, (4000, 3)) * h
    steps = rng.integers(-3, 4, pos.shape)
    for s in range(3):
        pos = np.where(steps > s, np.nextafter(pos, np.inf), pos)
        pos = np.where(steps < -s, np.nextafter(pos, -np.inf), pos)
    # one to three ulps below the box side, where x / h can round up to M
    # (cell index clamped to M - 1, offset taken from the unclamped quotient)
    top = [L]
    for _ in range(3):
        top.append(float(np.nextafter(top[-1], -np.inf)))
    pos[:60] = np.array(top[1:])[rng.integers(0, 3, (60, 3))]
    vols = [(pos, L)]
    plan = _run_bin(vols, dict(rc=3.0, eps=0.1, sigma=0.8), sub_bits=b, n_cells=[n_c])
    _compare(plan, vols)


def test_bin_edge_positions():
    L = 16.0
    pos = gen.uniform_box(500, L, 3)
    pos[:6] = [[0, 0, 0], [L - 1e-13, L - 1e-13, L - 1e-13], [-1e-300, 5, 5],
               [-L, 2 * L - 1e-9, 3.0], [L, 0.5, 0.5], [4.0, 4.0, 4.0]]
    pos[6:40] = pos[5]                               # duplicates: stable tie order
    vols = [(pos, L)]
    plan = _run_bin(vols, dict(rc=3.0, eps=0.1, sigma=0.8))
    _compare(plan, vols)
    plan.status()


def test_bin_flags_out_of_range():
    from paper_1411_3396_b300 import SrError
    L = 16.0
    pos = gen.uniform_box(100, L, 4)
    pos[7, 1] = 2 * L + 1.0
    pos[9, 2] = np.nan
    plan = _run_bin([(pos, L)], dict(rc=3.0, eps=0.1, sigma=0.8))
    with pytest.raises(SrError) as e:
        plan.status()
    assert e.value.code == 5
    plan.status()                                    # flag cleared


def test_bin_capacity_errors():
    from paper_1411_3396_b300 import Plan, SrError
    plan = Plan(16.0, 3.0, 0.1, 0.8, 100)
    with pytest.raises(SrError) as e:
        plan.bin(torch.zeros((101, 3), dtype=torch.float64, device="cuda"))
    assert e.value.code == 3
    with pytest.raises(SrError):
        Plan(5.0, 3.0, 0.1, 0.8, 100)                # box <= 2 r_c
    with pytest.raises(SrError):
        Plan(16.0, 3.0, 0.0, 0.8, 100)               # eps must be > 0
    with pytest.raises(SrError):
        Plan(16.0, 3.0, 0.1, 0.8, 100, n_cells=6)    # cell side 2.67 < r_c
    with pytest.raises(SrError):
        Plan(16.0, 3.0, 0.1, 0.8, 100, chunk_size=48)


def test_bin_partial_fill_and_rebin():
    L = 16.0
    plan = make_plan([(np.zeros((1, 3)), L)], dict(rc=3.0, eps=0.1, sigma=0.8))
    from paper_1411_3396_b300 import Plan
    plan = Plan(L, 3.0, 0.1, 0.8, 5000)
    for seed, n in [(1, 5000), (2, 1234), (3, 1), (4, 4999)]:
        pos = gen.uniform_box(n, L, seed)
        plan.bin(torch.from_numpy(pos).cuda())
        torch.cuda.synchronize()
        _compare(plan, [(pos, L)])


def _cells_of_sizes(sizes, L, n_c, seed, spread=None):
    """Positions with sizes[k] particles in cell k (cells in x order along
    the first row; spread: side of the cube inside the cell that holds them,
    0 = all at one point), shuffled into random caller order."""
    rng = np.random.default_rng(seed)
    side = L / n_c
    parts = []
    for k, m in enumerate(sizes):
        w = side if spread is None else spread
        lo = np.array([k * side, 0.0, 0.0]) + (side - w) / 2
        parts.append(lo + rng.random((m, 3)) * w)
    pos = np.concatenate(parts)
    return pos[rng.permutation(len(pos))]


@pytest.mark.parametrize("chunk", [32, 64])
def test_bin_dense_cells_every_sort_path(chunk):
    # cells of 0..kSmallCell particles are sorted by one warp in registers,
    # up to kSegTile in shared memory by one block, larger ones split on
    # their top bits first (and a bucket still above kSegTile sorted through
    # global memory); sizes at and next to each threshold, a dense blob,
    # and coincident positions (a single fine cell: ties on the Morton code
    # broken by caller index alone)
    L, n_c = 32.0, 8
    side = L / n_c
    sizes = [1, 31, 32, 33, 64, 65, 127, 128]
    pos_a = _cells_of_sizes(sizes, L, n_c, 51) + [0.0, 2 * side, 0.0]                 # cells (k, 2, 0)
    pos_b = _cells_of_sizes([129, 200, 1000, 2047, 2048, 2049, 9000, 0], L, n_c, 52)  # cells (k, 0, 0)
    blob = _cells_of_sizes([0, 0, 20000], L, n_c, 53, spread=0.05) + [0.0, 0.0, 3 * side]   # a few fine cells
    same = np.tile([[3.375 * side, 3.375 * side, 0.375 * side]], (6000, 1))             # one point
    rest = gen.uniform_box(5000, L, 54) * [1.0, 1.0, 3 * side / L] + [0.0, 0.0, 5 * side]   # z cells 5..7
    pos = np.concatenate([pos_a, pos_b, blob, same, rest])
    pos = pos[np.random.default_rng(55).permutation(len(pos))]
    vols = [(pos, L)]
    plan = _run_bin(vols, dict(rc=3.0, eps=0.1, sigma=0.8), n_cells=[n_c], chunk_size=chunk)
    _compare(plan, vols)
    plan.status()
    # the same particles again: the atomics' order changes, the result not
    first = [to_np(plan.export(k)).copy() for k in ("perm", "slot_pos", "slot_idx")]
    plan.bin(torch.from_numpy(pos).cuda())
    for a, k in zip(first, ("perm", "slot_pos", "slot_idx")):
        assert a.tobytes() == to_np(plan.export(k)).tobytes()


@pytest.mark.parametrize("chunk", [32, 64])
def test_bin_tie_runs_each_sort_path(chunk):
    # cells sorted by a warp (129..512 particles) or a block (513..2048 in
    # shared memory, larger ones split and their buckets sorted) order the
    # Morton code first and then each run of equal codes by caller index;
    # a run longer than 32 makes them sort the range on every bit instead.
    # Runs of 2..32 and of 33 and 40 in each path, in distinct cells
    L, n_c = 32.0, 8
    side = L / n_c
    cells = [                           # (particles, extent of the cube that holds them, runs)
        (300, 3.6, [2, 3, 17, 32]),     # warp LSD, runs fixed in place
        (300, 3.6, [2, 33]),            # warp LSD, a run over the limit
        (1500, 3.6, [2, 5, 32, 32]),    # block sort in shared memory
        (1500, 3.6, [40]),              # the same, over the limit
        (6000, 0.8, [2, 9, 31, 32]),    # split: four buckets of about 1500, block sort
        # split: one bucket of 6000 (a 0.5 x 0.5 x 1 box of 1024 fine cells)
        # sorted through global memory, with and without a run over the limit
        (6000, [0.85, 0.35, 0.35], [2, 32]),
        (6000, [0.85, 0.35, 0.35], [33, 3]),
    ]
    # ranges of up to 128 sorted in registers on 32-bit keys (Morton code,
    # position): without runs, and with runs that send the range to the
    # full 64-bit sort (second row of cells)
    small = [(20, 3.6, []), (40, 3.6, [2, 5]), (64, 3.6, [2]), (100, 3.6, [3, 32]), (128, 3.6, [2, 2, 2])]
    parts = []
    for k, (m, ext, runs) in enumerate(small):
        corner = np.array([k * side, 4 * side, 0.0])
        rng = np.random.default_rng(90 + k)
        parts.append(corner + 0.1 + rng.random((m - sum(runs), 3)) * ext)
        for j, r in enumerate(runs):
            parts.append(np.tile(corner + [0.11 + 0.1 * j, 0.02, 0.02], (r, 1)))
    for k, (m, ext, runs) in enumerate(cells):
        corner = np.array([k * side, 2 * side, 0.0])
        rng = np.random.default_rng(60 + k)
        parts.append(corner + 0.1 + rng.random((m - sum(runs), 3)) * ext)
        # each run: coincident particles alone in a fine cell (y, z below
        # the cloud's 0.1; the first row of fine cells), distinct along x
        for j, r in enumerate(runs):
            parts.append(np.tile(corner + [0.11 + 0.1 * j, 0.02, 0.02], (r, 1)))
    pos = np.concatenate(parts)
    pos = pos[np.random.default_rng(77).permutation(len(pos))]
    vols = [(pos, L)]
    plan = _run_bin(vols, dict(rc=3.0, eps=0.1, sigma=0.8), n_cells=[n_c], chunk_size=chunk)
    _compare(plan, vols)
    plan.status()


@pytest.mark.parametrize("sub_bits,chunk", [(6, 32), (3, 64), (6, 64)])
def test_bin_power_of_two_side_with_sub_cells(sub_bits, chunk):
    # box 32, 8 cells: h = 4 / 2^b is a power of two (the integer path of the
    # binning kernels), sub-cells put anchors and slots in different fine cells
    w = wc.make_workload(wc.small_variant("clustered256"))
    plan = _run_bin(w["volumes"], w["params"], sub_bits=sub_bits, n_cells=[8], chunk_size=chunk)
    _compare(plan, w["volumes"])


def _rn(value: Fraction, bits: int) -> Fraction:
    """value rounded to `bits` significant bits, to nearest, ties to even."""
    if value == 0:
        return value
    sign = -1 if value < 0 else 1
    a = abs(value)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    scale = Fraction(2) ** (bits - 1 - e)
    m = a * scale
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return sign * Fraction(fl) / scale


def test_bin_offsets_round_twice_like_the_spec():
    # the offset is binary32(t - qa) with the subtraction in binary64; for a
    # slot near a cell's start under a far anchor the difference needs more
    # than 53 bits, and these pairs are built so that the binary64 rounding
    # lands exactly on a binary32 tie (or just short of one)
    box, b = 32.0, 6                     # 8 cells of 64 fine cells, h = 1/16
    m24 = 10092545                       # odd: a tie rounds it up to even
    tie = Fraction(2 * m24 + 1, 2 ** 19)  # (m24 + 1/2) 2^-18, in [38, 39)
    eps_cases = [Fraction(1, 2 ** 51), Fraction(1, 2 ** 50), Fraction(1, 2 ** 49), Fraction(1, 2 ** 48),
                 Fraction(3, 2 ** 49), Fraction(1, 2 ** 52)]
    pts, expect = [], []
    for n, eps in enumerate(eps_cases):
        cy, cz = n % 4, n // 4            # one cell per case along y, z; x in the first cell
        oy, oz = 64 * cy, 64 * cz        # cell origins in fine units
        t = 40 - tie + eps               # exact in binary64: t in [1, 2), ulp 2^-52
        assert Fraction(float(t)) == t
        d = t - 40                       # offset of the slot against the anchor qa = 40
        twice = _rn(_rn(d, 53), 24)
        once = _rn(d, 24)
        expect.append((n, twice, once))
        # anchor (first in Morton order: its key has only x bits), then the slot
        pts.append([40.25 / 16, (oy + 0.25) / 16, (oz + 0.25) / 16])
        pts.append([float(t) / 16, (oy + 32.5) / 16, (oz + 0.25) / 16])
    # the same on the y axis: the slot's z sub-cell orders it after the anchor
    t = 40 - tie + eps_cases[0]
    pts.append([(64 * 5 + 0.25) / 16, 40.25 / 16, (64 * 5 + 0.25) / 16])
    pts.append([(64 * 5 + 0.25) / 16, float(t) / 16, (64 * 5 + 32.5) / 16])
    pos = np.array(pts)
    assert sum(1 for _, tw, on in expect if tw != on) >= 3      # real double-rounding cases
    vols = [(pos, box)]
    plan = _run_bin(vols, dict(rc=3.0, eps=0.1, sigma=0.8), sub_bits=b, n_cells=[8], chunk_size=32)
    _compare(plan, vols)
    # and the offsets are the twice-rounded values
    sp = to_np(plan.export("slot_pos"))
    idx = to_np(plan.export("slot_idx"))
    for n, twice, _ in expect:
        row = int(np.nonzero(idx == 2 * n + 1)[0][0])
        assert Fraction(float(sp.reshape(-1, 4)[row, 0])) == twice
