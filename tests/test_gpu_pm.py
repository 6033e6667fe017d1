"""Long-range side (sr_pm_*) against the FP64 oracle: the FFT against a
library FFT, CIC counts, delta(k), the CIC-compensated power spectrum and
the PM accelerations element by element, plus conservation, accumulation,
argument errors and the full 256^3 clustered set."""
import numpy as np
import pytest

from oracle import pm as opm
from workloads import configs as wc
from workloads import generators as gen

from helpers import rel_errors

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# binary32 FFT: error relative to the transform's norm grows like
# log2(n) * 2^-24; 3e-6 leaves margin up to n = 1024
FFT_TOL = 3e-6
# power per shell: binary32 delta_k against the FP64 oracle
PK_TOL = 1e-4


def _pm(ng, box, sigma, n):
    from paper_1411_3396_b300 import PM
    return PM(ng, box, sigma, n)


@pytest.mark.parametrize("ng", [16, 32, 64, 128, 256, 512])
def test_fft_matches_library_fft(ng):
    rng = np.random.default_rng(ng)
    x = (rng.standard_normal((ng, ng, ng)) + 1j * rng.standard_normal((ng, ng, ng))).astype(np.complex64)
    p = _pm(ng, float(ng), 0.8, 10)
    d = torch.from_numpy(x).cuda()
    p.fft(d)
    ref = np.fft.fftn(x.astype(np.complex128))
    got = d.cpu().numpy()
    assert np.linalg.norm(got - ref) <= FFT_TOL * np.linalg.norm(ref)
    p.fft(d, inverse=True)
    back = d.cpu().numpy() / ng ** 3
    assert np.linalg.norm(back - x) <= 2 * FFT_TOL * np.linalg.norm(x)
    p.close()


@pytest.fixture(scope="module")
def clustered():
    cfg = wc.small_variant("clustered256")
    w = wc.make_workload(cfg)
    (pos, box), = w["volumes"]
    return pos, box


@pytest.mark.parametrize("ng", [16, 32])
def test_deposit_delta_k_and_power(clustered, ng):
    pos, box = clustered
    p = _pm(ng, box, 0.8, len(pos))
    x = torch.from_numpy(pos).cuda()
    p.deposit(x)
    counts = p.export("counts").cpu().numpy()
    ref = opm.cic_deposit(pos, box, ng)
    # corner weights are binary32 (relative error a few 2^-24 each)
    assert np.all(np.abs(counts - ref) <= 4e-7 * np.maximum(ref, 1.0))
    assert counts.sum() == pytest.approx(len(pos), rel=1e-6)
    dk = p.export("delta_k").cpu().numpy()
    dref = np.fft.fftn(ref / (len(pos) / ng ** 3) - 1.0)
    assert np.linalg.norm(dk - dref) <= FFT_TOL * np.linalg.norm(dref)
    k, pk, modes = (t.cpu().numpy() for t in p.power())
    k_o, p_o, m_o = opm.power_spectrum(pos, box, ng)
    np.testing.assert_array_equal(modes, m_o)
    np.testing.assert_allclose(k, k_o, rtol=1e-12)
    rel = np.abs(pk - p_o) / p_o
    print(f"ng {ng}: P(k) rel err max {rel.max():.2e}")
    assert rel.max() <= PK_TOL
    p.close()


@pytest.mark.parametrize("ng", [16, 32])
def test_pm_accelerations_match_oracle(clustered, ng):
    pos, box = clustered
    sigma = 0.8
    p = _pm(ng, box, sigma, len(pos))
    x = torch.from_numpy(pos).cuda()
    p.deposit(x)
    acc = p.force(x)
    torch.cuda.synchronize()
    a = acc.cpu().numpy()
    ref = opm.pm_accel(pos, box, ng, sigma)
    rel = rel_errors(a[:, :3].astype(np.float64), ref)
    print(f"ng {ng}: PM accel rel err median {np.median(rel):.2e} max {rel.max():.2e}")
    assert np.median(rel) <= 1e-5 and rel.max() <= 1e-4
    assert np.all(a[:, 3] == 0.0)
    # Newton's third law holds for the CIC deposit/interpolation pair
    assert np.all(np.abs(a[:, :3].astype(np.float64).sum(axis=0)) <= 1e-5 * np.abs(a[:, :3]).sum())
    grid = p.export("accel").cpu().numpy()[..., :3]
    gref = opm.pm_accel_grid(opm.cic_deposit(pos, box, ng), box, sigma)
    assert np.linalg.norm(grid - gref) <= 1e-5 * np.linalg.norm(gref)
    # accumulate onto existing accelerations (e.g. the short-range ones)
    base = torch.randn((len(pos), 4), dtype=torch.float32, device="cuda")
    both = p.force(x, base.clone(), accumulate=True)
    np.testing.assert_allclose(both.cpu().numpy()[:, :3], base.cpu().numpy()[:, :3] + a[:, :3], rtol=0,
                               atol=1e-5 * np.abs(a).max() + 1e-6)
    p.close()


def test_mesh_spacing_not_a_power_of_two():
    # box 20 on a 16^3 mesh: d = 1.25, so n / L is not a power of two and the
    # CIC kernels place particles with binary64 arithmetic; positions include
    # values outside [0, L) (folded) and exactly on cell walls
    L, ng, sigma = 20.0, 16, 0.8
    pos, _, _ = gen.nfw_clustered(6000, L, 33, m_lo=40.0, m_hi=900.0)
    pos = pos.copy()
    pos[:4] = [[0.0, 1.25, 2.5], [L - 1e-12, 10.0, 5.0], [-0.625, 3.0, 21.25], [1.25 * 7, 1.25 * 3, 1.25 * 15]]
    p = _pm(ng, L, sigma, len(pos))
    x = torch.from_numpy(pos).cuda()
    p.deposit(x)
    counts = p.export("counts").cpu().numpy()
    ref = opm.cic_deposit(pos, L, ng)
    assert np.all(np.abs(counts - ref) <= 4e-7 * np.maximum(ref, 1.0))
    k, pk, modes = (t.cpu().numpy() for t in p.power())
    k_o, p_o, m_o = opm.power_spectrum(pos, L, ng)
    np.testing.assert_array_equal(modes, m_o)
    assert np.max(np.abs(pk - p_o) / p_o) <= PK_TOL
    a = p.force(x).cpu().numpy()
    rel = rel_errors(a[:, :3].astype(np.float64), opm.pm_accel(pos, L, ng, sigma))
    assert np.median(rel) <= 1e-5 and rel.max() <= 1e-4
    p.close()


def test_lattice_on_grid_and_shot_noise():
    # a lattice on the grid points has delta = 0; uniform points have the
    # closed-form shot-noise level (checked against the oracle's value)
    L, ng = 16.0, 16
    lat = gen.lattice(16, L, offset=0.0)
    p = _pm(ng, L, 0.8, len(lat))
    p.deposit(torch.from_numpy(lat).cuda())
    _, pk, _ = p.power()
    assert float(pk.abs().max()) < 1e-10
    acc = p.force(torch.from_numpy(lat).cuda())
    assert float(acc.abs().max()) < 1e-4
    p.close()


def test_pm_state_and_argument_errors():
    from paper_1411_3396_b300 import SrError
    p = _pm(16, 16.0, 0.8, 100)
    x = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(SrError):
        p.power()                                         # nothing deposited yet
    p.deposit(x, transform=False)
    with pytest.raises(SrError):
        p.force(x)                                        # deposited, not transformed
    with pytest.raises(SrError):
        p.force(x)
    big = torch.zeros((101, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(SrError):
        p.deposit(big)                                    # above n_max
    p.close()


def test_full_clustered_256_power_and_sampled_forces():
    w = wc.make_workload(wc.CONFIGS["clustered256"])
    (pos, box), = w["volumes"]
    ng, sigma = 256, 0.8
    p = _pm(ng, box, sigma, len(pos))
    x = torch.from_numpy(pos).cuda()
    p.deposit(x)
    k, pk, modes = (t.cpu().numpy() for t in p.power())
    acc = p.force(x).cpu().numpy()
    p.close()
    k_o, p_o, m_o = opm.power_spectrum(pos, box, ng)
    np.testing.assert_array_equal(modes, m_o)
    rel = np.abs(pk - p_o) / p_o
    print(f"256^3: P(k) rel err max {rel.max():.2e}")
    assert rel.max() <= PK_TOL
    idx = np.random.default_rng(0).choice(len(pos), 20000, replace=False)
    grid = opm.pm_accel_grid(opm.cic_deposit(pos, box, ng), box, sigma)
    ref = opm.cic_interpolate(grid, pos[idx], box)
    r = rel_errors(acc[idx, :3].astype(np.float64), ref)
    print(f"256^3: sampled PM accel rel err median {np.median(r):.2e} max {r.max():.2e}")
    assert np.median(r) <= 1e-5 and r.max() <= 1e-4


def _binned_vs_plain(pos, box, ng, chunk=32, n_cells=0, sub_bits=0):
    from paper_1411_3396_b300 import Plan
    x = torch.from_numpy(pos).cuda()
    plan = Plan(box, 3.0, 0.1, 0.8, len(pos), n_cells=n_cells, chunk_size=chunk, sub_bits=sub_bits)
    plan.bin(x)
    p = _pm(ng, box, 0.8, len(pos))
    p.deposit(x, transform=False)
    ref = p.export("counts").cpu().numpy()
    p.deposit(x, transform=False, plan=plan)
    got = p.export("counts").cpu().numpy()
    p.close()
    plan.close()
    return got, ref


@pytest.mark.parametrize("ng,chunk", [(16, 32), (32, 32), (32, 64), (64, 32)])
def test_binned_deposit_same_bits(clustered, ng, chunk):
    # the deposit over the short-range binning's cell order (on-chip tiles
    # per brick of cells) adds the same integers as the caller-order one
    pos, box = clustered
    got, ref = _binned_vs_plain(pos, box, ng, chunk)
    assert got.tobytes() == ref.tobytes()
    # unwrapped positions in [-L, 2L) and a mesh that is not a multiple of
    # the cells (box 20: 5 cells of side 4 against a 16^3 mesh of spacing
    # 1.25): tiles with margins, corners past them go straight to the grid
    L = 20.0
    q, _, _ = gen.nfw_clustered(5000, L, 41, m_lo=40.0, m_hi=900.0)
    q = q + np.random.default_rng(3).choice([-1.0, 0.0, 1.0], size=q.shape) * L
    q = np.where(q < -L, q + L, np.where(q >= 2 * L, q - L, q))
    got, ref = _binned_vs_plain(q, L, 16, chunk)
    assert got.tobytes() == ref.tobytes()
    got, ref = _binned_vs_plain(q, L, 16, chunk, n_cells=6)       # cell side 3.33: tiles of 2.67 mesh cells
    assert got.tobytes() == ref.tobytes()


def test_binned_deposit_full_clustered_256():
    w = wc.make_workload(wc.CONFIGS["clustered256"])
    (pos, box), = w["volumes"]
    got, ref = _binned_vs_plain(pos, box, 256)
    assert got.tobytes() == ref.tobytes()
