"""Full-size parity of the short-range step in the launch configuration the
benchmark times: the library's default geometry (32-particle chunks, 6
sub-cell bits), the autotuned pair-kernel variant and the kick fused into
the force kernel's epilogue.  Sampled rows (random ones and the most
strongly accelerated ones) are compared with the FP64 oracle row by row;
per-particle pair counts of sampled rows are compared bit for bit with the
oracle's binary32 predicate; the fused kick must equal sr_kick applied to
the returned accelerations."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle import binning as obin
from oracle import fit as ofit
from oracle import force as oforce
from workloads import configs as wc

from helpers import MAX_TOL, MEDIAN_TOL, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("name", ["clustered256", "zeldovich128"])
def test_full_size_step_sampled(name):
    from paper_1411_3396_b300 import Plan, kick
    w = wc.make_workload(wc.CONFIGS[name])
    (pos, box), = w["volumes"]
    prm = w["params"]
    n = len(pos)
    plan = Plan(box, prm["rc"], prm["eps"], prm["sigma"], n)
    x = torch.from_numpy(pos).cuda()
    plan.bin(x)
    plan.autotune(reps=1)
    info = plan.info()
    assert info["chunk_size"] == 32 and info["sub_bits"] == 6

    vel0 = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    vel0[:, :3] = torch.from_numpy(w["velocities"]).float().cuda()
    vel = vel0.clone()
    acc = torch.empty_like(vel)
    plan.force_kick(acc, vel, prm["dt"])
    vref = vel0.clone()
    kick(acc, vref, prm["dt"])
    torch.cuda.synchronize()
    assert torch.equal(vel, vref)

    a_gpu = to_np(acc)[:, :3].astype(np.float64)
    rng = np.random.default_rng(17)
    rand = rng.choice(n, 1500, replace=False)
    strong = np.argsort(-np.linalg.norm(a_gpu, axis=1))[:500]
    rows = np.unique(np.concatenate([rand, strong]))
    c = ofit.fit_poly(prm["rc"], prm["sigma"], prm["eps"])
    tree = cKDTree(oforce._wrap_for_tree(pos, box), boxsize=box)
    a_ref, _ = oforce.accel_rows(pos, box, prm["rc"], prm["eps"], c, rows, tree=tree)
    mag = np.linalg.norm(a_ref, axis=1)
    rms_random = np.sqrt(np.mean(np.linalg.norm(a_ref[np.isin(rows, rand)], axis=1) ** 2))
    rel = np.linalg.norm(a_gpu[rows] - a_ref, axis=1) / np.maximum(mag, 1e-3 * rms_random)
    med, mx = float(np.median(rel)), float(rel.max())
    assert med <= MEDIAN_TOL and mx <= MAX_TOL, f"{name}: median {med:.3g} max {mx:.3g}"

    # per-particle pair counts (counting variant) against the binary32 predicate
    _, pairs, pp = plan.force(torch.empty_like(acc), count=True, per_particle=True)
    pp = to_np(pp).astype(np.int64)
    assert int(pairs.item()) == int(pp.sum())
    binned = obin.bin_particles([(pos, box)], [plan.volume(0)["n_cells"]], info["sub_bits"], info["chunk_size"])
    crow = np.unique(np.concatenate([rng.choice(n, 800, replace=False), np.argsort(-pp)[:200]]))
    ref_counts = oforce.pair_counts_fp32(binned, [(pos, box)], prm["rc"], prm["eps"], rows=crow)
    np.testing.assert_array_equal(pp[crow], ref_counts)
    print(f"{name}: variant {info['variant']}, {n} particles, {int(pairs.item())} pairs; "
          f"{len(rows)} rows median {med:.2e} max {mx:.2e}; {len(crow)} counts exact")
    plan.close()
