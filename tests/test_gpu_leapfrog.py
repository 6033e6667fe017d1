"""Fused force-kick epilogue and the native KDK leapfrog stepper, against
the unfused calls (bit for bit) and the FP64 oracle's leapfrog."""
import numpy as np
import pytest

from oracle import fit as ofit
from oracle import force as oforce
from oracle import integrate as oint
from workloads import configs as wc

from helpers import make_plan, rel_errors, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("chunk,variant", [(32, None), (64, None), (32, 14), (32, 15), (32, 16)])
def test_force_kick_equals_force_then_kick(chunk, variant):
    from paper_1411_3396_b300 import kick
    w = wc.make_workload(wc.small_variant("clustered256"))
    (pos, box), = w["volumes"]
    n = len(pos)
    v0 = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    v0[:, :3] = torch.from_numpy(w["velocities"]).float()
    plan = make_plan(w["volumes"], w["params"], chunk_size=chunk)
    plan.bin(torch.from_numpy(pos).cuda())
    if variant is not None:                   # the grouped kernel's epilogue
        plan.set_variant(variant)
    a1 = plan.force()
    v1 = v0.clone()
    kick(a1, v1, 0.01)
    a2 = torch.empty_like(a1)
    v2 = v0.clone()
    plan.force_kick(a2, v2, 0.01)
    assert to_np(a1).tobytes() == to_np(a2).tobytes()
    assert to_np(v1).tobytes() == to_np(v2).tobytes()


def test_leapfrog_matches_oracle():
    cfg = wc.small_variant("zeldovich128")
    w = wc.make_workload(cfg)
    (pos, box), = w["volumes"]
    prm = w["params"]
    n = len(pos)
    steps, dt = 10, 0.02
    v0 = 0.1 * w["velocities"]
    plan = make_plan(w["volumes"], prm)
    x = torch.from_numpy(pos).cuda()
    v = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    v[:, :3] = torch.from_numpy(v0).float()
    acc = torch.empty_like(v)
    plan.bin(x)
    plan.force(acc)
    plan.leapfrog(x, v, acc, dt, steps)
    plan.status()
    c = ofit.fit_poly(prm["rc"], prm["sigma"], prm["eps"])
    xr, vr, ar = oint.leapfrog(pos, v0, box, prm["rc"], prm["eps"], c, dt, steps)
    assert np.max(np.abs(oforce.min_image(to_np(x) - xr, box))) < 1e-5
    rv = rel_errors(to_np(v)[:, :3], vr)
    ra = rel_errors(to_np(acc)[:, :3], ar)
    assert np.median(rv) <= 1e-5 and rv.max() <= 1e-3, (np.median(rv), rv.max())
    assert np.median(ra) <= 1e-5 and ra.max() <= 1e-3, (np.median(ra), ra.max())
    # momentum is conserved by the pairwise-antisymmetric force
    inv = to_np(plan.invariants(v, acc))
    assert np.all(np.abs(inv[0:3] - v0.sum(axis=0)) < 1e-4 * np.abs(v0).sum())


def test_leapfrog_on_a_batch_plan():
    # independent volumes of different sides in one plan: each volume's
    # trajectory (drift folded into its own box) against the oracle's
    w = wc.make_workload(wc.small_variant("batch64"))
    vols, prm = w["volumes"], w["params"]
    pos = np.concatenate([p for p, _ in vols])
    n = len(pos)
    steps, dt = 5, 0.02
    v0 = 0.1 * w["velocities"]
    plan = make_plan(vols, prm)
    x = torch.from_numpy(pos).cuda()
    v = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    v[:, :3] = torch.from_numpy(v0).float()
    acc = torch.empty_like(v)
    plan.bin(x)
    plan.force(acc)
    plan.leapfrog(x, v, acc, dt, steps)
    plan.status()
    c = ofit.fit_poly(prm["rc"], prm["sigma"], prm["eps"])
    xg, vg = to_np(x), to_np(v)[:, :3]
    off = 0
    for p, box in vols:
        m = len(p)
        xr, vr, _ = oint.leapfrog(p, v0[off:off + m], box, prm["rc"], prm["eps"], c, dt, steps)
        assert np.all((xg[off:off + m] >= 0) & (xg[off:off + m] < box))
        assert np.max(np.abs(oforce.min_image(xg[off:off + m] - xr, box))) < 1e-5
        rv = rel_errors(vg[off:off + m], vr)
        assert np.median(rv) <= 1e-5 and rv.max() <= 1e-3, (np.median(rv), rv.max())
        off += m


def test_leapfrog_zero_steps_is_identity():
    w = wc.make_workload(wc.small_variant("uniform4k"))
    (pos, box), = w["volumes"]
    plan = make_plan(w["volumes"], w["params"])
    x = torch.from_numpy(pos).cuda()
    v = torch.ones((len(pos), 4), dtype=torch.float32, device="cuda")
    a = torch.zeros_like(v)
    x0, v0 = x.clone(), v.clone()
    plan.leapfrog(x, v, a, 0.01, 0)
    assert torch.equal(x, x0) and torch.equal(v, v0)
