"""Overload slab decomposition (Sec. 2, Sec. 2.1) on the GPU: every rank's
owned + ghost set is binned in a plan of the whole box and forced; the
owned particles' accelerations and pair counts must be bit-identical to the
undivided volume's, and within the force tolerance of the oracle; a
kick-drift-kick run in slabs (drift of the owned particles, migration to the
new owners, ghost exchange, binning, fused force and kick) must end in the
same state, bit for bit, as the native leapfrog on the undivided volume.  The
ranks' sub-problems run one after another on one device (independent
launches, no rank waits on another), with the migration and exchange taken
as selections from the whole arrays (the selection the point-to-point
exchange reproduces, checked with gloo ranks on the CPU)."""
import numpy as np
import pytest

from workloads import configs as wc

from helpers import assert_force_close, oracle_force, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _force(pos, box, prm, n_cells, chunk, active=None, variant=None):
    from paper_1411_3396_b300 import Plan
    plan = Plan(box, prm["rc"], prm["eps"], prm["sigma"], len(pos), n_cells=n_cells, chunk_size=chunk)
    plan.bin(pos, active=active)
    if variant is not None:
        plan.set_variant(variant)
    # sentinels: rows the kernels must not write (passive particles) keep them
    acc = torch.full((len(pos), 4), float("nan"), dtype=torch.float32, device="cuda")
    pp = torch.full((len(pos),), -7, dtype=torch.int32, device="cuda")
    acc, pairs, pp = plan.force(acc, count=True, per_particle=pp)
    torch.cuda.synchronize()
    return plan, acc, int(pairs.item()), pp


def _check_ranks(pos_np, box, prm, world, chunk, active=False, variant=None):
    """Every rank's owned + ghost set forced in a plan of the whole box; with
    active, the ghosts are binned as passive (sr_bin_active): then only the
    chunks holding owned particles are work items, so the ranks' candidate
    evaluations add up to the whole volume's, and ghost rows stay unwritten."""
    from paper_1411_3396_b300.decomp import Slabs
    pos = torch.from_numpy(pos_np).cuda()
    plan, acc_full, pairs_full, pp_full = _force(pos, box, prm, 0, chunk, variant=variant)
    ctr_full = plan.export("counters").cpu().numpy()
    slabs = Slabs.of_plan(plan, world)
    n_c = plan.volume(0)["n_cells"]
    n_chunks = plan.info()["n_chunks"]
    assert slabs.h == plan.volume(0)["h"]
    plan.close()
    ids_all = torch.arange(len(pos), device="cuda")
    seen = torch.zeros(len(pos), dtype=torch.int32, device="cuda")
    pairs_owned = pairs_sum = evals = items = 0
    for r in range(world):
        p, ids, own = slabs.local_set(pos, ids_all, r)
        pl, acc, pairs, pp = _force(p, box, prm, n_c, chunk, active=own if active else None, variant=variant)
        ctr = pl.export("counters").cpu().numpy()
        pl.close()
        mine = ids[own]
        assert torch.equal(acc[own], acc_full[mine]), f"rank {r}: forces differ from the whole volume"
        assert torch.equal(pp[own], pp_full[mine])
        seen[mine] += 1
        pairs_owned += int(pp[own].sum().item())
        pairs_sum += pairs
        evals += int(ctr[3])
        items += int(ctr[5])
        if active:
            assert torch.all(torch.isnan(acc[~own])), f"rank {r}: a passive row was written"
            assert torch.all(pp[~own] == -7)
    assert torch.all(seen == 1)
    assert pairs_owned == pairs_full
    if active:
        assert pairs_sum == pairs_full                 # the pair total counts owned rows only
        assert evals == int(ctr_full[3])               # no evaluation spent on passive chunks
        assert items == n_chunks == int(ctr_full[5])
    else:
        assert evals > int(ctr_full[3])                # ghost chunks forced and thrown away
    return to_np(acc_full)


@pytest.mark.parametrize("variant", [None, 14, 15])
@pytest.mark.parametrize("world", [2, 3])
def test_slabs_with_passive_ghosts(world, variant):
    w = wc.make_workload(wc.small_variant("clustered256"))
    (pos, box), = w["volumes"]
    _check_ranks(pos, box, w["params"], world, 32, active=True, variant=variant)
    w = wc.make_workload(wc.small_variant("zeldovich128"))
    (pos, box), = w["volumes"]
    _check_ranks(pos, box, w["params"], world, 32, active=True, variant=variant)


@pytest.mark.parametrize("world", [2, 3, 4])
@pytest.mark.parametrize("chunk", [32, 64])
def test_clustered_slabs_bit_identical(world, chunk):
    w = wc.make_workload(wc.small_variant("clustered256"))
    (pos, box), = w["volumes"]
    acc = _check_ranks(pos, box, w["params"], world, chunk)
    a_ref, _ = oracle_force(w["volumes"], w["params"])
    assert_force_close(acc, a_ref, f"slabs {world}")


def test_zeldovich_slabs_with_positions_outside_the_box():
    # unwrapped positions in [-L, 2L): slab membership follows the same fold
    w = wc.make_workload(wc.small_variant("zeldovich128"))
    (pos, box), = w["volumes"]
    pos = pos.copy()
    rng = np.random.default_rng(11)
    shift = rng.choice([-1.0, 0.0, 1.0], size=pos.shape) * box
    pos = pos + shift
    pos = np.where(pos < -box, pos + box, pos)
    pos = np.where(pos >= 2 * box, pos - box, pos)
    _check_ranks(pos, box, w["params"], 3, 32)


def test_full_clustered_256_four_slabs():
    w = wc.make_workload(wc.CONFIGS["clustered256"])
    (pos, box), = w["volumes"]
    _check_ranks(pos, box, w["params"], 4, 32)


@pytest.mark.parametrize("world", [2, 3])
def test_slab_leapfrog_bit_identical(world):
    from paper_1411_3396_b300 import Plan, kick
    from paper_1411_3396_b300.decomp import Slabs
    w = wc.make_workload(wc.small_variant("zeldovich128"))
    (pos, box), = w["volumes"]
    prm = w["params"]
    n = len(pos)
    steps, dt = 4, 0.02
    v_init = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    # velocities large enough that particles cross slab faces every step
    v_init[:, :3] = torch.from_numpy(4.0 * w["velocities"]).float()
    whole = Plan(box, prm["rc"], prm["eps"], prm["sigma"], n, chunk_size=32)
    x = torch.from_numpy(pos).cuda()
    whole.bin(x)
    a = whole.force()
    xs, vs, acc = x.clone(), v_init.clone(), a.clone()
    v = v_init.clone()
    whole.leapfrog(x, v, a, dt, steps)
    whole.status()
    slabs = Slabs.of_plan(whole, world)
    n_c = whole.volume(0)["n_cells"]
    whole.close()
    plans = [Plan(box, prm["rc"], prm["eps"], prm["sigma"], n, n_cells=n_c, chunk_size=32)
             for _ in range(world)]
    ids = torch.arange(n, device="cuda")
    kick(acc, vs, 0.5 * dt)                          # opening half kick
    moved = 0
    for k in range(steps):
        owner = slabs.owner(xs)
        for r in range(world):                       # drift of the owned particles
            mine = ids[owner == r]
            xr = xs[mine].contiguous()
            plans[r].drift(xr, vs[mine].contiguous(), dt)
            xs[mine] = xr
        moved += int((slabs.owner(xs) != owner).sum())
        for r in range(world):
            # migration (new owners) and ghost exchange, then the rank's force
            p, loc, own = slabs.local_set(xs, ids, r)
            vl = vs[loc].contiguous()
            al = torch.empty_like(vl)
            plans[r].bin(p)
            plans[r].force_kick(al, vl, dt if k + 1 < steps else 0.5 * dt)
            plans[r].status()
            vs[loc[own]] = vl[own]
            acc[loc[own]] = al[own]
    for pl in plans:
        pl.close()
    assert torch.equal(xs, x), "positions differ from the undivided leapfrog"
    assert torch.equal(vs, v), "velocities differ from the undivided leapfrog"
    assert torch.equal(acc, a), "accelerations differ from the undivided leapfrog"
    assert moved > 0
