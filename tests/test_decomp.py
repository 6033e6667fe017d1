"""Host logic of the overload slab decomposition (Sec. 2, Sec. 2.1) on CPU:
slab bounds, cell membership against the oracle's binning, owned sets that
partition the volume, ghost shells of exactly the neighbouring cells, and the
point-to-point exchange between gloo ranks (world sizes 2 and 3), which must
hand every rank the same owned + ghost set as a selection from the whole
array, and the migration of drifted particles (with the fields that travel
with them) to their new owners over several steps."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest
import torch

from oracle import binning as obin
from workloads import generators as gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _clustered(n=6000, box=24.0, seed=5):
    pos, _, _ = gen.nfw_clustered(n, box, seed, m_lo=40.0, m_hi=600.0)
    pos[:7, 0] = [0.0, box / 8 * 3, -1e-12, box - 1e-12, 3.0 * box / 8, 1.5 * box, -0.5 * box]
    return pos


def test_slab_bounds_partition():
    from paper_1411_3396_b300.decomp import slab_bounds
    for n_c in (1, 3, 7, 64):
        for world in range(1, min(n_c, 9) + 1):
            b = slab_bounds(n_c, world)
            assert b[0][0] == 0 and b[-1][1] == n_c
            assert all(b[r][1] == b[r + 1][0] for r in range(world - 1))
            w = [c1 - c0 for c0, c1 in b]
            assert min(w) >= 1 and max(w) - min(w) <= 1
    with pytest.raises(ValueError):
        slab_bounds(4, 5)
    with pytest.raises(ValueError):
        slab_bounds(4, 0)


@pytest.mark.parametrize("n_c,b", [(8, 0), (6, 2), (5, 3)])
def test_cells_follow_the_binning(n_c, b):
    from paper_1411_3396_b300.decomp import Slabs
    box = 24.0
    pos = _clustered(box=box)
    s = Slabs(box, n_c, b, 3)
    _, q = obin.fine_coords(pos, box, n_c, b)
    np.testing.assert_array_equal(s.cell_x(torch.from_numpy(pos)).numpy(), q[:, 0] >> b)


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_owned_partition_and_ghost_shell(world):
    from paper_1411_3396_b300.decomp import Slabs
    box, n_c = 24.0, 6
    pos = _clustered(box=box)
    x = torch.from_numpy(pos)
    s = Slabs(box, n_c, 1, world)
    _, q = obin.fine_coords(pos, box, n_c, 1)
    cx = q[:, 0] >> 1
    owners = np.zeros(len(pos), dtype=np.int64)
    for r in range(world):
        own = s.owned(x, r).numpy()
        owners += own
        c0, c1 = s.bounds[r]
        ghost = s.ghost(x, r).numpy()
        assert not np.any(own & ghost)
        want = np.isin(cx, [(c0 - 1) % n_c, c1 % n_c]) & ~((cx >= c0) & (cx < c1))
        np.testing.assert_array_equal(ghost, want)
        p, ids, flag = s.local_set(x, torch.arange(len(pos)), r)
        assert torch.all(ids[1:] > ids[:-1])
        np.testing.assert_array_equal(flag.numpy(), own[ids.numpy()])
        np.testing.assert_array_equal(p.numpy(), pos[ids.numpy()])
    np.testing.assert_array_equal(owners, np.ones(len(pos), dtype=np.int64))


def test_owner_matches_owned_masks():
    from paper_1411_3396_b300.decomp import Slabs
    box = 24.0
    x = torch.from_numpy(_clustered(box=box))
    for n_c, world in [(6, 1), (6, 4), (7, 3), (5, 5)]:
        s = Slabs(box, n_c, 2, world)
        own = s.owner(x)
        for r in range(world):
            assert torch.equal(own == r, s.owned(x, r))


def _matches_local_set(got, want, s, box, own_in):
    """The exchange's result holds the selection's particles (the same rows
    once sorted by id), its own particles first as given, and every cell's
    particles in increasing id order (what the stable binning needs)."""
    pos, ids, own = got
    order = torch.argsort(ids)
    ok = all(torch.equal(a[order], b) for a, b in zip(got, want))
    ok &= torch.equal(pos[:len(own_in[0])], own_in[0]) and torch.equal(ids[:len(own_in[1])], own_in[1])
    ok &= bool(own[:len(own_in[1])].all()) and not bool(own[len(own_in[1]):].any())
    _, q = obin.fine_coords(pos.numpy(), box, s.n_cells, s.sub_bits)
    c = q >> s.sub_bits
    cell = (c[:, 2] * s.n_cells + c[:, 1]) * s.n_cells + c[:, 0]
    key = np.lexsort((np.arange(len(cell)), cell))         # rows of each cell, in the returned order
    same = cell[key][1:] == cell[key][:-1]
    idn = ids.numpy()[key]
    ok &= bool(np.all(idn[1:][same] > idn[:-1][same]))
    return bool(ok)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    from paper_1411_3396_b300.decomp import Slabs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        box = 24.0
        pos = torch.from_numpy(_clustered(box=box))
        ids = torch.arange(len(pos), dtype=torch.int64)
        s = Slabs(box, 6, 0, world)
        mine = s.owned(pos, rank)
        # every rank starts with its owned particles only, in id order
        p0, i0 = pos[mine], ids[mine]
        got = s.exchange(p0, i0)
        want = s.local_set(pos, ids, rank)
        ok = _matches_local_set(got, want, s, box, (p0, i0))
        q.put((rank, ok, int(got[2].sum()), len(got[1])))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, ok, _, _ in res)
    assert sum(n_own for _, _, n_own, _ in res) == 6000
    assert all(n_loc > n_own for _, _, n_own, n_loc in res)


def _migrate_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    from paper_1411_3396_b300.decomp import Slabs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        box, n_c = 24.0, 8
        pos = torch.from_numpy(_clustered(box=box))
        n = len(pos)
        ids = torch.arange(n, dtype=torch.int64)
        vel = torch.from_numpy(np.random.default_rng(9).normal(size=(n, 4)).astype(np.float32))
        lab = torch.from_numpy(np.random.default_rng(10).integers(-5, 1000, n).astype(np.int32))
        s = Slabs(box, n_c, 1, world)
        mine = s.owned(pos, rank)
        p, i, v, lb = pos[mine], ids[mine], vel[mine], lab[mine]
        ok, moved = True, 0
        for step in range(4):
            # the same displacement field on every rank (drawn for all ids),
            # up to 1.5 slab widths, so particles also skip a rank
            g = np.random.default_rng(100 + step).uniform(-9.0, 9.0, size=(n, 3))
            disp = torch.from_numpy(g)
            p = torch.remainder(p + disp[i], box)
            pos = torch.remainder(pos + disp, box)
            moved += int((s.owner(p) != rank).sum())
            p, i, v, lb = s.migrate(p, i, v, lb)          # a (n, 4) and a (n,) field travel along
            want = s.owned(pos, rank)
            ok &= torch.equal(i, ids[want]) and torch.equal(p, pos[want]) and torch.equal(v, vel[want])
            ok &= lb.dtype == torch.int32 and torch.equal(lb, lab[want])
            got = s.exchange(p, i)
            ok &= _matches_local_set(got, s.local_set(pos, ids, rank), s, box, (p, i))
        q.put((rank, bool(ok), len(i), moved))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_migrate_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_migrate_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, ok, _, _ in res), res
    assert sum(n for _, _, n, _ in res) == 6000
    assert all(m > 0 for _, _, _, m in res)


def _slab_step_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import bench
    from oracle import fit as ofit
    from oracle import force as oforce
    from paper_1411_3396_b300.decomp import Slabs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        box, rc, eps, dt = 24.0, 3.0, 0.1, 0.01
        pos = torch.from_numpy(_clustered(box=box))
        n = len(pos)
        s = Slabs(box, 6, 0, world)
        mine = s.owned(pos, rank)
        x_own, ids_own = pos[mine], torch.arange(n)[mine]
        n_own = len(x_own)
        vel = torch.zeros((n, 4), dtype=torch.float32)
        vel[:n_own, :3] = torch.from_numpy(np.random.default_rng(3).normal(size=(n, 3))[mine.numpy()]).float()
        v0 = vel[:n_own].clone()
        acc = torch.full((n, 4), float("nan"), dtype=torch.float32)
        c = ofit.fit_poly(rc, 0.8, eps)
        got = {}

        def force_kick(xl, own, a, v):
            # the FP64 oracle stands in for the kernels: each owned row gets
            # the force from every local particle (its slab and the ghosts)
            ref, _ = oforce.accel_kdtree(xl.numpy(), box, rc, eps, c)
            o = own.numpy()
            got["own"] = ref[o]
            a[own, :3] = torch.from_numpy(ref[o]).float()
            a[own, 3] = 0.0
            v[own, :3] += a[own, :3] * dt
            got["m"], got["n_own_flags"] = len(xl), int(o.sum())

        m = bench.slab_step(s, x_own, ids_own, acc, vel, force_kick)
        untouched = bool(torch.isnan(acc[n_own:]).all())
        kicked = bool(torch.equal(vel[:n_own, :3], v0[:, :3] + acc[:n_own, :3] * dt))
        q.put((rank, ids_own.numpy(), got["own"], m, got["m"], got["n_own_flags"] == n_own, untouched, kicked))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_bench_slab_step_gloo(world):
    # the bench's multi-GPU step (exchange, passive ghosts, owned rows
    # written and kicked), driven with gloo ranks on the CPU and the oracle
    # in place of the kernels: the ranks' owned forces assemble the
    # undivided volume's forces
    from oracle import fit as ofit
    from oracle import force as oforce
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_step_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pos = _clustered(box=24.0)
    ref, _ = oforce.accel_kdtree(pos, 24.0, 3.0, 0.1, ofit.fit_poly(3.0, 0.8, 0.1))
    full = np.full_like(ref, np.nan)
    for rank, ids, own_acc, m, m_seen, flags_ok, untouched, kicked in res:
        assert m == m_seen and flags_ok and untouched and kicked
        assert m > len(ids)                                  # ghosts arrived
        full[ids] = own_acc
    scale = np.abs(ref).max()
    np.testing.assert_allclose(full, ref, rtol=0, atol=1e-12 * scale)
