"""Slab decomposition of one periodic volume over ranks with an overload
(ghost) shell, after the paper's overloading scheme (Sec. 2, Sec. 2.1):
every rank owns the particles of a slab of whole cells along x and, before
the force, receives from the other ranks the particles of the cells next to
its slab (periodic in x).  Each rank bins its owned and ghost particles in a
plan of the whole box (same side, same cells, so the cells away from its
slab are simply empty) and keeps the forces of its owned particles only;
ghosts are read-only, so no reduction follows.

Cells are at least r_c wide and the pair kernel reads only the 27 cells
around a particle's own, so one ghost cell on each side of the slab holds
every neighbour within r_c.  Cell membership here follows the binning
kernel's definition exactly (fold into [0, L), t = x / h in binary64,
q = min(floor(t), M - 1), cell = q >> b), and every cell's particles are
kept in increasing global-id order; the binning sort is stable, so every
cell an owned particle reads holds the same particles in the same order as
in the undivided volume, and the owned particles' forces are bit-identical
to the single-volume result.  The ghosts are binned with an active mask
(Plan.bin(pos, active=owned)): only chunks holding owned particles are work
items of the pair kernels, and only owned rows are written.

Index bookkeeping (cells, masks, selection, ordering) runs in PyTorch on the
tensors' device, and the exchange in torch.distributed (gloo or NCCL); this
is orchestration around the library's kernels, not part of the force
arithmetic.
"""
from __future__ import annotations

import torch


def slab_bounds(n_cells: int, world: int):
    """Cell-index ranges [c0, c1) along x of each rank (as even as possible)."""
    if world < 1 or world > n_cells:
        raise ValueError("need 1 <= world <= n_cells")
    base, extra = divmod(n_cells, world)
    out, c = [], 0
    for r in range(world):
        w = base + (1 if r < extra else 0)
        out.append((c, c + w))
        c += w
    return out


class Slabs:
    """x-slabs of whole cells of one periodic volume of side `box` with
    `n_cells` cells per axis, each split into 2^sub_bits fine cells of side
    h = box / (n_cells 2^sub_bits) (the binning's grid)."""

    def __init__(self, box: float, n_cells: int, sub_bits: int, world: int):
        self.box = float(box)
        self.n_cells = int(n_cells)
        self.sub_bits = int(sub_bits)
        self.M = self.n_cells << self.sub_bits
        self.h = self.box / self.M
        self.world = int(world)
        self.bounds = slab_bounds(self.n_cells, self.world)

    @classmethod
    def of_plan(cls, plan, world: int, volume: int = 0):
        """Slabs on the cell grid of a plan's volume."""
        v = plan.volume(volume)
        return cls(v["box"], v["n_cells"], plan.info()["sub_bits"], world)

    def cell_x(self, pos: torch.Tensor) -> torch.Tensor:
        """Cell index along x of every particle (the binning's definition)."""
        x = pos[:, 0]
        x = torch.where(x < 0, x + self.box, x)
        x = torch.where(x >= self.box, x - self.box, x)
        q = torch.clamp(torch.floor(x / self.h), max=self.M - 1).to(torch.int64)
        return q >> self.sub_bits

    def owner(self, pos: torch.Tensor) -> torch.Tensor:
        """Rank whose slab holds each particle."""
        starts = torch.tensor([c0 for c0, _ in self.bounds[1:]], dtype=torch.int64, device=pos.device)
        return torch.bucketize(self.cell_x(pos), starts, right=True)

    def owned(self, pos: torch.Tensor, rank: int) -> torch.Tensor:
        """Mask of the particles in rank's slab."""
        c0, c1 = self.bounds[rank]
        cx = self.cell_x(pos)
        return (cx >= c0) & (cx < c1)

    def ghost(self, pos: torch.Tensor, rank: int) -> torch.Tensor:
        """Mask of the particles outside rank's slab in the cells next to
        it (c0 - 1 and c1, periodically)."""
        c0, c1 = self.bounds[rank]
        cx = self.cell_x(pos)
        inside = (cx >= c0) & (cx < c1)
        near = (cx == (c0 - 1) % self.n_cells) | (cx == c1 % self.n_cells)
        return near & ~inside

    def local_set(self, pos: torch.Tensor, ids: torch.Tensor, rank: int):
        """Owned and ghost particles of `rank` drawn from one array holding
        every particle: (positions, global ids, owned flags) in increasing
        global-id order."""
        own = self.owned(pos, rank)
        sel = torch.nonzero(own | self.ghost(pos, rank)).squeeze(1)
        sel = sel[torch.argsort(ids[sel])]
        return pos[sel].contiguous(), ids[sel].contiguous(), own[sel].contiguous()

    def exchange(self, pos: torch.Tensor, ids: torch.Tensor, group=None):
        """Overload exchange between ranks that each hold exactly their owned
        particles (pos, ids), in increasing global-id order (as migrate
        returns them): returns this rank's owned + ghost particles
        (positions, global ids, owned flags): its own particles first, as
        given, then the ghosts of each other rank in rank order, each in that
        rank's order.  A cell belongs wholly to one slab, so every cell's
        particles arrive from one rank in increasing id order, which is all
        the stable binning needs for the owned forces to equal the undivided
        volume's bit for bit; no sort.  One all-gather of the send counts
        (read on the host once), then point-to-point sends to every rank of
        the particles in the cells next to its slab."""
        import torch.distributed as dist
        world = dist.get_world_size(group)
        rank = dist.get_rank(group)
        if world != self.world:
            raise ValueError("slab count differs from the process group size")
        dev = pos.device
        # every peer's ghost rows in one selection (rows grouped by peer, in
        # increasing row order within each)
        none = torch.zeros(len(pos), dtype=torch.bool, device=dev)
        masks = torch.stack([none if q == rank else self.ghost(pos, q) for q in range(world)])
        peer, rows = masks.nonzero(as_tuple=True)
        counts = torch.bincount(peer, minlength=world)
        table = [torch.zeros_like(counts) for _ in range(world)]
        dist.all_gather(table, counts, group=group)
        table = torch.stack(table).tolist()                   # one device-to-host read: all counts
        sends = list(torch.split(rows, table[rank]))
        incoming = [table[q][rank] for q in range(world)]
        # one batch of point-to-point operations (grouped, so that NCCL does
        # not block on the first receive while its peer waits on its own)
        recv_pos, recv_ids, ops = [], [], []
        for q in range(world):
            if q == rank:
                continue
            nq = int(incoming[q])
            rp = torch.empty((nq, 3), dtype=pos.dtype, device=dev)
            ri = torch.empty(nq, dtype=ids.dtype, device=dev)
            recv_pos.append(rp)
            recv_ids.append(ri)
            if nq:
                ops.append(dist.P2POp(dist.irecv, rp, q, group))
                ops.append(dist.P2POp(dist.irecv, ri, q, group))
            if len(sends[q]):
                ops.append(dist.P2POp(dist.isend, pos[sends[q]].contiguous(), q, group))
                ops.append(dist.P2POp(dist.isend, ids[sends[q]].contiguous(), q, group))
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()
        own = torch.zeros(len(pos) + sum(len(r) for r in recv_ids), dtype=torch.bool, device=dev)
        own[:len(pos)] = True
        return torch.cat([pos] + recv_pos).contiguous(), torch.cat([ids] + recv_ids).contiguous(), own

    def migrate(self, pos: torch.Tensor, ids: torch.Tensor, *fields: torch.Tensor, group=None):
        """Hand every particle to the rank whose slab holds it, after a drift
        has moved particles across slab faces (any number of slabs, positions
        within one period of [0, box)).  `fields` are per-particle arrays
        (velocities, accelerations, ...) that travel with the positions.
        Returns (pos, ids, *fields) of the particles this rank owns, in
        increasing global-id order: after a drift a cell can hold kept and
        received particles together, and the stable binning needs each
        cell's particles in id order, so the merged set is sorted by id here
        (once per migration; the exchange then needs no sort).  One
        all-gather of the send counts (read on the host once), then one batch
        of point-to-point sends to the ranks that gain particles."""
        import torch.distributed as dist
        world = dist.get_world_size(group)
        rank = dist.get_rank(group)
        if world != self.world:
            raise ValueError("slab count differs from the process group size")
        if any(len(f) != len(pos) for f in fields) or len(ids) != len(pos):
            raise ValueError("ids and fields need one row per particle")
        dev = pos.device
        dest = self.owner(pos)
        arrays = (pos, ids) + fields
        rows = torch.argsort(dest, stable=True)                # rows grouped by new owner
        counts = torch.bincount(dest, minlength=world)
        table = [torch.zeros_like(counts) for _ in range(world)]
        dist.all_gather(table, counts, group=group)
        table = torch.stack(table).tolist()                   # one device-to-host read: all counts
        sends = list(torch.split(rows, table[rank]))
        incoming = [0 if q == rank else table[q][rank] for q in range(world)]
        kept = [a[sends[rank]] for a in arrays]
        recv, ops = [], []
        for q in range(world):
            if q == rank:
                continue
            nq = int(incoming[q])
            bufs = [torch.empty((nq,) + tuple(a.shape[1:]), dtype=a.dtype, device=dev) for a in arrays]
            recv.append(bufs)
            if nq:
                ops += [dist.P2POp(dist.irecv, b, q, group) for b in bufs]
            if len(sends[q]):
                ops += [dist.P2POp(dist.isend, a[sends[q]].contiguous(), q, group) for a in arrays]
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()
        out = [torch.cat([kept[k]] + [b[k] for b in recv]) for k in range(len(arrays))]
        order = torch.argsort(out[1])
        return tuple(a[order].contiguous() for a in out)
