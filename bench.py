#!/usr/bin/env python
"""Benchmark of the short-range particle-particle step on B300.

Metric: short-range pair interactions per second (binary32), i.e. ordered
in-range pairs (i, j), i != j, counted bit-exactly by the library's
binary32 predicate, divided by the time of one whole step.  A step is
sr_bin (binning + stable counting sort + chunking + cost/order) ->
sr_force_kick (persistent pair kernel with the kick v += a dt fused into
its epilogue) -> sr_invariants, through the C ABI, on inputs already
resident in HBM.

Default workload: the clustered 256^3 set (16,777,216 particles, half in
NFW halos of 100..200,000 particles, half uniform, box 256, r_c = 3,
eps = 0.05), seeded synthetic data.  Inputs exceed L2 (positions alone are
402 MB), so no explicit L2 flush is done between steps.

Also reported: the pair kernel against the binary32 ALU roofline
(28 flops per in-range pair), the plain one-launch-per-slab kernel on the
same input, an end-to-end step from pinned host buffers, SM clocks sampled
during the timed region, and the FP64 oracle timed on a bounded sample on
the host cores.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Multi-GPU (torchrun): every rank runs an independent replica of the
workload (no data-path collective); value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOPS_PER_PAIR = 28          # 3 sub, 3 fma (s'), 1 mul + 1 fma (r^3 - q), 5 fma Horner, 3 fma accumulate
FP32_LANES_PER_SM = 128
PROFILE_NOTE = os.path.join(ROOT, "profiles", "force_clustered256.md")
CENTERS_NOTE = os.path.join(ROOT, "profiles", "centers_clustered256.md")

_CPU_STATE = {}


# ---------------------------------------------------------------------------
# CPU oracle leg (fork pool created before any CUDA call)
# ---------------------------------------------------------------------------

def _cpu_rows(rows):
    from oracle import force as oforce
    st = _CPU_STATE
    t0 = time.perf_counter()
    _, cnt = oforce.accel_rows(st["pos"], st["box"], st["rc"], st["eps"], st["coef"], rows, tree=st["tree"])
    return int(cnt.sum()), time.perf_counter() - t0


def cpu_oracle_sample(pos, box, prm, n_rows, seed, cores, reps=1):
    """Time the FP64 oracle's per-row force on n_rows random particles
    (k-d tree built before timing).  Returns (pairs/s, pairs, seconds)."""
    from scipy.spatial import cKDTree

    from oracle import fit as ofit
    wrapped = np.mod(pos, box)
    wrapped[wrapped >= box] = 0.0
    _CPU_STATE.update(pos=wrapped, box=box, rc=prm["rc"], eps=prm["eps"],
                      coef=ofit.fit_poly(prm["rc"], prm["sigma"], prm["eps"]),
                      tree=cKDTree(wrapped, boxsize=box))
    rng = np.random.default_rng(seed)
    results = []
    ctx = mp.get_context("fork")
    with ctx.Pool(cores) as pool:
        for _ in range(reps):
            rows = rng.choice(len(pos), n_rows, replace=False)
            # one call per worker: each call of the oracle's row function
            # re-wraps the whole position array, a fixed cost per call
            parts = np.array_split(rows, cores)
            t0 = time.perf_counter()
            out = pool.map(_cpu_rows, parts)
            el = time.perf_counter() - t0
            results.append((sum(o[0] for o in out), el))
    pairs = sum(r[0] for r in results)
    secs = sum(r[1] for r in results)
    return pairs / secs, pairs, secs, [r[0] / r[1] for r in results]


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

# Metric names: each workload's own arm and its oracle reference arm print
# the same metric, so the two lines compare directly.
METRICS = {
    "force": "short-range pair interactions/sec (FP32) and % of B300 FP32 peak vs plain kernel",
    "centers256": "halo center finding: unordered member pair potentials/sec (FP32, most-bound particle)",
    "pm256": "long-range PM step (CIC deposit, FFT, P(k), filtered PM accelerations): particles/sec",
    "fof256": "friends-of-friends halo finding (b=0.168, >=40 particles) incl. binning: particles/sec",
    "step256": "whole force-split time step (binning, short-range pairs, PM with P(k), kick): particles/sec",
    "diff64": "short-range pair interactions/sec (FP32), forward + VJP of a differentiable trajectory",
}


def host_cpu_model():
    """Model name of the host CPU (the oracle's timing context), or None."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def emit(line):
    """Print the bench line; a CPU baseline also names the host CPU model."""
    if isinstance(line.get("cpu_baseline"), dict):
        line["cpu_baseline"].setdefault("cpu_model", host_cpu_model())
    print(json.dumps(line), flush=True)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def kernel_source_hash(names=("force.cu", "pairs.cuh", "sr_internal.h")):
    h = hashlib.sha1()
    for name in names:
        with open(os.path.join(ROOT, "paper_1411_3396_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


BIN_BYTES_PER_PARTICLE = 44    # 24 B of binary64 position read, 16 B slot offsets + 4 B slot index written
KICK_BYTES_PER_PARTICLE = 48   # acceleration and velocity rows read (16 + 16 B), velocity row written (16 B)


def time_hbm_kernels(plan, x, acc, vel, n, hbm_gbs, reps=5):
    """sr_bin and the separate sr_kick timed alone (CUDA events on the
    current stream, after the timed step; inputs larger than L2), against
    their algorithmic bytes and the measured HBM copy bandwidth."""
    import torch
    from paper_1411_3396_b300 import kick
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    plan.bin(x)
    kick(acc, vel, 0.0)
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(reps):
        plan.bin(x)
    ev[1].record()
    ev[2].record()
    for _ in range(reps):
        kick(acc, vel, 0.0)                    # dt = 0: velocities unchanged
    ev[3].record()
    torch.cuda.synchronize()
    out = {}
    for name, ms, bpp in (("sr_bin", ev[0].elapsed_time(ev[1]) / reps, BIN_BYTES_PER_PARTICLE),
                          ("sr_kick", ev[2].elapsed_time(ev[3]) / reps, KICK_BYTES_PER_PARTICLE)):
        gbs = n * bpp / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "bytes_per_particle": bpp, "GB/s": gbs, "frac_of_measured_hbm": gbs / hbm_gbs}
    out["note"] = ("sr_bin includes the counting sort by cell, the per-cell sorts and the gather of "
                   "positions into slots; the time step fuses the kick into the force kernel")
    return out


def recorded_traffic(note=PROFILE_NOTE, names=("force.cu", "pairs.cuh", "sr_internal.h")):
    """DRAM bytes per launch of a kernel from its committed ncu summary, or
    None if the summary is missing or was taken on a different kernel source."""
    if not os.path.exists(note):
        return None
    text = open(note).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s+source_hash:\s*([0-9a-f]+)", text)
    if not m or m.group(2) != kernel_source_hash(names):
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi sampling of SM clock, power and throttle reasons."""
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 10:
                    continue
                if self.uuid and self.uuid not in parts[1] and parts[1] not in self.uuid:
                    continue
                try:
                    rows.append(dict(sm=float(parts[2]), max=float(parts[3]),
                                     power=float(parts[4]) if parts[4] not in ("[N/A]", "N/A") else 0.0,
                                     hw=parts[6], hwt=parts[7], swt=parts[8], pcap=parts[9]))
                except ValueError:
                    continue
        os.unlink(self.file.name)
        if not rows:
            return None
        load = [r for r in rows if r["power"] > 250.0] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return dict(sm_mhz=float(np.median([r["sm"] for r in load])), sm_max_mhz=max(r["max"] for r in rows),
                    reasons=sorted(reasons), samples=len(load))


def shard_volumes(sizes, world, rank):
    """Indices of the volumes rank `rank` evaluates: longest-first greedy
    assignment of independent volumes to ranks by size (no data exchange)."""
    loads = [0] * world
    owner = {}
    for v in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda k: (loads[k], k))
        owner[v] = r
        loads[r] += sizes[v]
    return [v for v in range(len(sizes)) if owner[v] == rank]


def slab_step(slabs, x_own, ids_own, acc_local, vel_local, force_kick, group=None):
    """One step of the overload slab decomposition (Sec. 2, Sec. 2.1) on
    this rank: the ghost exchange (this rank's owned particles, in id
    order, first; then the particles of the neighbouring slabs' edge
    cells), then force_kick(x_local, owned, acc_rows, vel_rows) on the local
    set, which bins the ghosts as passive and writes and kicks the owned
    rows only.  The owned rows are the first len(x_own) rows of acc_local
    and vel_local.  Returns the local set's size."""
    xl, _, own = slabs.exchange(x_own, ids_own, group=group)
    m = len(xl)
    force_kick(xl, own, acc_local[:m], vel_local[:m])
    return m


def reduce_over_ranks(pairs, ms, world, device):
    """Whole-job pairs (sum over ranks) and step time (max over ranks)."""
    if world == 1:
        return pairs, ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(pairs)], dtype=torch.float64, device=device)
    m = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return int(t.item()), float(m.item())


def make_inputs(name, n_particles=0, world=1, rank=0):
    """Volumes this rank evaluates: a batch is sharded across ranks; a single
    volume is returned whole on every rank (each rank then keeps its slab,
    run_ours)."""
    from workloads import configs as wc
    cfg = wc.resized(name, n_particles) if n_particles else wc.CONFIGS[name]
    w = wc.make_workload(cfg)
    vols = w["volumes"]
    vel = w["velocities"]
    if len(vols) > 1 and world > 1:
        mine = shard_volumes([len(p) for p, _ in vols], world, rank)
        starts = np.cumsum([0] + [len(p) for p, _ in vols])
        vel = np.concatenate([vel[starts[v]:starts[v + 1]] for v in mine])
        vols = [vols[v] for v in mine]
    return cfg, vols, vel, w["params"]


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def cpu_diff_sample(n_req, reps, warmup=0):
    """The oracle's own differentiable trajectory on the diff64 workload
    resized to a bounded sample (16^3 particles, or n_req if fewer): FP64
    kick-drift substeps and the hand-written reverse sweep, each repetition
    timed; pairs counted as in the GPU arm (forward pairs twice).  Returns
    (pairs/s per timed repetition, n, substeps)."""
    from scipy.spatial import cKDTree

    from oracle import fit as ofit
    from oracle import integrate as oint
    from workloads import configs as wc
    from workloads import generators as gen
    cfg = wc.resized("diff64", min(n_req or 16 ** 3, 16 ** 3))
    box, n_side, steps, dt = cfg["box"], cfg["n_side"], cfg["steps"], cfg["dt"]
    x0, psi = gen.zeldovich(n_side, box, cfg.get("rms", 0.5), cfg["seed"])
    xt, _ = gen.zeldovich(n_side, box, cfg.get("rms", 0.5), cfg["seed"] + 1)
    v0 = 0.1 * psi
    c = ofit.fit_poly(cfg["rc"], cfg["sigma"], cfg["eps"])
    xs, _ = oint.trajectory(x0, v0, box, cfg["rc"], cfg["eps"], c, dt, steps)
    pairs = 0
    for x in xs[:-1]:
        pairs += 2 * len(cKDTree(x, boxsize=box).query_pairs(cfg["rc"], output_type="ndarray"))   # ordered
    rates = []
    for k in range(warmup + reps):
        t0 = time.perf_counter()
        oint.loss_and_grad(x0, v0, xt, box, cfg["rc"], cfg["eps"], c, dt, steps)
        el = time.perf_counter() - t0
        if k >= warmup:
            rates.append(2 * pairs / el)
    return rates, len(x0), steps


def diff_sample_note(n, steps):
    return (f"the diff64 workload resized to {n} particles: FP64 trajectory of {steps} substeps and its "
            "reverse sweep (k-d tree pair sums, NumPy, one thread)")


def run_reference_diff(args, rank, world):
    rates, n, steps = cpu_diff_sample(args.n_particles, args.steps, args.warmup)
    value = float(np.mean(rates))
    line = {
        "impl": "reference", "metric": METRICS["diff64"],
        "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "diff64", "n_particles": n, "substeps": steps},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                         "sample": diff_sample_note(n, steps)},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    emit(line)


def run_reference(args, rank, world):
    cfg, vols, vel, prm = make_inputs(args.workload, args.n_particles)
    if rank != 0:
        return
    pos, box = max(vols, key=lambda v: len(v[0]))
    cores = os.cpu_count() or 1
    total = args.warmup + args.steps
    rows = min(args.ref_rows, len(pos))
    rate, pairs, secs, per = cpu_oracle_sample(pos, box, prm, rows, 7, cores, reps=total)
    per = per[args.warmup:]
    value = float(np.mean(per))
    line = {
        "impl": "reference", "metric": METRICS["force"],
        "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n_particles": int(sum(len(p) for p, _ in vols)),
                   "volumes": len(vols), "r_c": prm["rc"], "eps": prm["eps"], "sigma": prm["sigma"]},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                         "sample": f"{rows} random rows per step of the largest volume "
                                   "(FP64 k-d tree row sums; tree build untimed)"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    emit(line)


def run_ours(args, rank, world, local_rank):
    cfg, vols, vel_np, prm = make_inputs(args.workload, args.n_particles, world, rank)
    pos = np.concatenate([p for p, _ in vols])
    box = vols[0][1]
    batch = len(vols) > 1 or cfg.get("kind") == "batch"
    n = len(pos)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        cores = os.cpu_count() or 1
        big_pos, big_box = max(vols, key=lambda v: len(v[0]))
        rows = min(args.cpu_rows, len(big_pos))
        rate, pairs, secs, _ = cpu_oracle_sample(big_pos, big_box, prm, rows, 11, cores)
        cpu = {"value": rate, "unit": "pairs/s", "cores": cores, "kind": "oracle",
               "sample": f"{rows} random particles of the same workload"
                         f"{' (largest volume)' if batch else ''}, {pairs} pairs in {secs:.1f} s "
                         "(FP64 k-d tree row sums, tree build untimed)"}

    import torch
    import torch.distributed as dist

    from paper_1411_3396_b300 import Plan, kick, launch_count

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    props = torch.cuda.get_device_properties(dev)
    x = torch.from_numpy(pos).to(dev)
    vel = torch.zeros((n, 4), dtype=torch.float32, device=dev)
    vel[:, :3] = torch.from_numpy(vel_np).to(dev).float()
    acc = torch.empty((n, 4), dtype=torch.float32, device=dev)
    inv = torch.empty(7, dtype=torch.float64, device=dev)
    if batch:
        plan = Plan.batch([b for _, b in vols], [len(p) for p, _ in vols], prm["rc"], prm["eps"], prm["sigma"],
                          sub_bits=args.sub_bits, chunk_size=args.chunk_size)
    elif args.tune_geometry and world == 1:
        plan, tune_geometry = Plan.tune(box, prm["rc"], prm["eps"], prm["sigma"], x, reps=1, sub_bits=args.sub_bits)
    else:
        plan = Plan(box, prm["rc"], prm["eps"], prm["sigma"], n, n_cells=args.n_cells, sub_bits=args.sub_bits,
                    chunk_size=args.chunk_size)
    if not (args.tune_geometry and world == 1 and not batch):
        tune_geometry = None
    dt = prm["dt"]
    slabbed = world > 1 and not batch
    graphed = not slabbed            # bin + force with the fused kick replayed as one captured CUDA graph
    graph_stream = torch.cuda.Stream() if graphed else None
    if slabbed:
        # overload slab decomposition of the one volume: every rank keeps the
        # particles of its slab of cells (in id order) and, each step,
        # receives the ghosts of the neighbouring slabs' edge cells, binned
        # as passive (forced only as neighbours)
        from paper_1411_3396_b300.decomp import Slabs
        slabs = Slabs.of_plan(plan, world)
        mine = slabs.owned(x, rank)
        x_own = x[mine].contiguous()
        ids_own = torch.arange(n, device=dev)[mine].contiguous()
        n_own = len(x_own)
        vel_loc = torch.zeros_like(vel)
        vel_loc[:n_own] = vel[mine]
        acc_loc = torch.zeros_like(acc)
        slab_ev = [None]

        def slab_force_kick(xl, own, a, v):
            plan.bin(xl, active=own)
            if slab_ev[0] is not None:
                slab_ev[0][0].record()
            plan.force_kick(a, v, dt)
            if slab_ev[0] is not None:
                slab_ev[0][1].record()

    def step(ev=None):
        if slabbed:
            slab_ev[0] = ev
            slab_step(slabs, x_own, ids_own, acc_loc, vel_loc, slab_force_kick)
            plan.invariants(vel_loc[:n_own], acc_loc[:n_own], inv)
            return
        if graphed:
            # one captured graph: bin + persistent force + kick (over all volumes of a batch)
            if ev is not None:
                ev[0].record()
            plan.graph_launch()
            if ev is not None:
                ev[1].record()
        else:
            plan.bin(x)
            if ev is not None:
                ev[0].record()
            plan.force_kick(acc, vel, dt)          # pair sums with the kick fused into the epilogue
            if ev is not None:
                ev[1].record()
        plan.invariants(vel, acc, inv)

    # pair count of this configuration (binary32 predicate, counting variant)
    if slabbed:
        xl, _, own = slabs.exchange(x_own, ids_own)
        plan.bin(xl, active=own)
    else:
        plan.bin(x)
    tune_ms = None
    if args.variant >= 0:
        plan.set_variant(args.variant)
    elif not args.no_autotune and tune_geometry is None:
        tune_ms = plan.autotune(reps=1)
    _, pairs_t, _ = plan.force(acc_loc[:len(xl)] if slabbed else acc, count=True)   # slabs: owned rows' pairs
    torch.cuda.synchronize()
    pairs = int(pairs_t.item())
    info = plan.info()
    ctr = plan.export("counters").cpu().numpy()
    evals, lane_evals = int(ctr[3]), int(ctr[4])

    if graphed:
        torch.cuda.set_stream(graph_stream)
        plan.graph_capture(x, vel, acc, dt)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    uuid = str(getattr(props, "uuid", "")) if hasattr(props, "uuid") else ""
    sampler = ClockSampler(uuid if rank == 0 else "")
    if rank == 0 and not args.no_clocks:
        sampler.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = launch_count()
    t_start.record()
    for k in range(args.steps):
        step(evs[k])
    t_end.record()
    torch.cuda.synchronize()
    l1 = launch_count()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if (rank == 0 and not args.no_clocks) else None
    ms = t_start.elapsed_time(t_end) / args.steps
    force_ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    plan.status()

    pairs_all, ms_max = reduce_over_ranks(pairs, ms, world, dev)
    value = pairs_all / (ms_max * 1e-3)
    graph_ms = None
    if graphed:
        # the timed step is the captured graph (bin + pair kernel + kick);
        # the pair kernel itself is timed on the graph's binning, on the
        # same stream, with the kick applied to a scratch copy of vel
        graph_ms = force_ms
        vel_s = vel.clone()
        kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
        plan.force_kick(acc, vel_s, dt)
        for a, b in kev:
            a.record()
            plan.force_kick(acc, vel_s, dt)
            b.record()
        torch.cuda.synchronize()
        force_ms = float(np.mean([a.elapsed_time(b) for a, b in kev]))

    # plain one-launch-per-slab kernel on the same binned input
    plain = None
    if not args.no_plain and not slabbed:
        torch.cuda.set_stream(torch.cuda.default_stream())
        plan.bin(x)
        plan.force_plain(acc)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.force_plain(acc)
        e1.record()
        torch.cuda.synchronize()
        plain_ms = e0.elapsed_time(e1)
        plain = {"ms": plain_ms, "pairs_per_s": pairs / (plain_ms * 1e-3),
                 "speedup_of_persistent_kernel": plain_ms / force_ms}

    # end to end: pinned host buffers, H2D + step + D2H inside the timed region.
    # A stream of independent steps through sr_step_host_submit: each step
    # uploads its inputs and reads back its kicked velocities (the step's
    # result); the uploads of one step overlap the step before it.  Two
    # velocity buffers used in turn (a step's read-back and the next step's
    # upload are in flight together); the positions are only read.
    e2e = None
    if not args.no_e2e and not slabbed:
        torch.cuda.set_stream(torch.cuda.default_stream())
        pos_h = torch.from_numpy(pos).pin_memory()
        vel_h = [vel.cpu().pin_memory(), vel.cpu().pin_memory()]
        acc_h = [torch.empty((n, 4), dtype=torch.float32).pin_memory() for _ in range(2)]
        k_e2e = max(args.e2e_steps, 8)

        def pipelined(with_acc):
            for k in range(2):
                plan.step_host_submit(pos_h, vel_h[k], acc_h[k] if with_acc else None, dt)
            plan.step_host_wait()
            t0 = time.perf_counter()
            for k in range(k_e2e):
                plan.step_host_submit(pos_h, vel_h[k % 2], acc_h[k % 2] if with_acc else None, dt)
            plan.step_host_wait()
            return (time.perf_counter() - t0) / k_e2e

        e2e_s = pipelined(False)
        e2e_acc_s = pipelined(True)
        # one step at a time (sr_step_host: upload, step, read-back, wait)
        plan.step_host(pos_h, vel_h[0], None, dt)
        ts = []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            plan.step_host(pos_h, vel_h[0], None, dt)
            ts.append(time.perf_counter() - t0)
        e2e = {"value": pairs / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": int(n * (24 + 16)),
               "d2h_bytes_per_step": int(n * 16), "ms_per_step": e2e_s * 1e3,
               "ms_per_step_with_accelerations_read_back": e2e_acc_s * 1e3,
               "steps": k_e2e, "api": "sr_step_host_submit (stream of independent steps, copies overlapped)",
               "ms_per_step_one_at_a_time": float(np.median(ts)) * 1e3}

    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = pairs * FLOPS_PER_PAIR / (force_ms * 1e-3) / 1e12
    # the recorded counters are for the full clustered 256^3 launch only
    traffic = recorded_traffic() if (args.workload == "clustered256" and not args.n_particles) else None
    hbm_kernels = None if (batch or slabbed) else time_hbm_kernels(plan, x, acc, vel, n, float(peaks.get("hbm_gbs", 6400.0)))

    if rank != 0:
        return
    line = {
        "metric": METRICS["force"],
        "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "n_particles": n, "volumes": len(vols),
                   "box": box if not batch else [min(b for _, b in vols), max(b for _, b in vols)],
                   "graph": bool(graphed), "r_c": prm["rc"],
                   "eps": prm["eps"], "sigma": prm["sigma"], "dt": dt, "pairs_per_step": pairs,
                   "n_chunks": info["n_chunks"], "workers": info["workers"],
                   "variant": info["variant"], "autotune_ms": tune_ms, "tune_geometry": tune_geometry,
                   "chunk_size": info["chunk_size"],
                   "sub_bits": info["sub_bits"], "n_cells": plan.volume(0)["n_cells"],
                   "in_range_fraction": pairs / max(evals, 1),
                   "lane_fill": evals / max(lane_evals, 1),
                   "l2": f"inputs larger than L2 ({n * 24 / 1e6:.0f} MB positions); no flush",
                   "parallelism": (f"sharded{world}" if batch else f"slabs{world}") if world > 1 else "single"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": traffic,
                     "kernel": "k_pairs<force> (kick fused)", "kernel_ms": force_ms, "graph_ms": graph_ms,
                     "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (derived, not measured)",
                     "flops_per_pair": FLOPS_PER_PAIR},
        "plain": plain,
        "hbm_kernels": hbm_kernels,
        "e2e": e2e,
        "gpu_launches": int(l1 - l0),
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    emit(line)
    plan.close()


FOF_FLOPS_PER_TEST = 11    # 3 adds (anchor shift), 3 differences, 1 mul + 2 FMA for |d|^2
MUFU_PER_SM_CLK = 16      # rsqrt results per SM per clock (measured on B300: 16; ex2 runs at 32)


def _centers_inputs(n_particles=0):
    from workloads import configs as wc
    cfg = wc.resized("clustered256", n_particles) if n_particles else wc.CONFIGS["clustered256"]
    w = wc.make_workload(cfg)
    pos, box = w["volumes"][0]
    return pos, box, w["labels"].astype(np.int32), len(w["halo_sizes"]), w["params"]["eps"]


def cpu_centers_sample(pos, lab, box, eps, nh, budget, seed):
    """Time the FP64 oracle's halo potentials on a seeded sample of whole
    halos holding about `budget` ordered member pairs.  Returns
    (unordered pairs/s, pairs, seconds, halos)."""
    from oracle import centers as octr
    rng = np.random.default_rng(seed)
    sizes = np.bincount(lab[lab >= 0], minlength=nh).astype(np.int64)
    pick, terms = [], 0
    for h in rng.permutation(nh):
        if sizes[h] < 2 or terms + sizes[h] ** 2 > budget:
            continue
        pick.append(h)
        terms += int(sizes[h] ** 2)
    sel = np.isin(lab, pick)
    sub_pos, sub_lab = pos[sel], lab[sel]
    remap = -np.ones(nh, np.int64)
    remap[pick] = np.arange(len(pick))
    sub_lab = remap[sub_lab]
    t0 = time.perf_counter()
    octr.halo_potentials(sub_pos, sub_lab, box, eps)
    secs = time.perf_counter() - t0
    pairs = int(np.sum(sizes[pick] * (sizes[pick] - 1) // 2))
    return pairs / secs, pairs, secs, len(pick)


def run_centers(args, rank, world, local_rank):
    """Halo center finder on the 8,127 NFW halos of the clustered 256^3 set:
    one step = sr_centers_run (sort by halo, member slots, symmetric pair
    potential kernel, phi in caller order, per-halo argmin).  Metric:
    unordered member pairs per second (sum over halos of N_h (N_h - 1) / 2
    divided by the step time)."""
    pos, box, lab, nh, eps = _centers_inputs(args.n_particles)
    n = len(pos)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        rate, cp, secs, nsel = cpu_centers_sample(pos, lab, box, eps, nh, args.cpu_center_terms, 11)
        cpu = {"value": rate, "unit": "pairs/s", "cores": 1, "kind": "oracle",
               "sample": f"{nsel} whole halos of the same catalogue, {cp} unordered pairs in {secs:.1f} s "
                         "(FP64 NumPy blocked pair sums, one thread)"}

    import torch

    from paper_1411_3396_b300 import Centers, launch_count

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    props = torch.cuda.get_device_properties(dev)
    xd = torch.from_numpy(pos).to(dev)
    ld = torch.from_numpy(lab).to(dev)
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    cen = torch.empty(nh, dtype=torch.int64, device=dev)
    cphi = torch.empty(nh, dtype=torch.float64, device=dev)
    ctr = Centers(n, nh, "symmetric")

    def step(ev=None):
        ctr.prepare(xd, ld, nh, box, eps)
        if ev is not None:
            ev[0].record()
        ctr.potential()
        if ev is not None:
            ev[1].record()
        ctr.finish(phi, cen, cphi)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    info = ctr.info()
    pairs = int(info["pairs"])
    uuid = str(getattr(props, "uuid", "")) if hasattr(props, "uuid") else ""
    sampler = ClockSampler(uuid if rank == 0 else "")
    if rank == 0 and not args.no_clocks:
        sampler.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    l0 = launch_count()
    t_start.record()
    for k in range(args.steps):
        step(evs[k])
    t_end.record()
    torch.cuda.synchronize()
    l1 = launch_count()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if (rank == 0 and not args.no_clocks) else None
    ms = t_start.elapsed_time(t_end) / args.steps
    kern_ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    pairs_all, ms_max = reduce_over_ranks(pairs, ms, world, dev)

    # plain gather kernel (thread per member, two rsqrt per unordered pair)
    plain = None
    if not args.no_plain:
        ctr.set_variant("plain")
        ctr.prepare(xd, ld, nh, box, eps)
        ctr.potential()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctr.potential()
        e1.record()
        torch.cuda.synchronize()
        plain_ms = e0.elapsed_time(e1)
        plain = {"ms": plain_ms, "pairs_per_s": pairs / (plain_ms * 1e-3),
                 "speedup_of_symmetric_kernel": plain_ms / kern_ms}
        ctr.set_variant("symmetric")

    # end to end: positions and labels from pinned host memory, potentials
    # and centers back to pinned host memory, inside the timed region
    e2e = None
    if not args.no_e2e:
        pos_h = torch.from_numpy(pos).pin_memory()
        lab_h = torch.from_numpy(lab).pin_memory()
        phi_h = torch.empty(n, dtype=torch.float64).pin_memory()
        cen_h = torch.empty(nh, dtype=torch.int64).pin_memory()
        ts = []
        for k in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            xd.copy_(pos_h, non_blocking=True)
            ld.copy_(lab_h, non_blocking=True)
            step()
            phi_h.copy_(phi, non_blocking=True)
            cen_h.copy_(cen, non_blocking=True)
            torch.cuda.synchronize()
            if k:
                ts.append(time.perf_counter() - t0)
        e2e_s = float(np.median(ts))
        e2e = {"value": pairs / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": int(n * (24 + 4)),
               "d2h_bytes_per_step": int(n * 8 + nh * 8), "ms_per_step": e2e_s * 1e3}

    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    peak = props.multi_processor_count * MUFU_PER_SM_CLK * sm_max * 1e6
    achieved = pairs / (kern_ms * 1e-3)
    if rank != 0:
        ctr.close()
        return
    line = {
        "metric": METRICS["centers256"],
        "value": pairs_all / (ms_max * 1e-3), "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "centers256", "catalogue": "clustered256 NFW halos", "n_particles": n,
                   "n_members": info["n_members"], "n_halos": nh, "max_members": info["max_members"],
                   "eps": eps, "box": box, "pairs_per_step": pairs, "evaluated_per_step": info["evaluated"],
                   "items": info["items"], "fixed_shift": info["fixed_shift"],
                   "l2": "inputs larger than L2 (402 MB positions); no flush",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "rsqrt/s (MUFU)",
                     "frac": achieved / peak,
                     "traffic": recorded_traffic(CENTERS_NOTE, ("centers.cu",)) if not args.n_particles else None,
                     "kernel": "k_ctr_pairs", "kernel_ms": kern_ms,
                     "peak_basis": f"{props.multi_processor_count} SMs x {MUFU_PER_SM_CLK} MUFU rsqrt/clk x "
                                   f"{sm_max:.0f} MHz (rate measured by a probe; one rsqrt per unordered pair)"},
        "plain": plain,
        "e2e": e2e,
        "gpu_launches": int(l1 - l0),
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    emit(line)
    ctr.close()


def _pm_inputs(n_particles=0):
    from workloads import configs as wc
    cfg = wc.resized("clustered256", n_particles) if n_particles else wc.CONFIGS["clustered256"]
    w = wc.make_workload(cfg)
    (pos, box), = w["volumes"]
    return pos, box, w["params"]["sigma"]


def cpu_pm_sample(seed_n=128 ** 3):
    """Time the FP64 oracle's long-range step (CIC deposit, FFT, P(k), PM
    accelerations of every particle) on the clustered set resized to
    seed_n particles and a seed_n grid.  Returns (particles/s, n, seconds)."""
    from oracle import pm as opm
    pos, box, sigma = _pm_inputs(seed_n)
    ng = int(round(len(pos) ** (1.0 / 3.0)))
    t0 = time.perf_counter()
    opm.power_spectrum(pos, box, ng)
    opm.pm_accel(pos, box, ng, sigma)
    secs = time.perf_counter() - t0
    return len(pos) / secs, len(pos), secs


def run_pm(args, rank, world, local_rank):
    """Long-range side on the clustered 256^3 set with a 256^3 mesh: one
    step = sr_pm_deposit (CIC counts, delta, forward FFT) + sr_pm_power
    (CIC-compensated P(k)) + sr_pm_force (filtered spectral accelerations,
    two inverse FFTs, CIC interpolation to every particle).  Metric:
    particles per second through the step."""
    pos, box, sigma = _pm_inputs(args.n_particles)
    n = len(pos)
    ng = args.n_grid or int(round(n ** (1.0 / 3.0)))
    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        rate, cn, secs = cpu_pm_sample()
        cpu = {"value": rate, "unit": "particles/s", "cores": 1, "kind": "oracle",
               "sample": f"the same clustered catalogue resized to {cn} particles on a {round(cn ** (1 / 3))}^3 "
                         f"mesh, whole step (deposit, FFT, P(k), accelerations) in {secs:.1f} s (FP64 NumPy)"}

    import torch

    from paper_1411_3396_b300 import PM, launch_count

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    props = torch.cuda.get_device_properties(dev)
    x = torch.from_numpy(pos).to(dev)
    acc = torch.empty((n, 4), dtype=torch.float32, device=dev)
    pm = PM(ng, box, sigma, n)

    def step(ev=None):
        if ev is not None:
            ev[0].record()
        pm.deposit(x, transform=False)
        if ev is not None:
            ev[1].record()
        pm.transform()
        if ev is not None:
            ev[2].record()
        k, p, m = pm.power()
        if ev is not None:
            ev[3].record()
        pm.force(x, acc)
        if ev is not None:
            ev[4].record()
        return k, p, m

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    uuid = str(getattr(props, "uuid", "")) if hasattr(props, "uuid") else ""
    sampler = ClockSampler(uuid if rank == 0 else "")
    if rank == 0 and not args.no_clocks:
        sampler.start()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    l0 = launch_count()
    t_start.record()
    for kk in range(args.steps):
        step(evs[kk])
    t_end.record()
    torch.cuda.synchronize()
    l1 = launch_count()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if (rank == 0 and not args.no_clocks) else None
    ms = t_start.elapsed_time(t_end) / args.steps
    phases = {name: float(np.mean([e[i].elapsed_time(e[i + 1]) for e in evs]))
              for i, name in enumerate(("deposit_ms", "transform_ms", "power_ms", "force_ms"))}
    n_all, ms_max = reduce_over_ranks(n, ms, world, dev)

    # FFT pass against the HBM roofline: one forward transform (three
    # passes, each reading and writing every complex64 point) timed alone
    scratch = torch.randn((ng, ng, ng), dtype=torch.complex64, device=dev)
    for _ in range(2):
        pm.fft(scratch)
    reps = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        pm.fft(scratch)
    e1.record()
    torch.cuda.synchronize()
    pass_ms = e0.elapsed_time(e1) / (3 * reps)
    pass_bytes = 16 * ng ** 3
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    fft_gbs = pass_bytes / (pass_ms * 1e-3) / 1e9
    # dominant kernel: the CIC deposit (positions read once, the 8-byte
    # fixed-point counters read and written once)
    dep_bytes = 24 * n + 16 * ng ** 3
    dep_gbs = dep_bytes / (phases["deposit_ms"] * 1e-3) / 1e9
    # the same deposit over a short-range binning's cell order (as in the
    # force-split step, where the binning is there anyway): timed alone
    from paper_1411_3396_b300 import Plan
    bplan = Plan(box, 3.0, 0.05, sigma, n)
    bplan.bin(x)
    pm.deposit(x, transform=False, plan=bplan)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        pm.deposit(x, transform=False, plan=bplan)
    e1.record()
    torch.cuda.synchronize()
    dep_binned_ms = e0.elapsed_time(e1) / reps
    bplan.close()

    e2e = None
    if not args.no_e2e:
        pos_h = torch.from_numpy(pos).pin_memory()
        acc_h = torch.empty((n, 4), dtype=torch.float32).pin_memory()
        pk_h = torch.empty(ng // 2, dtype=torch.float64).pin_memory()
        ts = []
        for kk in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x.copy_(pos_h, non_blocking=True)
            _, p, _ = step()
            acc_h.copy_(acc, non_blocking=True)
            pk_h.copy_(p, non_blocking=True)
            torch.cuda.synchronize()
            if kk:
                ts.append(time.perf_counter() - t0)
        e2e_s = float(np.median(ts))
        e2e = {"value": n / e2e_s, "unit": "particles/s", "h2d_bytes_per_step": int(n * 24),
               "d2h_bytes_per_step": int(n * 16 + (ng // 2) * 8), "ms_per_step": e2e_s * 1e3}
    if rank != 0:
        pm.close()
        return
    line = {
        "metric": METRICS["pm256"],
        "value": n_all / (ms_max * 1e-3), "unit": "particles/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "pm256", "catalogue": "clustered256 particles", "n_particles": n, "n_grid": ng,
                   "box": box, "sigma": sigma, **phases,
                   "l2": "inputs larger than L2 (402 MB positions, 134 MB complex grid); no flush",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": dep_gbs, "peak": hbm, "unit": "GB/s", "frac": dep_gbs / hbm,
                     "traffic": None, "kernel": "k_cic_deposit (caller-order particles, 8 fixed-point atomics each)",
                     "kernel_ms": phases["deposit_ms"], "bytes_per_launch": dep_bytes,
                     "peak_basis": "measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "fft_pass": {"achieved": fft_gbs, "frac": fft_gbs / hbm, "kernel_ms": pass_ms,
                                  "bytes_per_launch": pass_bytes, "kernel": "k_fft_pass (one axis)"},
                     "deposit_binned": {"kernel": "k_cic_deposit_chunks (over a short-range binning's "
                                                  "chunks, on-chip tiles; same counts bit for bit)",
                                        "kernel_ms": dep_binned_ms,
                                        "achieved": dep_bytes / (dep_binned_ms * 1e-3) / 1e9,
                                        "frac": dep_bytes / (dep_binned_ms * 1e-3) / 1e9 / hbm}},
        "e2e": e2e,
        "gpu_launches": int(l1 - l0),
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    emit(line)
    pm.close()


def cpu_fof_sample(seed_n=128 ** 3, link=0.168):
    """Time the FP64 oracle's FOF (k-d tree pairs, exact predicate, graph
    components) on the clustered set resized to seed_n particles."""
    from oracle import fof as ofof
    pos, box, _ = _pm_inputs(seed_n)
    t0 = time.perf_counter()
    ofof.fof(pos, box, link, 40)
    secs = time.perf_counter() - t0
    return len(pos) / secs, len(pos), secs


def run_fof(args, rank, world, local_rank):
    """Friends-of-friends on the clustered 256^3 set (linking length 0.168
    mean spacings, halos of at least 40 particles), then the most-bound
    particle of every FOF halo: the in-situ analysis chain.  One step =
    sr_bin + sr_fof_run (+ the center finder, timed separately).  Metric:
    particles per second through binning and FOF."""
    pos, box, _ = _pm_inputs(args.n_particles)
    n = len(pos)
    link = args.fof_b * box / round(n ** (1.0 / 3.0))
    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        rate, cn, secs = cpu_fof_sample(link=args.fof_b)
        cpu = {"value": rate, "unit": "particles/s", "cores": 1, "kind": "oracle",
               "sample": f"the same clustered catalogue resized to {cn} particles, FOF in {secs:.1f} s "
                         "(FP64 k-d tree pairs + exact predicate + graph components)"}

    import torch

    from paper_1411_3396_b300 import FOF, Centers, Plan, launch_count
    from workloads import configs as wc

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    props = torch.cuda.get_device_properties(dev)
    prm = wc.CONFIGS["clustered256"]
    x = torch.from_numpy(pos).to(dev)
    plan = Plan(box, prm["rc"], prm["eps"], prm["sigma"], n)
    fof = FOF(n)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    hsizes = torch.empty(n, dtype=torch.int32, device=dev)

    def step(ev=None):
        if ev is not None:
            ev[0].record()
        plan.bin(x)
        if ev is not None:
            ev[1].record()
        fof.run(plan, x, link, 40, labels, hsizes)
        if ev is not None:
            ev[2].record()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    info = fof.info()
    uuid = str(getattr(props, "uuid", "")) if hasattr(props, "uuid") else ""
    sampler = ClockSampler(uuid if rank == 0 else "")
    if rank == 0 and not args.no_clocks:
        sampler.start()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    l0 = launch_count()
    t_start.record()
    for k in range(args.steps):
        step(evs[k])
    t_end.record()
    torch.cuda.synchronize()
    l1 = launch_count()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if (rank == 0 and not args.no_clocks) else None
    ms = t_start.elapsed_time(t_end) / args.steps
    bin_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
    fof_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in evs]))
    n_all, ms_max = reduce_over_ranks(n, ms, world, dev)

    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = info["tests"] * FOF_FLOPS_PER_TEST / (fof_ms * 1e-3) / 1e12

    # end to end: positions from pinned host memory, labels back
    e2e = None
    if not args.no_e2e:
        pos_h = torch.from_numpy(pos).pin_memory()
        lab_h = torch.empty(n, dtype=torch.int32).pin_memory()
        ts = []
        for k in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x.copy_(pos_h, non_blocking=True)
            step()
            lab_h.copy_(labels, non_blocking=True)
            torch.cuda.synchronize()
            if k:
                ts.append(time.perf_counter() - t0)
        e2e_s = float(np.median(ts))
        e2e = {"value": n / e2e_s, "unit": "particles/s", "h2d_bytes_per_step": int(n * 24),
               "d2h_bytes_per_step": int(n * 4), "ms_per_step": e2e_s * 1e3}

    # centers of the FOF halos (the catalogue the paper's center finder reads)
    nh = int(info["n_halos"])
    ctr = Centers(n, max(nh, 1))
    phi, cen, cphi = ctr.run(x, labels, nh, box, prm["eps"])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctr.run(x, labels, nh, box, prm["eps"], phi, cen, cphi)
    e1.record()
    torch.cuda.synchronize()
    cinfo = ctr.info()
    centers_ms = e0.elapsed_time(e1)
    ctr.close()
    fof.close()
    plan.close()
    if rank != 0:
        return
    line = {
        "metric": METRICS["fof256"],
        "value": n_all / (ms_max * 1e-3), "unit": "particles/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "fof256", "catalogue": "clustered256 particles", "n_particles": n, "box": box,
                   "link": link, "b": args.fof_b, "min_members": 40, "bin_ms": bin_ms, "fof_ms": fof_ms,
                   "n_halos": nh, "n_members": info["n_members"], "max_members": info["max_members"],
                   "links": info["links"], "band_checks": info["band_checks"],
                   "centers_of_fof_halos": {"ms": centers_ms, "pairs": cinfo["pairs"],
                                            "pairs_per_s": cinfo["pairs"] / (centers_ms * 1e-3)},
                   "l2": "inputs larger than L2 (402 MB positions); no flush",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": None, "kernel": "k_fof_pairs",
                     "kernel_ms": fof_ms, "flops_per_test": FOF_FLOPS_PER_TEST, "tests": info["tests"],
                     "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz "
                                   "(derived); the kernel is bound by union-find and load latency, not by the ALU"},
        "e2e": e2e,
        "gpu_launches": int(l1 - l0),
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    emit(line)


def run_step(args, rank, world, local_rank):
    """One whole time step of the force split on the clustered 256^3 set:
    sr_bin -> sr_force (short range) -> sr_pm_deposit + sr_pm_transform +
    sr_pm_power (on-the-fly P(k)) -> sr_pm_force added onto the short-range
    accelerations -> sr_kick -> sr_invariants.  Metric: particles per
    second through the whole step."""
    cfg, vols, vel_np, prm = make_inputs("clustered256", args.n_particles, world, rank)
    (pos, box), = vols
    n = len(pos)
    ng = args.n_grid or int(round(n ** (1.0 / 3.0)))

    import torch

    from paper_1411_3396_b300 import PM, Plan, kick, launch_count

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    props = torch.cuda.get_device_properties(dev)
    x = torch.from_numpy(pos).to(dev)
    vel = torch.zeros((n, 4), dtype=torch.float32, device=dev)
    vel[:, :3] = torch.from_numpy(vel_np).to(dev).float()
    acc = torch.empty((n, 4), dtype=torch.float32, device=dev)
    inv = torch.empty(7, dtype=torch.float64, device=dev)
    plan = Plan(box, prm["rc"], prm["eps"], prm["sigma"], n)
    pm = PM(ng, box, prm["sigma"], n)
    dt = prm["dt"]
    plan.bin(x)
    if args.variant >= 0:
        plan.set_variant(args.variant)
    else:
        plan.autotune(reps=1)
    _, pairs_t, _ = plan.force(acc, count=True)
    torch.cuda.synchronize()
    pairs = int(pairs_t.item())

    def step(ev=None):
        if ev is not None:
            ev[0].record()
        plan.bin(x)
        if ev is not None:
            ev[3].record()
        plan.force(acc)
        if ev is not None:
            ev[1].record()
        pm.deposit(x, plan=plan)                   # over the short-range binning's cell order
        pk = pm.power()
        pm.force(x, acc, accumulate=True)
        if ev is not None:
            ev[2].record()
        kick(acc, vel, dt)
        plan.invariants(vel, acc, inv)
        return pk

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    uuid = str(getattr(props, "uuid", "")) if hasattr(props, "uuid") else ""
    sampler = ClockSampler(uuid if rank == 0 else "")
    if rank == 0 and not args.no_clocks:
        sampler.start()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    l0 = launch_count()
    t_start.record()
    for k in range(args.steps):
        step(evs[k])
    t_end.record()
    torch.cuda.synchronize()
    l1 = launch_count()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if (rank == 0 and not args.no_clocks) else None
    ms = t_start.elapsed_time(t_end) / args.steps
    sr_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
    force_ms = float(np.mean([e[3].elapsed_time(e[1]) for e in evs]))
    lr_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in evs]))
    n_all, ms_max = reduce_over_ranks(n, ms, world, dev)
    plan.status()

    # end to end: positions and velocities from pinned host memory, the kicked
    # velocities back, every step
    e2e = None
    if not args.no_e2e:
        pos_h = torch.from_numpy(pos).pin_memory()
        vel_h = vel.cpu().pin_memory()
        out_h = torch.empty_like(vel_h).pin_memory()
        ts = []
        for k in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x.copy_(pos_h, non_blocking=True)
            vel.copy_(vel_h, non_blocking=True)
            step()
            out_h.copy_(vel, non_blocking=True)
            torch.cuda.synchronize()
            if k:
                ts.append(time.perf_counter() - t0)
        e2e_s = float(np.median(ts))
        e2e = {"value": n / e2e_s, "unit": "particles/s", "h2d_bytes_per_step": int(n * (24 + 16)),
               "d2h_bytes_per_step": int(n * 16), "ms_per_step": e2e_s * 1e3}
    pm.close()
    plan.close()
    if rank != 0:
        return
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = pairs * FLOPS_PER_PAIR / (force_ms * 1e-3) / 1e12
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rate, cn, el = cpu_step_sample(32 ** 3)
        cpu = {"value": rate, "unit": "particles/s", "cores": 1, "kind": "oracle",
               "sample": f"the whole oracle step on the clustered catalogue resized to {cn} particles "
                         f"({el:.1f} s, FP64 NumPy, one thread)"}
    line = {
        "metric": METRICS["step256"],
        "value": n_all / (ms_max * 1e-3), "unit": "particles/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "step256", "catalogue": "clustered256 particles", "n_particles": n, "n_grid": ng,
                   "box": box, "r_c": prm["rc"], "eps": prm["eps"], "sigma": prm["sigma"], "dt": dt,
                   "short_range_ms": sr_ms, "long_range_ms": lr_ms, "pairs_per_step": pairs,
                   "short_range_pairs_per_s": pairs / (sr_ms * 1e-3),
                   "l2": "inputs larger than L2 (402 MB positions); no flush",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": None,
                     "kernel": "k_pairs<force> (the step's dominant kernel; kick applied separately after PM)",
                     "kernel_ms": force_ms, "flops_per_pair": FLOPS_PER_PAIR,
                     "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz "
                                   "(derived, not measured)"},
        "e2e": e2e,
        "gpu_launches": int(l1 - l0),
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    emit(line)


def cpu_step_sample(sample_n):
    """The FP64 oracle's whole force-split step (short-range accelerations
    by k-d tree, P(k), PM accelerations) on the clustered catalogue resized
    to sample_n particles, one thread.  Returns (particles/s, n, seconds)."""
    from oracle import fit as ofit
    from oracle import force as oforce
    from oracle import pm as opm
    from workloads import configs as wc
    pos, box, sigma = _pm_inputs(sample_n)
    prm = wc.CONFIGS["clustered256"]
    c = ofit.fit_poly(prm["rc"], sigma, prm["eps"])
    ng = int(round(len(pos) ** (1 / 3)))
    t0 = time.perf_counter()
    oforce.accel_kdtree(pos, box, prm["rc"], prm["eps"], c)
    opm.power_spectrum(pos, box, ng)
    opm.pm_accel(pos, box, ng, sigma)
    el = time.perf_counter() - t0
    return len(pos) / el, len(pos), el


def run_reference_other(args, rank, world):
    """Reference arm of the pm256, fof256 and step256 modes: the FP64
    oracle of the same step on a bounded sample of the same catalogue."""
    if rank != 0:
        return
    per = []
    sample_n = 32 ** 3 if args.workload == "step256" else 64 ** 3
    for k in range(args.warmup + args.steps):
        if args.workload == "pm256":
            rate, cn, _ = cpu_pm_sample(sample_n)
        elif args.workload == "fof256":
            rate, cn, _ = cpu_fof_sample(sample_n, args.fof_b)
        else:
            rate, cn, _ = cpu_step_sample(sample_n)
        per.append(rate)
    value = float(np.mean(per[args.warmup:]))
    line = {
        "impl": "reference", "metric": METRICS[args.workload],
        "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "catalogue": "clustered256 resized", "sample_particles": sample_n},
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": 1, "kind": "oracle",
                         "sample": f"per step the whole oracle step on the clustered catalogue resized to "
                                   f"{sample_n} particles"},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    emit(line)


def run_reference_centers(args, rank, world):
    pos, box, lab, nh, eps = _centers_inputs(args.n_particles)
    if rank != 0:
        return
    per = []
    for k in range(args.warmup + args.steps):
        rate, cp, secs, nsel = cpu_centers_sample(pos, lab, box, eps, nh, args.cpu_center_terms // 16, 100 + k)
        per.append(rate)
    value = float(np.mean(per[args.warmup:]))
    line = {
        "impl": "reference",
        "metric": METRICS["centers256"],
        "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "centers256", "catalogue": "clustered256 NFW halos", "n_particles": len(pos),
                   "n_halos": nh, "eps": eps, "box": box},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                         "sample": "per step, a seeded sample of whole halos (FP64 NumPy blocked pair sums)"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    emit(line)


VJP_FLOPS_PER_PAIR = 55   # d, s', r^2, r^3, q and q' (Horner), f, f', g_j - g_i, d.dg, w, two FMA per component


def run_diff(args, rank, world, local_rank):
    """Differentiable workload: one timed step = a 10-substep kick-drift
    trajectory forward and its backward sweep (autograd over sr_force_vjp).
    Metric: pair interactions per second, forward force pairs plus VJP
    pairs (the same pair sets again in the backward sweep)."""
    import torch

    from paper_1411_3396_b300 import Plan, TrajectoryGraph, launch_count, trajectory
    from workloads import configs as wc
    from workloads import generators as gen

    cfg = wc.resized("diff64", args.n_particles) if args.n_particles else wc.CONFIGS["diff64"]
    box, n_side, steps, dt = cfg["box"], cfg["n_side"], cfg["steps"], cfg["dt"]
    x0, psi = gen.zeldovich(n_side, box, cfg.get("rms", 0.5), cfg["seed"])
    xt, _ = gen.zeldovich(n_side, box, cfg.get("rms", 0.5), cfg["seed"] + 1)
    v0 = 0.1 * psi
    n = len(x0)
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    props = torch.cuda.get_device_properties(dev)
    plan = Plan(box, cfg["rc"], cfg["eps"], cfg["sigma"], n, chunk_size=args.chunk_size)
    xd = torch.from_numpy(x0).to(dev)
    vd = torch.zeros((n, 4), dtype=torch.float32, device=dev)
    vd[:, :3] = torch.from_numpy(v0).to(dev).float()
    target = torch.from_numpy(xt).to(dev)

    def loss_fn(xk, vk):
        d = xk - target
        d = d - box * torch.round(d / box)
        return (d * d).sum()

    def eager(xi, vi):
        x = xi.detach().clone().requires_grad_(True)
        v = vi.detach().clone().requires_grad_(True)
        xk, vk = trajectory(traj_plans, x, v, steps, dt)
        loss = loss_fn(xk, vk)
        loss.backward()
        return loss, x.grad, v.grad

    # pairs of every substep's configuration (counting kernel, untimed)
    pairs = 0
    with torch.no_grad():
        x = xd.clone()
        v = vd.clone()
        acc = torch.empty_like(v)
        from paper_1411_3396_b300 import kick
        for _ in range(steps):
            plan.bin(x)
            _, pt, _ = plan.force(acc, count=True)
            pairs += int(pt.item())
            kick(acc, v, dt)
            plan.drift(x, v, dt)
    if args.variant >= 0:
        plan.set_variant(args.variant)
    else:
        plan.bin(xd)
        plan.autotune(reps=2)
    # one plan per substep (each substep binned once, its binning kept for
    # the backward sweep), unless --shared-plan (binned again backwards)
    traj_plans = plan
    if not args.shared_plan and steps > 1:
        variant = plan.info()["variant"]
        traj_plans = [plan] + [Plan(box, cfg["rc"], cfg["eps"], cfg["sigma"], n, chunk_size=args.chunk_size)
                               for _ in range(steps - 1)]
        for p in traj_plans[1:]:
            p.set_variant(variant)
    # eager trajectories (autograd issuing every launch from the host), then
    # the same sweep captured once in a CUDA graph and replayed
    for _ in range(args.warmup):
        eager(xd, vd)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        eager(xd, vd)
    e1.record()
    torch.cuda.synchronize()
    eager_ms = e0.elapsed_time(e1) / args.steps
    if args.no_graph:
        one = eager
    else:
        tg = TrajectoryGraph(traj_plans, xd, vd, steps, dt, loss_fn)

        def one(xi, vi):
            return tg.run(xi, vi)
    for _ in range(args.warmup):
        one(xd, vd)
    torch.cuda.synchronize()
    uuid = str(getattr(props, "uuid", "")) if hasattr(props, "uuid") else ""
    sampler = ClockSampler(uuid if rank == 0 else "")
    if rank == 0 and not args.no_clocks:
        sampler.start()
    l0 = launch_count()
    e0.record()
    for _ in range(args.steps):
        loss, gx, gv = one(xd, vd)
    e1.record()
    torch.cuda.synchronize()
    l1 = launch_count()
    clocks = sampler.stop() if (rank == 0 and not args.no_clocks) else None
    if not args.no_graph:
        l1 = l0 + tg.kernels * args.steps         # replays launch the captured kernels
    ms = e0.elapsed_time(e1) / args.steps
    total_pairs = 2 * pairs
    # kernel roofline on the initial configuration: force + VJP
    plan.bin(xd)
    g = torch.randn((n, 4), dtype=torch.float32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(2):
        plan.force(acc)
        plan.vjp(g)
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(5):
        plan.force(acc)
    ev[1].record()
    for _ in range(5):
        plan.vjp(g)
    ev[2].record()
    torch.cuda.synchronize()
    t_f = ev[0].elapsed_time(ev[1]) / 5
    t_v = ev[1].elapsed_time(ev[2]) / 5
    p0 = pairs / steps
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = p0 * (FLOPS_PER_PAIR + VJP_FLOPS_PER_PAIR) / ((t_f + t_v) * 1e-3) / 1e12
    # end to end: H2D of x0, v0 from pinned memory, D2H of both gradients
    x_h = torch.from_numpy(x0).pin_memory()
    v_h = vd.cpu().pin_memory()
    gx_h = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    gv_h = torch.empty((n, 4), dtype=torch.float32).pin_memory()
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        xi = x_h.to(dev, non_blocking=True)
        vi = v_h.to(dev, non_blocking=True)
        _, gx, gv = one(xi, vi)
        gx_h.copy_(gx, non_blocking=True)
        gv_h.copy_(gv, non_blocking=True)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    e2e_s = float(np.median(ts))
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rates, n_s, st_s = cpu_diff_sample(0, 2)
        cpu = {"value": float(np.mean(rates)), "unit": "pairs/s", "cores": 1, "kind": "oracle",
               "sample": diff_sample_note(n_s, st_s)}
    line = {
        "metric": METRICS["diff64"],
        "value": total_pairs / (ms * 1e-3), "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "diff64", "n_particles": n, "box": box, "substeps": steps, "dt": dt,
                   "r_c": cfg["rc"], "eps": cfg["eps"], "sigma": cfg["sigma"],
                   "pairs_forward": pairs, "pairs_per_step": total_pairs,
                   "trajectories_per_s": 1e3 / ms, "loss": float(loss.item()),
                   "graph": not args.no_graph, "eager_ms_per_step": eager_ms,
                   "plans": 1 if isinstance(traj_plans, Plan) else len(traj_plans),
                   "variant": plan.info()["variant"],
                   "binnings_per_trajectory": steps if not isinstance(traj_plans, Plan) else 2 * steps,
                   "parallelism": "single"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": None,
                     "kernel": "k_pairs<force> + k_pairs<vjp> on x_0", "force_ms": t_f, "vjp_ms": t_v,
                     "flops_per_pair": [FLOPS_PER_PAIR, VJP_FLOPS_PER_PAIR]},
        "e2e": {"value": total_pairs / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": int(n * (24 + 16)),
                "d2h_bytes_per_step": int(n * (24 + 16)), "ms_per_step": e2e_s * 1e3},
        "gpu_launches": int(l1 - l0),
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    emit(line)
    plan.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="clustered256")
    ap.add_argument("--n-particles", type=int, default=0,
                    help="resize the workload (box scaled to keep density 1); 0 = as named")
    ap.add_argument("--cpu-rows", type=int, default=24576)
    ap.add_argument("--ref-rows", type=int, default=8192)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--n-grid", type=int, default=0, help="PM mesh points per axis (0 = cube root of n)")
    ap.add_argument("--fof-b", type=float, default=0.168, help="FOF linking length in mean spacings")
    ap.add_argument("--cpu-center-terms", type=int, default=250_000_000,
                    help="ordered member pairs in the oracle's center-finder sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="diff64: time eager trajectories only")
    ap.add_argument("--shared-plan", action="store_true",
                    help="diff64: one plan for every substep (binned again in the backward sweep)")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tune-geometry", action="store_true",
                    help="single volume: choose chunk size and cells per axis by timing as well (sr_plan_tune)")
    ap.add_argument("--variant", type=int, default=-1, help="force a pair-kernel variant (skips autotuning)")
    ap.add_argument("--chunk-size", type=int, default=0, help="particles per chunk: 32 or 64 (0 = library default)")
    ap.add_argument("--n-cells", type=int, default=0, help="cells per axis (0 = library default)")
    ap.add_argument("--sub-bits", type=int, default=0, help="Morton bits per axis in a cell (0 = default)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            if args.workload == "centers256":
                run_reference_centers(args, rank, world)
            elif args.workload in ("pm256", "fof256", "step256"):
                run_reference_other(args, rank, world)
            elif args.workload == "diff64":
                run_reference_diff(args, rank, world)
            else:
                run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.workload == "diff64":
        run_diff(args, rank, world, local_rank)
    elif args.workload == "centers256":
        run_centers(args, rank, world, local_rank)
    elif args.workload == "pm256":
        run_pm(args, rank, world, local_rank)
    elif args.workload == "fof256":
        run_fof(args, rank, world, local_rank)
    elif args.workload == "step256":
        run_step(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
