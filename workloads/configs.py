"""Named workloads: particle sets plus the physics parameters they run with.

Lengths are in cells (mean inter-particle spacing).  Seeds are 1000 + the
workload's index.  Where a workload's description leaves a parameter open
(softening or time step of the larger sets, initial velocities), the value
used here is recorded with the workload.
"""
from __future__ import annotations

import numpy as np

from . import generators as g

CONFIGS = {
    # 4,096 uniform particles, box 16, the plain-method case.
    "uniform4k": dict(kind="uniform", n=4096, box=16.0, rc=3.0, eps=0.1,
                      sigma=0.8, dt=0.01, seed=1000),
    # 128^3 Zel'dovich lattice, P(k) ~ k^-2, rms displacement 0.5 cell.
    "zeldovich128": dict(kind="zeldovich", n_side=128, box=128.0, rms=0.5,
                         rc=3.0, eps=0.1, sigma=0.8, dt=0.01, seed=1001),
    # 256^3 particles: half in NFW halos (100..200,000 particles), half uniform.
    "clustered256": dict(kind="nfw", n=256 ** 3, box=256.0, rc=3.0, eps=0.05,
                         sigma=0.8, dt=0.01, seed=1002, m_lo=100.0,
                         m_hi=200000.0),
    # 64 independent Zel'dovich sub-volumes, 10^4..10^6 particles each.
    "batch64": dict(kind="batch", n_vol=64, log_lo=4.0, log_hi=6.0, rms=0.5,
                    rc=3.0, eps=0.1, sigma=0.8, dt=0.01, seed=1003),
    # 64^3 Zel'dovich lattice, 10 kick-drift substeps, dt = 0.02.
    "diff64": dict(kind="zeldovich", n_side=64, box=64.0, rms=0.5, rc=3.0,
                   eps=0.1, sigma=0.8, dt=0.02, steps=10, seed=1004),
}

# Reduced versions of each workload, small enough for a full element-by-element
# oracle comparison in seconds, still spanning many chunks and ragged cells.
SMALL = {
    "uniform4k": dict(),
    "zeldovich128": dict(n_side=32, box=32.0),
    "clustered256": dict(n=32 ** 3, box=32.0, m_hi=3000.0),
    "batch64": dict(n_vol=4, log_lo=3.0, log_hi=3.6),
    "diff64": dict(n_side=16, box=16.0),
}


def small_variant(name: str) -> dict:
    cfg = dict(CONFIGS[name])
    cfg.update(SMALL[name])
    return cfg


def resized(name: str, n: int) -> dict:
    """A workload with n particles and the box scaled to keep the mean
    density of one particle per cell (box side round(n^(1/3)))."""
    cfg = dict(CONFIGS[name])
    side = float(round(n ** (1.0 / 3.0)))
    if cfg["kind"] == "zeldovich":
        cfg.update(n_side=int(side), box=side)
    else:
        cfg.update(n=int(n), box=side)
    return cfg


def make_workload(cfg: dict) -> dict:
    """Materialise a workload description.

    Returns dict(volumes=[(positions (n,3) float64, box)], velocities (N,3),
    params=dict(rc, eps, sigma, dt)) where N is the total over volumes and
    velocities follow the concatenated volume order.
    """
    kind = cfg["kind"]
    seed = int(cfg["seed"])
    extra = {}
    if kind == "uniform":
        vols = [(g.uniform_box(cfg["n"], cfg["box"], seed), cfg["box"])]
    elif kind == "zeldovich":
        pos, psi = g.zeldovich(cfg["n_side"], cfg["box"], cfg.get("rms", 0.5), seed)
        vols = [(pos, cfg["box"])]
        extra["psi"] = psi
    elif kind == "nfw":
        pos, labels, sizes = g.nfw_clustered(cfg["n"], cfg["box"], seed,
                                             m_lo=cfg.get("m_lo", 100.0),
                                             m_hi=cfg.get("m_hi", 200000.0))
        vols = [(pos, cfg["box"])]
        extra["labels"] = labels
        extra["halo_sizes"] = sizes
    elif kind == "batch":
        vols = g.batch_volumes(cfg["n_vol"], seed, cfg["log_lo"], cfg["log_hi"],
                               cfg.get("rms", 0.5))
    else:
        raise ValueError(kind)
    n_tot = sum(p.shape[0] for p, _ in vols)
    vel = g.velocities(n_tot, seed + 500)
    params = {k: cfg[k] for k in ("rc", "eps", "sigma", "dt")}
    out = dict(volumes=vols, velocities=vel, params=params, cfg=cfg)
    out.update(extra)
    return out


def concat_positions(work: dict) -> np.ndarray:
    return np.concatenate([p for p, _ in work["volumes"]], axis=0)
