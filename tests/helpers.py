"""Shared helpers of the GPU parity tests: run the CUDA path through the
C ABI, run the oracle on the same seeded inputs, compare."""
from __future__ import annotations

import numpy as np

from oracle import binning as obin
from oracle import fit as ofit
from oracle import force as oforce

# Force tolerance: rel_i = |a_gpu - a_ref| / max(|a_ref|, 1e-3 rms|a_ref|);
# median <= 1e-5 and max <= 1e-4.
MEDIAN_TOL = 1e-5
MAX_TOL = 1e-4


def rel_errors(a_gpu, a_ref):
    a_gpu = np.asarray(a_gpu, np.float64)[:, :3]
    a_ref = np.asarray(a_ref, np.float64)[:, :3]
    mag = np.linalg.norm(a_ref, axis=1)
    rms = np.sqrt(np.mean(mag * mag)) if mag.size else 1.0
    den = np.maximum(mag, 1e-3 * rms)
    den[den == 0] = 1.0
    return np.linalg.norm(a_gpu - a_ref, axis=1) / den


def assert_force_close(a_gpu, a_ref, what=""):
    rel = rel_errors(a_gpu, a_ref)
    med, mx = float(np.median(rel)), float(rel.max())
    assert med <= MEDIAN_TOL and mx <= MAX_TOL, f"{what}: median {med:.3g} max {mx:.3g}"
    return med, mx


def make_plan(vols, params, sub_bits=0, n_cells=None, chunk_size=0):
    """Plan for a list of (positions, box) volumes with physics params."""
    from paper_1411_3396_b300 import Plan
    if len(vols) == 1:
        pos, box = vols[0]
        return Plan(box, params["rc"], params["eps"], params["sigma"], len(pos),
                    n_cells=(n_cells or [0])[0], sub_bits=sub_bits, chunk_size=chunk_size)
    return Plan.batch([b for _, b in vols], [len(p) for p, _ in vols], params["rc"], params["eps"],
                      params["sigma"], n_cells=n_cells, sub_bits=sub_bits, chunk_size=chunk_size)


def oracle_binning(plan, vols):
    info = plan.info()
    cells = [plan.volume(v)["n_cells"] for v in range(len(vols))]
    return obin.bin_particles(vols, cells, info["sub_bits"], info["chunk_size"])


def oracle_force(vols, params):
    """FP64 accelerations and FP64-predicate counts, concatenated."""
    c = ofit.fit_poly(params["rc"], params["sigma"], params["eps"])
    out_a, out_c = [], []
    for pos, box in vols:
        a, n = oforce.accel_kdtree(pos, box, params["rc"], params["eps"], c)
        out_a.append(a)
        out_c.append(n)
    return np.concatenate(out_a), np.concatenate(out_c)


def to_np(t):
    return t.detach().cpu().numpy()
