"""Kick, drift, the kick-drift trajectory and its FP64 reverse mode, and a
kick-drift-kick leapfrog stepper.

The paper's short-range timestep (Sec. 2.1) ends with the particles updated
by the short-range force; the update is the kick v += a dt.  The
differentiable workload chains K substeps of symplectic Euler

    v_{k+1} = v_k + a(x_k) dt,     x_{k+1} = wrap(x_k + v_{k+1} dt),

with loss L = sum_i |minimg(x_K,i - x_target,i)|^2, and needs dL/dx_0 and
dL/dv_0.  The reverse mode is written by hand from the chain rule; its only
non-trivial piece is the vector-Jacobian product of the short-range force,
in gather form (each particle collects from its neighbours, no scatter):

    xbar_i = sum_j [ f(s) (g_j - g_i) + 2 f'(s) (d . (g_j - g_i)) d ],   d = x_j - x_i,

for a cotangent g on the accelerations.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from .fit import df_sr, f_sr
from .force import _wrap_for_tree, accel_kdtree, min_image


def kick(v, a, dt):
    return np.asarray(v, np.float64) + np.asarray(a, np.float64) * dt


def drift(x, v, dt, box):
    return _wrap_for_tree(np.asarray(x, np.float64) + np.asarray(v, np.float64) * dt, box)


def force_vjp(pos, box, rc, eps, c, gbar, absolute=False):
    """xbar = (da/dx)^T gbar for the short-range accelerations.  With
    absolute, also the per-row sums of the terms' magnitudes, sum_j |w_ij|
    per axis (the scale of the rounding error of any evaluation of the sum
    in finite precision)."""
    pos = _wrap_for_tree(pos, box)
    gbar = np.asarray(gbar, np.float64)
    n = len(pos)
    tree = cKDTree(pos, boxsize=box)
    pr = tree.query_pairs(rc, output_type="ndarray")
    i, j = pr[:, 0], pr[:, 1]
    d = min_image(pos[j] - pos[i], box)
    s = np.sum(d * d, axis=1)
    keep = s < rc * rc
    i, j, d, s = i[keep], j[keep], d[keep], s[keep]
    dg = gbar[j] - gbar[i]
    w = f_sr(s, eps, c)[:, None] * dg + \
        (2.0 * df_sr(s, eps, c) * np.sum(d * dg, axis=1))[:, None] * d
    out = np.zeros((n, 3))
    for ax in range(3):
        out[:, ax] = np.bincount(i, weights=w[:, ax], minlength=n) - \
            np.bincount(j, weights=w[:, ax], minlength=n)
    if not absolute:
        return out
    mag = np.zeros((n, 3))
    for ax in range(3):
        aw = np.abs(w[:, ax])
        mag[:, ax] = np.bincount(i, weights=aw, minlength=n) + np.bincount(j, weights=aw, minlength=n)
    return out, mag


def trajectory(x0, v0, box, rc, eps, c, dt, steps, accel=None):
    """Run K kick-drift substeps; returns the lists of x_k and v_k."""
    accel = accel or (lambda x: accel_kdtree(x, box, rc, eps, c)[0])
    xs = [_wrap_for_tree(x0, box)]
    vs = [np.asarray(v0, np.float64).copy()]
    for _ in range(steps):
        a = accel(xs[-1])
        v = kick(vs[-1], a, dt)
        xs.append(drift(xs[-1], v, dt, box))
        vs.append(v)
    return xs, vs


def loss(x_final, x_target, box):
    d = min_image(np.asarray(x_final, np.float64) - np.asarray(x_target, np.float64), box)
    return float(np.sum(d * d))


def loss_and_grad(x0, v0, x_target, box, rc, eps, c, dt, steps):
    """Loss and (dL/dx0, dL/dv0) by hand-written reverse mode."""
    xs, vs = trajectory(x0, v0, box, rc, eps, c, dt, steps)
    L = loss(xs[-1], x_target, box)
    xbar = 2.0 * min_image(xs[-1] - np.asarray(x_target, np.float64), box)
    vbar = np.zeros_like(xbar)
    for k in range(steps - 1, -1, -1):
        vbar = vbar + dt * xbar                         # x_{k+1} = x_k + v_{k+1} dt
        xbar = xbar + force_vjp(xs[k], box, rc, eps, c, dt * vbar)   # v_{k+1} = v_k + a(x_k) dt
    return L, xbar, vbar


def leapfrog(x0, v0, box, rc, eps, c, dt, steps, a0=None):
    """Kick-drift-kick leapfrog: per step v += a dt/2; x = fold(x + v dt);
    a = a(x); v += a dt/2.  Returns (x_K, v_K, a_K)."""
    x = _wrap_for_tree(x0, box)
    v = np.asarray(v0, np.float64).copy()
    a = accel_kdtree(x, box, rc, eps, c)[0] if a0 is None else np.asarray(a0, np.float64)
    for _ in range(steps):
        v = kick(v, a, 0.5 * dt)
        x = drift(x, v, dt, box)
        a = accel_kdtree(x, box, rc, eps, c)[0]
        v = kick(v, a, 0.5 * dt)
    return x, v, a


def invariants(v, a):
    """FP64 momentum sum(v), net force sum(a) and kinetic energy (unit masses)."""
    v = np.asarray(v, np.float64)
    a = np.asarray(a, np.float64)
    return dict(momentum=v.sum(axis=0), net_force=a.sum(axis=0),
                kinetic=0.5 * float(np.sum(v * v)))
