"""Differentiable kick-drift trajectories through the short-range force.

``trajectory(plan, x0, v0, steps, dt)`` runs ``steps`` substeps of

    v_{k+1} = v_k + a(x_k) dt,     x_{k+1} = fold(x_k + v_{k+1} dt)

in the library's kernels (sr_bin, sr_force, sr_kick, sr_drift) and returns
(x_K, v_K).  Gradients flow to x0 and v0 through a hand-written reverse
sweep.  The force depends on the positions alone, so the sweep needs only
each substep's binning of x_k: with one plan, per-substep checkpointing
keeps x_k and the backward pass bins it again; with one plan per substep
(a sequence of ``steps`` plans), substep k's binning stays in plan k and
the backward pass reuses it (half the binnings, one plan's workspace per
substep).  The sweep applies, from the last substep to the first,

    vbar += dt * xbar                 (adjoint of the drift)
    xbar += (da/dx)^T (dt * vbar)     (adjoint of the kick, sr_force_vjp)

Both adjoint updates run in the library's kernels (sr_kick for the first,
sr_force_vjp with accumulation for the second).  Positions are binary64
(n, 3); velocities and all adjoints are binary32 float4 rows (n, 4).
"""
from __future__ import annotations

import torch

from .api import Plan, kick, launch_count


def _plans(plan, steps: int):
    """A tuple of one shared plan, or of one plan per substep."""
    if isinstance(plan, Plan):
        return (plan,)
    try:
        plans = tuple(plan)
    except TypeError:
        plans = ()
    if len(plans) != steps or not all(isinstance(p, Plan) for p in plans):
        raise ValueError("give one Plan, or a sequence of one Plan per substep")
    if len(plans) > 1 and len({id(p) for p in plans}) != len(plans):
        # a plan listed twice would hold only its last substep's binning when
        # the backward pass reads it for an earlier one
        raise ValueError("the per-substep plans must be distinct objects; give one Plan to share it")
    return plans


class _Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, plans, steps: int, dt: float):
        x = x0.detach().clone()
        v = v0.detach().clone()
        acc = torch.empty_like(v)
        shared = len(plans) == 1
        checkpoints = []
        for k in range(steps):
            plan = plans[0] if shared else plans[k]
            if shared:
                checkpoints.append(x.clone())
            plan.bin(x)
            plan.force(acc)
            kick(acc, v, dt)
            plan.drift(x, v, dt)
        ctx.save_for_backward(*checkpoints)
        ctx.plans, ctx.steps, ctx.dt = plans, steps, dt
        ctx.binnings = [p.binnings for p in plans]
        ctx.n, ctx.device = x0.shape[0], x0.device
        return x, v

    @staticmethod
    def backward(ctx, gx, gv):
        plans, steps, dt = ctx.plans, ctx.steps, ctx.dt
        checkpoints = ctx.saved_tensors
        shared = len(plans) == 1
        if not shared and [p.binnings for p in plans] != ctx.binnings:
            raise RuntimeError("a substep's plan was binned again between the forward and the backward pass")
        xbar = torch.zeros((ctx.n, 4), dtype=torch.float32, device=ctx.device)
        if gx is not None:
            xbar[:, :3] = gx.to(torch.float32)
        vbar = torch.zeros((ctx.n, 4), dtype=torch.float32, device=ctx.device)
        if gv is not None:
            vbar.copy_(gv.to(torch.float32))
        for k in range(steps - 1, -1, -1):
            kick(xbar, vbar, dt)                                   # vbar += dt * xbar
            if shared:
                plans[0].bin(checkpoints[k])
            plan = plans[0] if shared else plans[k]
            plan.vjp(vbar, xbar, g_scale=dt, accumulate=True)      # xbar += J^T (dt vbar)
        gx0 = xbar[:, :3].to(torch.float64)
        gv0 = vbar.clone()
        gv0[:, 3] = 0.0
        return gx0, gv0, None, None, None


def trajectory(plan, x0: torch.Tensor, v0: torch.Tensor, steps: int, dt: float):
    """(x_K, v_K) after ``steps`` kick-drift substeps; differentiable in x0, v0.

    ``plan`` is one Plan (binned again in the backward pass) or a sequence of
    ``steps`` Plans of the same parameters and kernel variant (substep k
    binned once, in plan k).  The gradients are the same bits either way."""
    steps = int(steps)
    return _Trajectory.apply(x0, v0, _plans(plan, steps), steps, float(dt))


class TrajectoryGraph:
    """A trajectory, a scalar loss on its end state and the gradient sweep,
    captured once in a CUDA graph and replayed.

    ``plan`` is one Plan or one per substep, as for ``trajectory``.
    ``loss_fn(x_K, v_K)`` returns a scalar tensor.  Each ``run(x0, v0)``
    copies the inputs into the graph's static buffers and replays the
    captured kernels (the same kernels in the same order as the eager
    ``trajectory`` plus ``torch.autograd.grad``, so the results are
    bit-identical to it) without the per-launch host work; it returns
    static tensors (loss, dloss/dx0 (n, 3) binary64, dloss/dv0 (n, 4)
    binary32) that the next ``run`` overwrites.  The library calls on the
    path are capture-safe: they neither allocate nor synchronise.
    """

    def __init__(self, plan, x0: torch.Tensor, v0: torch.Tensor, steps: int, dt: float, loss_fn,
                 warmup: int = 2):
        self.plan, self.steps, self.dt, self.loss_fn = plan, int(steps), float(dt), loss_fn
        self.x = x0.detach().clone().requires_grad_(True)
        self.v = v0.detach().clone().requires_grad_(True)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(max(1, int(warmup))):
                self._sweep()
        torch.cuda.current_stream().wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        k0 = launch_count()
        with torch.cuda.graph(self.graph):
            self.loss, self.gx, self.gv = self._sweep()
        self.kernels = launch_count() - k0          # library kernels in one replay

    def _sweep(self):
        xk, vk = trajectory(self.plan, self.x, self.v, self.steps, self.dt)
        loss = self.loss_fn(xk, vk)
        gx, gv = torch.autograd.grad(loss, (self.x, self.v))
        return loss.detach(), gx, gv

    def run(self, x0: torch.Tensor | None = None, v0: torch.Tensor | None = None):
        with torch.no_grad():
            if x0 is not None:
                self.x.copy_(x0)
            if v0 is not None:
                self.v.copy_(v0)
        self.graph.replay()
        return self.loss, self.gx, self.gv
