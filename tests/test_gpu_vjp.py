"""sr_force_vjp and the differentiable trajectory against the FP64 oracle's
reverse mode and FP64 finite differences."""
import numpy as np
import pytest

from oracle import fit as ofit
from oracle import force as oforce
from oracle import integrate as oint
from workloads import configs as wc
from workloads import generators as gen

from helpers import assert_force_close, make_plan, rel_errors, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _g(n, seed):
    g = np.zeros((n, 4), np.float32)
    g[:, :3] = np.random.default_rng(seed).standard_normal((n, 3))
    return g


@pytest.mark.parametrize("chunk", [32, 64])
@pytest.mark.parametrize("name", ["uniform4k", "diff64", "clustered256"])
def test_vjp_matches_oracle(name, chunk):
    w = wc.make_workload(wc.small_variant(name))
    (pos, box), = w["volumes"]
    prm = w["params"]
    plan = make_plan(w["volumes"], prm, chunk_size=chunk)
    plan.bin(torch.from_numpy(pos).cuda())
    g = _g(len(pos), 3)
    xbar = to_np(plan.vjp(torch.from_numpy(g).cuda()))
    c = ofit.fit_poly(prm["rc"], prm["sigma"], prm["eps"])
    ref = oint.force_vjp(pos, box, prm["rc"], prm["eps"], c, g[:, :3].astype(np.float64))
    assert_force_close(xbar, ref, f"vjp {name}")


@pytest.mark.parametrize("chunk", [32, 64])
def test_vjp_on_a_batch_plan(chunk):
    # a batch of independent volumes (per-item constants in the packed loop):
    # each volume's rows against the oracle's VJP of that volume alone
    w = wc.make_workload(wc.small_variant("batch64"))
    vols, prm = w["volumes"], w["params"]
    pos = np.concatenate([p for p, _ in vols])
    plan = make_plan(vols, prm, chunk_size=chunk)
    plan.bin(torch.from_numpy(pos).cuda())
    g = _g(len(pos), 11)
    xbar = to_np(plan.vjp(torch.from_numpy(g).cuda()))
    c = ofit.fit_poly(prm["rc"], prm["sigma"], prm["eps"])
    off = 0
    for p, box in vols:
        n = len(p)
        ref = oint.force_vjp(p, box, prm["rc"], prm["eps"], c, g[off:off + n, :3].astype(np.float64))
        assert_force_close(xbar[off:off + n], ref, f"vjp batch volume of {n}")
        off += n


@pytest.mark.parametrize("name", ["diff64", "clustered256"])
def test_vjp_follows_the_force_variant(name):
    # the VJP follows the selected force variant: the flat neighbour
    # enumeration with 13-16 (the same chunks in the same order, so the same
    # bits as cell by cell) and packed batches of 64 with 12 and 14-16
    # (else 128); both batch sizes meet the oracle bar
    prm_w = wc.make_workload(wc.small_variant(name))
    (pos, box), = prm_w["volumes"]
    prm = prm_w["params"]
    plan = make_plan(prm_w["volumes"], prm)
    plan.bin(torch.from_numpy(pos).cuda())
    g = torch.from_numpy(_g(len(pos), 5)).cuda()
    plan.set_variant(11)
    a128 = to_np(plan.vjp(g))
    plan.set_variant(13)
    assert to_np(plan.vjp(g)).tobytes() == a128.tobytes(), "variant 13"
    plan.set_variant(12)
    a64 = to_np(plan.vjp(g))
    for v in (14, 15, 16):
        plan.set_variant(v)
        assert to_np(plan.vjp(g)).tobytes() == a64.tobytes(), f"variant {v}"
    c = ofit.fit_poly(prm["rc"], prm["sigma"], prm["eps"])
    ref = oint.force_vjp(pos, box, prm["rc"], prm["eps"], c, g.cpu().numpy()[:, :3].astype(np.float64))
    assert_force_close(a128, ref, f"vjp {name} batches of 128")
    assert_force_close(a64, ref, f"vjp {name} batches of 64")


def test_vjp_scale_and_accumulate():
    w = wc.make_workload(wc.small_variant("uniform4k"))
    (pos, box), = w["volumes"]
    plan = make_plan(w["volumes"], w["params"])
    plan.bin(torch.from_numpy(pos).cuda())
    g = torch.from_numpy(_g(len(pos), 4)).cuda()
    base = plan.vjp(g)
    out = torch.ones_like(base)
    plan.vjp(g, out, g_scale=0.5, accumulate=True)
    half = plan.vjp(g, g_scale=0.5)
    np.testing.assert_allclose(to_np(out)[:, :3], 1.0 + to_np(half)[:, :3], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(to_np(half), 0.5 * to_np(base), rtol=1e-6, atol=1e-7)


def _diff_setup(n_side, box):
    x0, psi = gen.zeldovich(n_side, box, 0.5, 1004)
    xt, _ = gen.zeldovich(n_side, box, 0.5, 1005)
    v0 = 0.1 * psi
    return x0, v0, xt


def _gpu_loss_grad(x0, v0, xt, box, prm, steps, dt):
    from paper_1411_3396_b300 import Plan, trajectory
    plan = Plan(box, prm["rc"], prm["eps"], prm["sigma"], len(x0))
    x = torch.from_numpy(x0).cuda().requires_grad_(True)
    v = torch.zeros((len(x0), 4), dtype=torch.float32, device="cuda")
    v[:, :3] = torch.from_numpy(v0).float()
    v.requires_grad_(True)
    xk, vk = trajectory(plan, x, v, steps, dt)
    d = xk - torch.from_numpy(xt).cuda()
    d = d - box * torch.round(d / box)
    loss = (d * d).sum()
    loss.backward()
    return float(loss.item()), to_np(x.grad), to_np(v.grad)[:, :3], to_np(xk)


def test_trajectory_gradients_match_oracle_reverse_mode():
    cfg = wc.small_variant("diff64")
    box, n_side, steps, dt = cfg["box"], cfg["n_side"], cfg["steps"], cfg["dt"]
    prm = dict(rc=cfg["rc"], eps=cfg["eps"], sigma=cfg["sigma"])
    x0, v0, xt = _diff_setup(n_side, box)
    L, gx, gv, xk = _gpu_loss_grad(x0, v0, xt, box, prm, steps, dt)
    c = ofit.fit_poly(prm["rc"], prm["sigma"], prm["eps"])
    Lr, gxr, gvr = oint.loss_and_grad(x0, v0, xt, box, prm["rc"], prm["eps"], c, dt, steps)
    xs, _ = oint.trajectory(x0, v0, box, prm["rc"], prm["eps"], c, dt, steps)
    assert np.max(np.abs(oforce.min_image(xk - xs[-1], box))) < 1e-5
    assert L == pytest.approx(Lr, rel=1e-5)
    rx = rel_errors(gx, gxr)
    rv = rel_errors(gv, gvr)
    assert np.median(rx) <= 1e-5 and rx.max() <= 1e-4, (np.median(rx), rx.max())
    assert np.median(rv) <= 1e-5 and rv.max() <= 1e-4, (np.median(rv), rv.max())


def test_trajectory_gradient_against_fp64_finite_differences():
    # FD of the FP64 oracle loss along random directions and single
    # coordinates, compared with the GPU gradient (16^3 instance)
    cfg = wc.small_variant("diff64")
    box, n_side, steps, dt = cfg["box"], cfg["n_side"], cfg["steps"], cfg["dt"]
    prm = dict(rc=cfg["rc"], eps=cfg["eps"], sigma=cfg["sigma"])
    x0, v0, xt = _diff_setup(n_side, box)
    _, gx, gv, _ = _gpu_loss_grad(x0, v0, xt, box, prm, steps, dt)
    c = ofit.fit_poly(prm["rc"], prm["sigma"], prm["eps"])

    def lossf(x, v):
        xs, _ = oint.trajectory(x, v, box, prm["rc"], prm["eps"], c, dt, steps)
        return oint.loss(xs[-1], xt, box)

    rng = np.random.default_rng(5)
    h = 1e-6
    n = len(x0)
    for _ in range(6):
        ex = rng.standard_normal((n, 3)); ex /= np.linalg.norm(ex)
        ev = rng.standard_normal((n, 3)); ev /= np.linalg.norm(ev)
        fd = (lossf(x0 + h * ex, v0 + h * ev) - lossf(x0 - h * ex, v0 - h * ev)) / (2 * h)
        an = float(np.sum(gx * ex) + np.sum(gv * ev))
        assert an == pytest.approx(fd, rel=1e-4, abs=1e-6)
    for _ in range(6):
        i, ax = rng.integers(n), rng.integers(3)
        e = np.zeros((n, 3)); e[i, ax] = 1.0
        fd = (lossf(x0 + h * e, v0) - lossf(x0 - h * e, v0)) / (2 * h)
        assert gx[i, ax] == pytest.approx(fd, rel=1e-4, abs=1e-6)


def test_trajectory_full_size_64cubed():
    cfg = wc.CONFIGS["diff64"]
    box, n_side, steps, dt = cfg["box"], cfg["n_side"], cfg["steps"], cfg["dt"]
    prm = dict(rc=cfg["rc"], eps=cfg["eps"], sigma=cfg["sigma"])
    x0, v0, xt = _diff_setup(n_side, box)
    L, gx, gv, _ = _gpu_loss_grad(x0, v0, xt, box, prm, steps, dt)
    c = ofit.fit_poly(prm["rc"], prm["sigma"], prm["eps"])
    Lr, gxr, gvr = oint.loss_and_grad(x0, v0, xt, box, prm["rc"], prm["eps"], c, dt, steps)
    assert L == pytest.approx(Lr, rel=1e-5)
    # gradient tolerance after 10 binary32 substeps: per-particle median
    # 1e-5, normwise 1e-4, per-particle max 1e-3 (close encounters amplify
    # the binary32 forward-state differences of a few particles)
    for g, r in ((gx, gxr), (gv, gvr)):
        rel = rel_errors(g, r)
        norm = np.linalg.norm(g - r) / np.linalg.norm(r)
        assert np.median(rel) <= 1e-5 and norm <= 1e-4 and rel.max() <= 1e-3, \
            (np.median(rel), norm, rel.max())


def _rows_straddling_the_cutoff(x, box, rc, rel=5e-6):
    """Rows with a neighbour at a distance within rel of r_c.  The force is
    continuous at r_c but its derivative is not (f(r_c^2) = 0, f'(r_c^2) !=
    0), so the VJP of such a pair jumps by a term of its own size where the
    binary32 predicate of the kernel and the FP64 one of the oracle decide
    on different sides.  The kernel's distance differs from the FP64 one by
    at most about 1.3e-6 relative near r_c: half an ulp of each binary32
    offset (|offset| < 2^7 units of h) and of the shifted neighbour
    coordinate (< 2^8 units) per axis, and the fused s' chain."""
    from scipy.spatial import cKDTree
    t = cKDTree(np.mod(x, box), boxsize=box)
    hi = t.query_ball_point(np.mod(x, box), rc * (1 + rel), return_length=True)
    lo = t.query_ball_point(np.mod(x, box), rc * (1 - rel), return_length=True)
    return hi > lo


def test_vjp_per_substep_on_gpu_states_64cubed():
    # separates the VJP kernel's own error from trajectory divergence at full
    # size: each substep's GPU VJP is compared, at the force bar, with the
    # oracle's VJP at the GPU's own state x_k and the GPU's own cotangent
    # (the binary32 dt * vbar the kernel applies); the end-to-end bar of
    # test_trajectory_full_size_64cubed covers the whole trajectory.  Rows
    # with a pair straddling r_c (about a thousand of 262,144) are left out:
    # there the VJP has a jump of the size of one pair term.  The rest meet
    # the force bar (median 1e-5, and 1e-4 per row) except where a row's sum
    # cancels: binary32 partial sums of up to 64 terms carry an error of a
    # few 1e-7 of the terms' magnitude, so a row may instead stay within
    # 1e-5 of its sum of term magnitudes (the oracle's absolute sums)
    from paper_1411_3396_b300 import Plan, kick
    cfg = wc.CONFIGS["diff64"]
    box, n_side, steps, dt = cfg["box"], cfg["n_side"], cfg["steps"], cfg["dt"]
    rc, eps, sigma = cfg["rc"], cfg["eps"], cfg["sigma"]
    x0, v0, xt = _diff_setup(n_side, box)
    n = len(x0)
    plan = Plan(box, rc, eps, sigma, n)
    x = torch.from_numpy(x0).cuda()
    v = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    v[:, :3] = torch.from_numpy(v0).float()
    acc = torch.empty_like(v)
    states = []
    for _ in range(steps):                   # the forward substeps, checkpointing x_k
        states.append(x.clone())
        plan.bin(x)
        plan.force(acc)
        kick(acc, v, dt)
        plan.drift(x, v, dt)
    d = x - torch.from_numpy(xt).cuda()
    d = d - box * torch.round(d / box)
    xbar = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    xbar[:, :3] = (2.0 * d).float()
    vbar = torch.zeros_like(xbar)
    c = ofit.fit_poly(rc, sigma, eps)
    for k in range(steps - 1, -1, -1):       # the reverse sweep, one substep at a time
        kick(xbar, vbar, dt)                 # vbar += dt * xbar
        plan.bin(states[k])
        out = plan.vjp(vbar, g_scale=dt)
        g = (to_np(vbar)[:, :3] * np.float32(dt)).astype(np.float64)
        xk = to_np(states[k])
        ref, mag = oint.force_vjp(xk, box, rc, eps, c, g, absolute=True)
        edge = _rows_straddling_the_cutoff(xk, box, rc)
        assert edge.sum() <= 1e-2 * n, edge.sum()
        got = to_np(out)[~edge, :3]
        ref, mag = ref[~edge], mag[~edge]
        rel = rel_errors(got, ref)
        err = np.linalg.norm(got - ref, axis=1)
        cond = err / np.linalg.norm(mag, axis=1)
        assert np.median(rel) <= 1e-5, (k, np.median(rel))
        assert np.all((rel <= 1e-4) | (cond <= 1e-5)), (k, rel.max(), cond[rel > 1e-4].max())
        xbar += out


def test_trajectory_graph_is_bit_identical_to_eager():
    # the captured forward + loss + gradient sweep replays the eager kernels
    from paper_1411_3396_b300 import TrajectoryGraph, trajectory
    w = wc.make_workload(wc.small_variant("diff64"))
    (pos, box), = w["volumes"]
    prm = w["params"]
    plan = make_plan(w["volumes"], prm)
    n = len(pos)
    rng = np.random.default_rng(8)
    target = torch.from_numpy(np.mod(pos + rng.normal(0, 0.2, pos.shape), box)).cuda()

    def loss_fn(xk, vk):
        d = xk - target
        d = d - box * torch.round(d / box)
        return (d * d).sum() + 0.5 * (vk[:, :3].double() ** 2).sum()

    def eager(x0, v0):
        x = x0.clone().requires_grad_(True)
        v = v0.clone().requires_grad_(True)
        xk, vk = trajectory(plan, x, v, 4, prm["dt"])
        loss = loss_fn(xk, vk)
        gx, gv = torch.autograd.grad(loss, (x, v))
        return loss.detach(), gx, gv

    x0 = torch.from_numpy(pos).cuda()
    v0 = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    v0[:, :3] = torch.from_numpy(rng.normal(0, 0.3, (n, 3))).float().cuda()
    g = TrajectoryGraph(plan, x0, v0, 4, prm["dt"], loss_fn)
    for trial in range(2):
        if trial:
            x0 = torch.from_numpy(np.mod(pos + rng.normal(0, 0.05, pos.shape), box)).cuda()
            v0 = v0 * 0.5
        ref = eager(x0, v0)
        got = g.run(x0, v0)
        torch.cuda.synchronize()
        for a, b in zip(got, ref):
            assert torch.equal(a, b)


def test_per_substep_plans_give_the_shared_plans_bits():
    # one plan per substep keeps each substep's binning for the backward
    # sweep instead of binning it again: the same gradients, eager and
    # replayed in a graph, with fewer kernels per replay
    from paper_1411_3396_b300 import TrajectoryGraph, trajectory
    w = wc.make_workload(wc.small_variant("diff64"))
    (pos, box), = w["volumes"]
    prm = w["params"]
    steps, dt = 4, prm["dt"]
    shared = make_plan(w["volumes"], prm)
    per = [make_plan(w["volumes"], prm) for _ in range(steps)]
    n = len(pos)
    rng = np.random.default_rng(21)
    target = torch.from_numpy(np.mod(pos + rng.normal(0, 0.2, pos.shape), box)).cuda()

    def loss_fn(xk, vk):
        d = xk - target
        d = d - box * torch.round(d / box)
        return (d * d).sum() + 0.5 * (vk[:, :3].double() ** 2).sum()

    def grads(plans, x0, v0):
        x = x0.clone().requires_grad_(True)
        v = v0.clone().requires_grad_(True)
        xk, vk = trajectory(plans, x, v, steps, dt)
        loss = loss_fn(xk, vk)
        gx, gv = torch.autograd.grad(loss, (x, v))
        return loss.detach(), gx, gv, xk.detach(), vk.detach()

    x0 = torch.from_numpy(pos).cuda()
    v0 = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    v0[:, :3] = torch.from_numpy(rng.normal(0, 0.3, (n, 3))).float().cuda()
    ref = grads(shared, x0, v0)
    got = grads(per, x0, v0)
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    g_per = TrajectoryGraph(per, x0, v0, steps, dt, loss_fn)
    g_shared = TrajectoryGraph(shared, x0, v0, steps, dt, loss_fn)
    for a, b in zip(g_per.run(x0, v0), ref[:3]):
        assert torch.equal(a, b)
    assert g_per.kernels < g_shared.kernels
    # a plan binned again between the passes is refused, as is a plan list
    # of the wrong length
    x = x0.clone().requires_grad_(True)
    v = v0.clone().requires_grad_(True)
    xk, vk = trajectory(per, x, v, steps, dt)
    per[1].bin(x0)
    with pytest.raises(RuntimeError):
        torch.autograd.grad(loss_fn(xk, vk), (x, v))
    with pytest.raises(ValueError):
        trajectory(per[:2], x, v, steps, dt)
