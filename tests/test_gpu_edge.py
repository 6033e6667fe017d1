"""Degenerate inputs through every entry point: an empty particle set
(n = 0) for binning, forces (with and without the fused kick), pair counts,
the VJP, the invariants, the leapfrog and friends-of-friends; the PM side,
whose density contrast is undefined without particles, refuses it cleanly;
and a plan reused after an empty binning."""
import numpy as np
import pytest

from workloads import generators as gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_empty_short_range_step():
    from paper_1411_3396_b300 import Plan
    plan = Plan(16.0, 3.0, 0.1, 0.8, 1000)
    x = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    plan.bin(x)
    acc, pairs, pp = plan.force(count=True, per_particle=True)
    assert acc.shape == (0, 4) and int(pairs.item()) == 0 and pp.numel() == 0
    vel = torch.zeros((0, 4), dtype=torch.float32, device="cuda")
    plan.force_kick(torch.empty_like(vel), vel, 0.01)
    g = plan.vjp(torch.zeros((0, 4), dtype=torch.float32, device="cuda"))
    assert g.shape == (0, 4)
    inv = plan.invariants(vel, torch.empty_like(vel)).cpu().numpy()
    assert np.all(inv == 0.0)
    plan.leapfrog(x, vel, torch.empty_like(vel), 0.01, 2)
    torch.cuda.synchronize()
    # the same plan after an empty binning: a real set is exact again
    pos = gen.uniform_box(500, 16.0, 4)
    plan.bin(torch.from_numpy(pos).cuda())
    acc, pairs, _ = plan.force(count=True)
    torch.cuda.synchronize()
    assert int(pairs.item()) > 0 and torch.isfinite(acc).all()
    plan.close()


def test_empty_fof_and_pm():
    from paper_1411_3396_b300 import FOF, PM, Plan
    plan = Plan(16.0, 3.0, 0.1, 0.8, 100)
    x = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    plan.bin(x)
    f = FOF(100)
    lab, sizes = f.run(plan, x, 0.2, 2)
    info = f.info()
    assert lab.numel() == 0 and info["n_halos"] == 0 and info["links"] == 0
    f.close()
    # the density contrast of an empty set is undefined (mean density 0):
    # the PM calls refuse it with an argument error and stay usable
    from paper_1411_3396_b300 import SrError
    pm = PM(16, 16.0, 0.8, 100)
    with pytest.raises(SrError):
        pm.deposit(x)
    one = torch.from_numpy(np.array([[3.0, 4.0, 5.0]])).cuda()
    pm.deposit(one)
    k, pk, modes = pm.power()
    torch.cuda.synchronize()
    assert torch.isfinite(pk).all()
    pm.close()
    plan.close()


def test_host_step_submit_arguments_and_empty():
    # the pipelined host step: an empty step, a step above the capacity
    # (refused before any copy is enqueued), null buffers through the C ABI,
    # and a wait with nothing submitted
    import ctypes

    from paper_1411_3396_b300 import Plan
    from paper_1411_3396_b300._lib import SrError, load
    plan = Plan(16.0, 3.0, 0.1, 0.8, 1000)
    plan.step_host_wait()                               # nothing submitted: returns at once
    p0 = torch.zeros((0, 3), dtype=torch.float64).pin_memory()
    v0 = torch.zeros((0, 4), dtype=torch.float32).pin_memory()
    plan.step_host_submit(p0, v0, None, 0.01)
    plan.step_host_wait()
    plan.step_host(p0, v0, None, 0.01)                  # the synchronous form as well
    big = torch.zeros((1001, 3), dtype=torch.float64).pin_memory()
    vbig = torch.zeros((1001, 4), dtype=torch.float32).pin_memory()
    with pytest.raises(SrError) as e:
        plan.step_host_submit(big, vbig, None, 0.01)
    assert e.value.code == 3                            # SR_ERR_CAPACITY
    assert load().sr_step_host_submit(plan._h, None, None, None, ctypes.c_float(0.01), 10, None) == 1
    assert load().sr_step_host_wait(None) == 1
    # a real step after the refusals
    pos = torch.from_numpy(gen.uniform_box(500, 16.0, 5)).pin_memory()
    vel = torch.zeros((500, 4), dtype=torch.float32).pin_memory()
    acc = torch.zeros((500, 4), dtype=torch.float32).pin_memory()
    plan.step_host_submit(pos, vel, acc, 0.01)
    plan.step_host_wait()
    assert torch.isfinite(acc).all() and acc.abs().sum() > 0
    plan.close()
