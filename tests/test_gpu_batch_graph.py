"""Batched sub-volumes in one persistent launch, CUDA-graph capture and
replay, kick / drift / invariants against plain definitions."""
import numpy as np
import pytest

from oracle import binning as obin
from oracle import integrate as oint
from workloads import configs as wc
from workloads import generators as gen

from helpers import assert_force_close, make_plan, oracle_force, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("chunk", [32, 64])
def test_batch_equals_individual_plans(chunk):
    w = wc.make_workload(wc.small_variant("batch64"))
    vols, prm = w["volumes"], w["params"]
    pos = np.concatenate([p for p, _ in vols])
    plan = make_plan(vols, prm, chunk_size=chunk)
    plan.bin(torch.from_numpy(pos).cuda())
    acc = to_np(plan.force())
    k = 0
    for p, box in vols:
        single = make_plan([(p, box)], prm, chunk_size=chunk)
        single.bin(torch.from_numpy(p).cuda())
        a1 = to_np(single.force())
        assert a1.tobytes() == acc[k:k + len(p)].tobytes()
        k += len(p)


def _refresh(dst, src):
    dst.copy_(src)


def test_graph_replay_equals_eager():
    w = wc.make_workload(wc.small_variant("clustered256"))
    (pos, box), = w["volumes"]
    prm = w["params"]
    n = len(pos)
    x = torch.from_numpy(pos).cuda()
    v0 = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    v0[:, :3] = torch.from_numpy(w["velocities"]).float()
    eager = make_plan(w["volumes"], prm)
    ve = v0.clone()
    ae = torch.empty_like(ve)
    eager.bin(x)
    eager.force(ae)
    from paper_1411_3396_b300 import kick
    kick(ae, ve, prm["dt"])
    plan = make_plan(w["volumes"], prm)
    xg = x.clone()
    vg = v0.clone()
    ag = torch.zeros_like(vg)
    from paper_1411_3396_b300 import launch_count
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        k0 = launch_count()
        plan.graph_capture(xg, vg, ag, prm["dt"])
        assert launch_count() == k0                          # captured kernels count when replayed
        assert float(ag.abs().sum().item()) == 0.0          # capture ran nothing
        k1 = launch_count()
        plan.graph_launch()
        per_replay = launch_count() - k1
        assert per_replay >= 8                               # binning passes + the force kernel
        for _ in range(3):
            vg.copy_(v0)
            plan.graph_launch()
        assert launch_count() - k1 == 4 * per_replay
    torch.cuda.synchronize()
    assert to_np(ag).tobytes() == to_np(ae).tobytes()
    assert to_np(vg).tobytes() == to_np(ve).tobytes()


def test_graph_capture_rejects_default_stream():
    from paper_1411_3396_b300 import SrError
    pos = gen.uniform_box(100, 16.0, 1)
    plan = make_plan([(pos, 16.0)], dict(rc=3.0, eps=0.1, sigma=0.8))
    x = torch.from_numpy(pos).cuda()
    v = torch.zeros((100, 4), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(torch.cuda.default_stream()):
        with pytest.raises(SrError):
            plan.graph_capture(x, v, torch.empty_like(v), 0.01)
    with pytest.raises(SrError):
        plan.graph_launch()


def test_kick_drift_invariants():
    from paper_1411_3396_b300 import kick
    rng = np.random.default_rng(9)
    n, L = 5000, 16.0
    a = rng.standard_normal((n, 4)).astype(np.float32)
    v = rng.standard_normal((n, 4)).astype(np.float32)
    at, vt = torch.from_numpy(a).cuda(), torch.from_numpy(v).cuda()
    kick(at, vt, 0.01)
    vk = to_np(vt)
    ref = (v[:, :3].astype(np.float64) + a[:, :3].astype(np.float64) * np.float32(0.01))
    np.testing.assert_allclose(vk[:, :3], ref, rtol=1e-6, atol=1e-7)
    np.testing.assert_array_equal(vk[:, 3], v[:, 3])
    pos = gen.uniform_box(n, L, 2)
    plan = make_plan([(pos, L)], dict(rc=3.0, eps=0.1, sigma=0.8))
    xt = torch.from_numpy(pos).cuda()
    plan.drift(xt, vt, 0.5)
    xd = to_np(xt)
    ref = obin.wrap_positions(pos + vk[:, :3].astype(np.float64) * 0.5, L)
    np.testing.assert_array_equal(xd, ref)
    inv = to_np(plan.invariants(vt, at))
    o = oint.invariants(vk[:, :3], a[:, :3])
    np.testing.assert_allclose(inv[0:3], o["momentum"], rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(inv[3:6], o["net_force"], rtol=1e-12, atol=1e-9)
    assert inv[6] == pytest.approx(o["kinetic"], rel=1e-12)
    # deterministic
    inv2 = to_np(plan.invariants(vt, at))
    assert inv.tobytes() == inv2.tobytes()


def test_step_host_matches_device_path():
    w = wc.make_workload(wc.small_variant("zeldovich128"))
    (pos, box), = w["volumes"]
    prm = w["params"]
    n = len(pos)
    v0 = np.zeros((n, 4), np.float32)
    v0[:, :3] = w["velocities"]
    plan = make_plan(w["volumes"], prm)
    vh = torch.from_numpy(v0.copy()).pin_memory()
    ah = torch.empty((n, 4), dtype=torch.float32).pin_memory()
    dev = make_plan(w["volumes"], prm)
    vd = torch.from_numpy(v0.copy()).cuda()
    from paper_1411_3396_b300 import kick
    # two consecutive steps (the second from moved positions): the side-stream
    # velocity upload must see the first step's kicked velocities
    for step in range(2):
        p = pos if step == 0 else np.mod(pos + 0.3 * v0[:, :3].astype(np.float64), box)
        plan.step_host(torch.from_numpy(p).pin_memory(), vh, ah, prm["dt"])
        dev.bin(torch.from_numpy(p).cuda())
        acc = dev.force()
        kick(acc, vd, prm["dt"])
        assert ah.numpy().tobytes() == to_np(acc).tobytes()
        assert vh.numpy().tobytes() == to_np(vd).tobytes()


def test_step_host_submit_pipelined_matches_step_host():
    # five independent inputs (distinct positions and velocities) submitted
    # back to back with their own page-locked buffers: up to two steps in
    # flight on the two staging sets; every step's accelerations and kicked
    # velocities equal the synchronous sr_step_host's bit for bit, also for
    # a step submitted without an acceleration buffer
    w = wc.make_workload(wc.small_variant("zeldovich128"))
    (pos, box), = w["volumes"]
    prm = w["params"]
    n = len(pos)
    rng = np.random.default_rng(7)
    inputs = []
    for k in range(5):
        p = np.mod(pos + rng.normal(0.0, 0.2 * k, pos.shape), box)
        v = np.zeros((n, 4), np.float32)
        v[:, :3] = rng.normal(0.0, 1.0, (n, 3))
        inputs.append((p, v))
    ref = make_plan(w["volumes"], prm)
    expect = []
    for p, v in inputs:
        vh = torch.from_numpy(v.copy()).pin_memory()
        ah = torch.empty((n, 4), dtype=torch.float32).pin_memory()
        ref.step_host(torch.from_numpy(p).pin_memory(), vh, ah, prm["dt"])
        expect.append((ah.numpy().copy(), vh.numpy().copy()))
    plan = make_plan(w["volumes"], prm)
    bufs = [(torch.from_numpy(p).pin_memory(), torch.from_numpy(v.copy()).pin_memory(),
             torch.full((n, 4), np.nan, dtype=torch.float32).pin_memory()) for p, v in inputs]
    for k, (ph, vh, ah) in enumerate(bufs):
        plan.step_host_submit(ph, vh, None if k == 3 else ah, prm["dt"])
    plan.step_host_wait()
    for k, ((_, vh, ah), (a_ref, v_ref)) in enumerate(zip(bufs, expect)):
        assert vh.numpy().tobytes() == v_ref.tobytes(), k
        if k == 3:
            assert np.isnan(ah.numpy()).all()
        else:
            assert ah.numpy().tobytes() == a_ref.tobytes(), k
    # a second round on the same plan after the wait reuses the staging sets
    ph, vh, ah = bufs[0]
    vh.copy_(torch.from_numpy(inputs[0][1]))
    plan.step_host_submit(ph, vh, ah, prm["dt"])
    plan.step_host_wait()
    assert vh.numpy().tobytes() == expect[0][1].tobytes()
    assert ah.numpy().tobytes() == expect[0][0].tobytes()
    plan.status()


def test_batch_full_size_graph_and_sampled_oracle():
    # the 64-volume batched workload under one captured graph; rows of a few
    # volumes checked against the oracle
    w = wc.make_workload(wc.CONFIGS["batch64"])
    vols, prm = w["volumes"], w["params"]
    pos = np.concatenate([p for p, _ in vols])
    n = len(pos)
    plan = make_plan(vols, prm)
    x = torch.from_numpy(pos).cuda()
    v = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    a = torch.zeros_like(v)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.graph_capture(x, v, a, prm["dt"])
        plan.graph_launch()
    torch.cuda.synchronize()
    acc = to_np(a)
    eager = make_plan(vols, prm)
    eager.bin(x)
    assert to_np(eager.force()).tobytes() == acc.tobytes()
    k = 0
    sizes = [len(p) for p, _ in vols]
    pick = {int(np.argmin(sizes)), int(np.argmax(sizes)), 7}
    for i, (p, box) in enumerate(vols):
        if i in pick:
            a_ref, _ = oracle_force([(p, box)], prm)
            assert_force_close(acc[k:k + len(p)], a_ref, f"volume {i}")
        k += len(p)
