"""sr_force / sr_force_plain against the FP64 oracle: element-by-element
forces within tolerance, bit-exact pair counts, determinism, invariants."""
import numpy as np
import pytest

from oracle import binning as obin
from oracle import fit as ofit
from oracle import force as oforce
from workloads import configs as wc
from workloads import generators as gen

from helpers import assert_force_close, make_plan, oracle_binning, oracle_force, rel_errors, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SMALL = ["uniform4k", "zeldovich128", "clustered256", "batch64", "diff64"]


def _gpu(vols, params, count=True, **kw):
    pos = np.concatenate([p for p, _ in vols])
    plan = make_plan(vols, params, **kw)
    plan.bin(torch.from_numpy(pos).cuda())
    if count:
        acc, pairs, pp = plan.force(count=True, per_particle=True)
        torch.cuda.synchronize()
        return plan, to_np(acc), int(pairs.item()), to_np(pp)
    acc = plan.force()
    torch.cuda.synchronize()
    return plan, to_np(acc), None, None


_WORK = {}


def _work(name):
    if name not in _WORK:
        _WORK[name] = wc.make_workload(wc.small_variant(name))
    return _WORK[name]


@pytest.fixture(scope="module", params=[(n, c) for n in SMALL for c in (32, 64)],
                ids=lambda p: f"{p[0]}-c{p[1]}")
def small_case(request):
    name, chunk = request.param
    return name, _work(name), chunk


def test_force_matches_oracle(small_case):
    name, w, chunk = small_case
    plan, acc, pairs, pp = _gpu(w["volumes"], w["params"], chunk_size=chunk)
    a_ref, _ = oracle_force(w["volumes"], w["params"])
    assert_force_close(acc, a_ref, name)
    assert np.all(acc[:, 3] == 0)


def test_force_matches_oracle_on_dequantised_positions(small_case):
    # the kernel arithmetic alone (same binary32 inputs as the GPU)
    name, w, chunk = small_case
    plan, acc, _, _ = _gpu(w["volumes"], w["params"], count=False, chunk_size=chunk)
    B = oracle_binning(plan, w["volumes"])
    xr = obin.dequantized_positions(B, w["volumes"])
    vols_r, k = [], 0
    for pos, box in w["volumes"]:
        vols_r.append((xr[k:k + len(pos)], box))
        k += len(pos)
    a_ref, _ = oracle_force(vols_r, w["params"])
    rel = rel_errors(acc, a_ref)
    assert np.median(rel) <= 1e-5 and rel.max() <= 1e-4, (np.median(rel), rel.max())


def test_pair_counts_bit_exact(small_case):
    name, w, chunk = small_case
    plan, acc, pairs, pp = _gpu(w["volumes"], w["params"], chunk_size=chunk)
    B = oracle_binning(plan, w["volumes"])
    ref = oforce.pair_counts_fp32(B, w["volumes"], w["params"]["rc"], w["params"]["eps"])
    np.testing.assert_array_equal(pp, ref)
    assert pairs == int(ref.sum())


def test_all_kernel_variants_give_identical_forces(small_case):
    # variants 0-6 share the summation order of the counting kernel; the
    # packed two-wide variants 8-11 share theirs (batches of 128 neighbours,
    # even and odd entries apart) and agree bit for bit; 7 (scalar split
    # sums, batches of 32), 12 (packed, batches of 64) and all of them agree
    # with the oracle
    from paper_1411_3396_b300 import SrError
    name, w, chunk = small_case
    plan, acc_c, _, _ = _gpu(w["volumes"], w["params"], count=True, chunk_size=chunk)
    ref = acc_c.tobytes()
    first = range(7) if chunk == 32 else range(4)
    for v in first:
        plan.set_variant(v)
        acc = to_np(plan.force())
        assert acc.tobytes() == ref, f"variant {v}"
    if chunk == 64:
        with pytest.raises(SrError):
            plan.set_variant(8)
        return
    a_ref, _ = oracle_force(w["volumes"], w["params"])
    plan.set_variant(7)
    assert_force_close(to_np(plan.force()), a_ref, f"{name} variant 7")
    packed = None
    for v in range(8, 12):
        plan.set_variant(v)
        acc = to_np(plan.force())
        if packed is None:
            packed = acc
            assert_force_close(acc, a_ref, f"{name} variant {v}")
        assert acc.tobytes() == packed.tobytes(), f"variant {v}"
    plan.set_variant(12)                      # the packed loop in batches of 64
    acc12 = to_np(plan.force())
    assert_force_close(acc12, a_ref, f"{name} variant 12")
    # the flat neighbour enumeration visits the same chunks in the same
    # order: 13 gives 11's bits, 14 gives 12's
    plan.set_variant(13)
    assert to_np(plan.force()).tobytes() == packed.tobytes(), "variant 13"
    plan.set_variant(14)
    assert to_np(plan.force()).tobytes() == acc12.tobytes(), "variant 14"


GROUPED = range(15, 17)        # i-groups of 8 or 16 slots, each with its own ring


def test_grouped_variants_forces_and_counts(small_case):
    # the grouped kernel: forces within the oracle bar, per-particle pair
    # counts bit-exact (same binary32 predicate as the 32-lane kernel), and
    # its counting mode gives the force mode's bits
    from paper_1411_3396_b300 import SrError
    name, w, chunk = small_case
    pos = np.concatenate([p for p, _ in w["volumes"]])
    plan = make_plan(w["volumes"], w["params"], chunk_size=chunk)
    plan.bin(torch.from_numpy(pos).cuda())
    if chunk == 64:
        for v in GROUPED:
            with pytest.raises(SrError):
                plan.set_variant(v)
        return
    B = oracle_binning(plan, w["volumes"])
    ref = oforce.pair_counts_fp32(B, w["volumes"], w["params"]["rc"], w["params"]["eps"])
    a_ref, _ = oracle_force(w["volumes"], w["params"])
    for v in GROUPED:
        plan.set_variant(v)
        acc_c, pairs, pp = plan.force(count=True, per_particle=True)
        np.testing.assert_array_equal(to_np(pp), ref, err_msg=f"variant {v}")
        assert int(pairs.item()) == int(ref.sum()), f"variant {v}"
        acc = to_np(plan.force())
        assert acc.tobytes() == to_np(acc_c).tobytes(), f"variant {v}"
        assert_force_close(acc, a_ref, f"{name} variant {v}")
        assert np.all(acc[:, 3] == 0)
        again = to_np(plan.force())
        assert again.tobytes() == acc.tobytes(), f"variant {v} not deterministic"


def test_flat_and_grouped_variants_brute_force_tiny_boxes():
    # boxes of 1 to 2 cells per axis: the flat enumeration's 27 neighbour
    # lanes map to a few cells under several image shifts, chunks see their
    # own images through several faces, ragged groups in nearly every chunk
    for L, n, seed in [(7.0, 300, 1), (8.0, 512, 2), (10.0, 400, 3), (6.5, 64, 4), (9.0, 37, 5)]:
        pos = gen.uniform_box(n, L, seed)
        params = dict(rc=3.0, eps=0.1, sigma=0.8)
        c = ofit.fit_poly(3.0, 0.8, 0.1)
        a_ref, cnt = oforce.accel_brute(pos, L, 3.0, 0.1, c)
        plan = make_plan([(pos, L)], params)
        plan.bin(torch.from_numpy(pos).cuda())
        for v in (13, 14, *GROUPED):
            plan.set_variant(v)
            assert_force_close(to_np(plan.force()), a_ref, f"L={L} variant {v}")
            _, pairs, _ = plan.force(count=True)
            assert abs(int(pairs.item()) - int(cnt.sum())) <= 8


@pytest.mark.parametrize("name", ["zeldovich128", "clustered256"])
def test_geometry_tuner_plan_matches_oracle(name):
    # sr_plan_tune: chunk size, cells per axis and variant chosen by timing;
    # the kept plan is the fastest candidate and its forces meet the bar
    from paper_1411_3396_b300 import Plan
    w = _work(name)
    (pos, box), = w["volumes"]
    prm = w["params"]
    plan, cands = Plan.tune(box, prm["rc"], prm["eps"], prm["sigma"], torch.from_numpy(pos).cuda())
    assert len(cands) >= 4 and {c["chunk_size"] for c in cands} == {32, 64}
    info = plan.info()
    best = min(cands, key=lambda c: c["ms"])
    assert (info["chunk_size"], plan.volume(0)["n_cells"], info["variant"]) == \
        (best["chunk_size"], best["n_cells"], best["variant"])
    a_ref, _ = oracle_force(w["volumes"], prm)
    assert_force_close(to_np(plan.force()), a_ref, f"{name} tuned geometry")
    plan.close()


def test_plain_kernel_matches_oracle(small_case):
    name, w, chunk = small_case
    pos = np.concatenate([p for p, _ in w["volumes"]])
    plan = make_plan(w["volumes"], w["params"], chunk_size=chunk)
    plan.bin(torch.from_numpy(pos).cuda())
    acc = to_np(plan.force_plain())
    a_ref, _ = oracle_force(w["volumes"], w["params"])
    assert_force_close(acc, a_ref, name + " plain")


def test_force_of_unwrapped_positions():
    # positions anywhere in [-L, 2L) are folded by the binning: the forces of
    # periodic images of the set match the oracle's forces of the set
    w = _work("clustered256")
    (pos, box), = w["volumes"]
    rng = np.random.default_rng(21)
    shifted = pos + rng.choice([-1.0, 0.0, 1.0], size=pos.shape) * box
    shifted = np.where(shifted < -box, shifted + box, shifted)
    shifted = np.where(shifted >= 2 * box, shifted - box, shifted)
    plan, acc, _, _ = _gpu([(shifted, box)], w["params"], count=False)
    a_ref, _ = oracle_force([(pos, box)], w["params"])
    assert_force_close(acc, a_ref, "unwrapped positions")
    plan.close()


def test_force_is_deterministic():
    w = _work("clustered256")
    pos = torch.from_numpy(np.concatenate([p for p, _ in w["volumes"]])).cuda()
    plan = make_plan(w["volumes"], w["params"])
    outs = []
    for _ in range(3):
        plan.bin(pos)
        outs.append(to_np(plan.force()).tobytes())
    assert outs[0] == outs[1] == outs[2]


def test_force_brute_force_tiny_boxes():
    for L, n, seed in [(7.0, 300, 1), (8.0, 512, 2), (10.0, 400, 3), (6.5, 64, 4)]:
        pos = gen.uniform_box(n, L, seed)
        params = dict(rc=3.0, eps=0.1, sigma=0.8)
        _, acc, pairs, pp = _gpu([(pos, L)], params)
        c = ofit.fit_poly(3.0, 0.8, 0.1)
        a_ref, _ = oforce.accel_brute(pos, L, 3.0, 0.1, c)
        assert_force_close(acc, a_ref, f"L={L}")


def test_lattice_and_two_body():
    params = dict(rc=3.0, eps=0.1, sigma=0.8)
    pos = gen.lattice(12, 12.0)
    _, acc, pairs, pp = _gpu([(pos, 12.0)], params)
    assert np.max(np.abs(acc[:, :3])) < 1e-4           # binary32 of a zero sum
    assert np.all(pp == pp[0])
    c = ofit.fit_poly(3.0, 0.8, 0.1)
    for r in (0.05, 0.7, 2.9):
        pos = gen.two_body(r, 20.0, axis=2)
        _, acc, pairs, pp = _gpu([(pos, 20.0)], params)
        a_ref, _ = oforce.accel_brute(pos, 20.0, 3.0, 0.1, c)
        # binary32 cancellation in r^-3 - p near r_c: absolute error relative to 1/r^2
        np.testing.assert_allclose(acc[:, :3], a_ref, rtol=2e-6, atol=2e-6 / r ** 2)
        assert pairs == 2


def test_single_particle_and_far_pair():
    params = dict(rc=3.0, eps=0.1, sigma=0.8)
    _, acc, pairs, pp = _gpu([(np.array([[3.0, 4.0, 5.0]]), 16.0)], params)
    assert np.all(acc == 0) and pairs == 0
    _, acc, pairs, pp = _gpu([(np.array([[1.0, 1.0, 1.0], [9.0, 9.0, 9.0]]), 16.0)], params)
    assert np.all(acc == 0) and pairs == 0


def test_newton_third_law_on_gpu():
    w = _work("clustered256")
    plan, acc, _, _ = _gpu(w["volumes"], w["params"], count=False)
    vel = torch.zeros((acc.shape[0], 4), dtype=torch.float32, device="cuda")
    inv = to_np(plan.invariants(vel, torch.from_numpy(acc).cuda()))
    assert np.all(np.abs(inv[3:6]) <= 1e-5 * np.abs(acc[:, :3]).sum())


@pytest.mark.parametrize("chunk", [32, 64])
def test_passive_particles_every_variant(chunk):
    # sr_bin_active: with every other particle passive, each variant writes
    # the active rows with the unmasked run's bits (chunks holding an active
    # particle run unchanged), leaves passive rows untouched, and counts the
    # active rows' pairs; with no active particle nothing is written
    from paper_1411_3396_b300 import SrError
    w = _work("clustered256")
    (pos, box), = w["volumes"]
    x = torch.from_numpy(pos).cuda()
    n = len(pos)
    plan = make_plan(w["volumes"], w["params"], chunk_size=chunk)
    active = torch.zeros(n, dtype=torch.bool, device="cuda")
    active[::2] = True
    act = to_np(active)
    for v in range(17):
        plan.bin(x)
        try:
            plan.set_variant(v)
        except SrError:
            continue
        full, pairs_full, pp_full = plan.force(count=True, per_particle=True)
        full, pp_full = to_np(full), to_np(pp_full)
        ref = to_np(plan.force())
        plan.bin(x, active=active)
        acc = torch.full((n, 4), float("nan"), dtype=torch.float32, device="cuda")
        got = to_np(plan.force(acc))
        assert got[act].tobytes() == ref[act].tobytes(), f"variant {v}"
        assert np.all(np.isnan(got[~act])), f"variant {v}"
        pp = torch.full((n,), -5, dtype=torch.int32, device="cuda")
        _, pairs, pp = plan.force(count=True, per_particle=pp)
        pp = to_np(pp)
        assert np.array_equal(pp[act], pp_full[act]) and np.all(pp[~act] == -5), f"variant {v}"
        assert int(pairs.item()) == int(pp_full[act].sum()), f"variant {v}"
    plan.bin(x, active=torch.zeros(n, dtype=torch.bool, device="cuda"))
    acc = torch.full((n, 4), float("nan"), dtype=torch.float32, device="cuda")
    assert np.all(np.isnan(to_np(plan.force(acc))))
    assert plan.export("counters").cpu().numpy()[5] == 0          # no work items
    plan.status()
