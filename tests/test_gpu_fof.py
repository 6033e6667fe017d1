"""Friends-of-friends (sr_fof_run) against the FP64 oracle: labels and halo
sizes bit-exact on clustered sets, special configurations (chains at the
linking length, periodic links, lattices, the size threshold), batch plans,
64-particle chunks, and closure properties on the full 256^3 set."""
import numpy as np
import pytest

from oracle import fof as ofof
from workloads import configs as wc
from workloads import generators as gen

from helpers import make_plan

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _gpu_fof(vols, params, link, min_members, chunk_size=0):
    from paper_1411_3396_b300 import FOF
    pos = np.concatenate([p for p, _ in vols])
    plan = make_plan(vols, params, chunk_size=chunk_size)
    x = torch.from_numpy(pos).cuda()
    plan.bin(x)
    f = FOF(len(pos))
    lab, sizes = f.run(plan, x, link, min_members)
    info = f.info()
    lab = lab.cpu().numpy()
    sizes = sizes.cpu().numpy()[:info["n_halos"]]
    f.close()
    plan.close()
    assert info["error"] == 0
    return lab, sizes, info


PARAMS = dict(rc=3.0, eps=0.05, sigma=0.8)


@pytest.mark.parametrize("link,min_members", [(0.2, 40), (0.168, 40), (0.2, 5), (0.35, 10)])
@pytest.mark.parametrize("chunk", [32, 64])
def test_clustered_labels_bit_exact(link, min_members, chunk):
    cfg = wc.small_variant("clustered256")
    w = wc.make_workload(cfg)
    (pos, box), = w["volumes"]
    lab, sizes, info = _gpu_fof(w["volumes"], PARAMS, link, min_members, chunk)
    lab_o, sizes_o = ofof.fof(pos, box, link, min_members)
    np.testing.assert_array_equal(lab, lab_o)
    np.testing.assert_array_equal(sizes, sizes_o)
    assert info["n_members"] == int((lab_o >= 0).sum())
    assert info["links"] == len(ofof.friend_pairs(pos, box, link))
    print(f"link {link} min {min_members} chunk {chunk}: {info['n_halos']} halos, "
          f"{info['links']} links, {info['band_checks']} binary64 checks")


def test_cell_side_not_a_power_of_two():
    # box 30: 7 cells of side 30/7, so the fine-grid side h is not a power of
    # two and positions are scaled by a binary64 division
    pos, _, _ = gen.nfw_clustered(12000, 30.0, 71, m_lo=40.0, m_hi=2000.0)
    for link, mm in ((0.2, 20), (0.3, 5)):
        lab, sizes, info = _gpu_fof([(pos, 30.0)], PARAMS, link, mm)
        lab_o, sizes_o = ofof.fof(pos, 30.0, link, mm)
        np.testing.assert_array_equal(lab, lab_o)
        np.testing.assert_array_equal(sizes, sizes_o)
        assert info["links"] == len(ofof.friend_pairs(pos, 30.0, link))
        assert info["n_halos"] > 0


def test_special_configurations():
    L = 20.0
    line = np.zeros((60, 3)) + 7.0
    line[:, 0] = 2.0 + np.arange(60) * 0.99 * 0.2
    lab, sizes, _ = _gpu_fof([(line, L)], PARAMS, 0.2, 2)
    assert np.all(lab == 0) and list(sizes) == [60]
    line[:, 0] = 2.0 + np.arange(60) * 1.01 * 0.2
    lab, sizes, _ = _gpu_fof([(line, L)], PARAMS, 0.2, 2)
    assert np.all(lab == -1) and len(sizes) == 0
    pts = np.array([[19.9, 5.0, 5.0], [0.1, 5.0, 5.0], [0.35, 5.0, 5.0], [5.0, 19.95, 0.02],
                    [5.0, 0.1, 19.9], [10.0, 10.0, 10.0]])
    lab, sizes, _ = _gpu_fof([(pts, L)], PARAMS, 0.3, 2)
    np.testing.assert_array_equal(lab, [0, 0, 0, 1, 1, -1])
    lat = gen.lattice(8, 8.0)
    lab, _, _ = _gpu_fof([(lat, 8.0)], PARAMS, 0.99, 2)
    assert np.all(lab == -1)


def test_pairs_at_the_linking_length_use_the_exact_test():
    # separations within a relative 1e-9 of the linking length on both
    # sides: the binary32 predicate cannot decide them, the binary64 test
    # must agree with the oracle
    rng = np.random.default_rng(3)
    L, link = 16.0, 0.2
    base = rng.uniform(1.0, 15.0, (400, 3))
    dirs = gen.random_directions(400, 3, 4)
    eps = rng.choice([-1.0, 1.0], 400) * 1e-9
    other = base + dirs * (link * (1.0 + eps))[:, None]
    pos = np.empty((800, 3))
    pos[0::2], pos[1::2] = base, other
    lab, sizes, info = _gpu_fof([(pos, L)], PARAMS, link, 2)
    lab_o, sizes_o = ofof.fof(pos, L, link, 2)
    np.testing.assert_array_equal(lab, lab_o)
    assert info["band_checks"] >= 400


def test_batch_plan_volumes_are_independent():
    vols = []
    for v in range(3):
        pos, _, _ = gen.nfw_clustered(4000, 16.0, 50 + v, m_lo=40.0, m_hi=800.0)
        vols.append((pos, 16.0))
    lab, sizes, _ = _gpu_fof(vols, PARAMS, 0.2, 20)
    ref = []
    off = 0
    for pos, box in vols:
        l_o, _ = ofof.fof(pos, box, 0.2, 20)
        # renumber per-volume halos into the global tag order
        ref.append(np.where(l_o >= 0, l_o + off, -1))
        off += int(l_o.max()) + 1 if (l_o >= 0).any() else 0
    np.testing.assert_array_equal(lab, np.concatenate(ref))


def test_argument_errors():
    from paper_1411_3396_b300 import FOF, SrError
    pos = gen.uniform_box(1000, 12.0, 1)
    plan = make_plan([(pos, 12.0)], PARAMS)
    x = torch.from_numpy(pos).cuda()
    f = FOF(1000)
    with pytest.raises(SrError):
        f.run(plan, x, 0.2)                      # plan not binned yet
    plan.bin(x)
    with pytest.raises(SrError):
        f.run(plan, x, 50.0)                     # linking length above the cell side
    with pytest.raises(SrError):
        f.run(plan, x, -0.2)
    f.close()
    plan.close()


def test_full_clustered_256_closure():
    # full size: every sampled particle's friends (found directly) share its
    # group, the halo sizes are the label counts, and no halo is below the
    # minimum size
    from scipy.spatial import cKDTree
    w = wc.make_workload(wc.CONFIGS["clustered256"])
    (pos, box), = w["volumes"]
    link = 0.168
    lab, sizes, info = _gpu_fof(w["volumes"], PARAMS, link, 40)
    assert info["n_halos"] == len(sizes) and np.all(sizes >= 40)
    np.testing.assert_array_equal(np.bincount(lab[lab >= 0], minlength=len(sizes)), sizes)
    x = np.mod(pos, box)
    x[x >= box] = 0.0
    tree = cKDTree(x, boxsize=box)
    idx = np.random.default_rng(0).choice(len(pos), 5000, replace=False)
    for i in idx:
        nb = np.array(tree.query_ball_point(x[i], link * (1 + 1e-6)), dtype=np.int64)
        nb = nb[nb != i]
        d = x[nb] - x[i]
        d = d - box * np.round(d / box)
        s = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
        fr = nb[s < link * link]
        assert np.all(lab[fr] == lab[i]) or (lab[i] == -1 and np.all(lab[fr] == -1))
    print(f"256^3 FOF b=0.168: {info['n_halos']} halos, {info['n_members']} members, "
          f"largest {info['max_members']}, {info['links']} links")


def test_iteration_limit_reports_timeout_and_workspace_recovers():
    # the union-find loops run out on purpose (limit 1): the run returns,
    # the host reads SR_ERR_TIMEOUT, and the next run with the default limit
    # is exact again; nothing faults or hangs on the device
    from paper_1411_3396_b300 import FOF, SrError
    from paper_1411_3396_b300._lib import SR_ERR_TIMEOUT
    w = wc.make_workload(wc.small_variant("clustered256"))
    (pos, box), = w["volumes"]
    plan = make_plan(w["volumes"], PARAMS)
    x = torch.from_numpy(pos).cuda()
    plan.bin(x)
    f = FOF(len(pos))
    f.set_iteration_limit(1)
    f.run(plan, x, 0.2, 40)
    with pytest.raises(SrError) as e:
        f.info()
    assert e.value.code == SR_ERR_TIMEOUT
    f.set_iteration_limit(0)
    lab, _ = f.run(plan, x, 0.2, 40)
    info = f.info()
    assert info["error"] == 0
    np.testing.assert_array_equal(lab.cpu().numpy(), ofof.fof(pos, box, 0.2, 40)[0])
    f.close()
    plan.close()
