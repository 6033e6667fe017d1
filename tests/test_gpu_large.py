"""A particle set eight times the benchmark's (2^27 uniform particles,
box 512, mean density one per unit volume): binning and forces in the
library's default configuration, with sampled rows compared one by one
with the FP64 oracle (each row evaluated on its own neighbourhood, cut out
of the set on the host), and the capacity bound of plan creation."""
import numpy as np
import pytest

from oracle import fit as ofit
from oracle import force as oforce
from workloads import generators as gen

from helpers import MAX_TOL, MEDIAN_TOL, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_plan_capacity_bound():
    from paper_1411_3396_b300 import Plan, SrError
    with pytest.raises(SrError) as e:
        Plan(512.0, 3.0, 0.1, 0.8, (1 << 30) + 1)
    assert e.value.code == 1                         # SR_ERR_ARG: particle count out of range


def test_large_uniform_set_sampled_rows():
    from paper_1411_3396_b300 import Plan
    n, L, rc, eps, sigma = 1 << 27, 512.0, 3.0, 0.1, 0.8
    pos = gen.uniform_box(n, L, 2027)
    plan = Plan(L, rc, eps, sigma, n)
    x = torch.from_numpy(pos).cuda()
    plan.bin(x)
    acc, pairs, _ = plan.force(count=True)
    a_gpu = to_np(acc)[:, :3].astype(np.float64)
    assert np.all(np.isfinite(a_gpu))
    assert 100 * n < int(pairs.item()) < 130 * n        # about (4 pi / 3) r_c^3 = 113 per particle
    del x, acc
    torch.cuda.empty_cache()
    c = ofit.fit_poly(rc, sigma, eps)
    # host cell lists (side 4 >= r_c): each sampled row's 27 cells hold all
    # its neighbours; the oracle sums the row over that subset
    nc = int(L // 4.0)
    ci = np.floor(pos / (L / nc)).astype(np.int64) % nc
    key = (ci[:, 0] * nc + ci[:, 1]) * nc + ci[:, 2]
    order = np.argsort(key, kind="stable")
    starts = np.searchsorted(key[order], np.arange(nc ** 3 + 1))
    offs = np.array([(a, b, e) for a in (-1, 0, 1) for b in (-1, 0, 1) for e in (-1, 0, 1)])
    rows = np.random.default_rng(5).choice(n, 200, replace=False)
    ref = np.empty((len(rows), 3))
    for k, i in enumerate(rows):
        cc = (ci[i] + offs) % nc
        ks = (cc[:, 0] * nc + cc[:, 1]) * nc + cc[:, 2]
        near = np.concatenate([order[starts[q]:starts[q + 1]] for q in ks])
        j = int(np.nonzero(near == i)[0][0])
        a, _ = oforce.accel_rows(pos[near], L, rc, eps, c, [j])
        ref[k] = a[0]
    mag = np.linalg.norm(ref, axis=1)
    rms = np.sqrt(np.mean(mag * mag))
    rel = np.linalg.norm(a_gpu[rows] - ref, axis=1) / np.maximum(mag, 1e-3 * rms)
    med, mx = float(np.median(rel)), float(rel.max())
    assert med <= MEDIAN_TOL and mx <= MAX_TOL, f"median {med:.3g} max {mx:.3g}"
    print(f"2^27 particles: {int(pairs.item())} pairs, 200 rows median {med:.2e} max {mx:.2e}")
    plan.close()
