"""The whole force split on the GPU (short-range pair sums plus the PM
long-range accelerations accumulated onto them) against the sum of the two
FP64 oracles, and a two-body check that the split adds up to Newton."""
import numpy as np
import pytest

from oracle import fit as ofit
from oracle import force as oforce
from oracle import pm as opm
from workloads import configs as wc

from helpers import assert_force_close, make_plan, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _total_force(vols, params, ng):
    from paper_1411_3396_b300 import PM
    (pos, box), = vols
    plan = make_plan(vols, params)
    x = torch.from_numpy(pos).cuda()
    plan.bin(x)
    acc = plan.force()
    pm = PM(ng, box, params["sigma"], len(pos))
    pm.deposit(x)
    pm.force(x, acc, accumulate=True)
    torch.cuda.synchronize()
    out = to_np(acc)
    pm.close()
    plan.close()
    return out


def test_short_plus_long_range_matches_oracles():
    w = wc.make_workload(wc.small_variant("clustered256"))
    (pos, box), = w["volumes"]
    prm = w["params"]
    acc = _total_force(w["volumes"], prm, 32)
    c = ofit.fit_poly(prm["rc"], prm["sigma"], prm["eps"])
    a_sr, _ = oforce.accel_kdtree(pos, box, prm["rc"], prm["eps"], c)
    a_lr = opm.pm_accel(pos, box, 32, prm["sigma"])
    assert_force_close(acc, a_sr + a_lr, "short + long range")


def test_split_adds_up_to_newton_on_the_gpu():
    # an isolated pair in a 64^3 box: GPU short + long range ~ softened Newton
    prm = dict(rc=3.0, eps=0.05, sigma=0.8)
    for r in (1.0, 1.8, 2.6, 4.0):
        pos = np.array([[20.2, 30.1, 25.7], [20.2 + r, 30.1, 25.7]])
        acc = _total_force([(pos, 64.0)], prm, 64)
        newton = -r / (r * r + prm["eps"] ** 2) ** 1.5
        assert acc[1, 0] == pytest.approx(newton, rel=0.03), r
        assert acc[0, 0] == pytest.approx(-newton, rel=0.03), r
