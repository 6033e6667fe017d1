"""The bounds-checked build (libsr_b300_check.so, compiled with -DSR_CHECK):
the small parity cases run under it in a child process (SR_B300_CHECKED=1)
and under the release build in another; every bounds check passes
(sr_plan_status returns SR_OK, the center finder reports no check code),
and the two builds give the same bits for binning, forces in every
variant, pair counts, passive-ghost binning and the VJP.  The self-test
shows a failed check reaching sr_plan_status as SR_ERR_CHECK in the
checked build (with no memory access behind it) and nothing in the release
build."""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _child(out_path):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from helpers import make_plan, to_np
    from paper_1411_3396_b300 import Centers, SrError
    from paper_1411_3396_b300 import _lib as L
    from workloads import configs as wc
    from workloads import generators as gen
    lib = L.load()
    res = {"checked": np.array([lib.sr_build_checked()])}
    for name in ("uniform4k", "zeldovich128", "clustered256", "batch64", "diff64"):
        w = wc.make_workload(wc.small_variant(name))
        pos = np.concatenate([p for p, _ in w["volumes"]])
        x = torch.from_numpy(pos).cuda()
        for chunk in (32, 64):
            plan = make_plan(w["volumes"], w["params"], chunk_size=chunk)
            plan.bin(x)
            key = f"{name}_c{chunk}"
            res[key + "_slots"] = to_np(plan.export("slot_pos"))
            acc, pairs, pp = plan.force(count=True, per_particle=True)
            res[key + "_count_acc"], res[key + "_pp"] = to_np(acc), to_np(pp)
            for v in range(lib.sr_variant_count()):
                try:
                    plan.set_variant(v)
                except SrError:
                    continue
                res[f"{key}_v{v}"] = to_np(plan.force())
            g = np.zeros((len(pos), 4), np.float32)
            g[:, :3] = np.random.default_rng(3).standard_normal((len(pos), 3))
            res[key + "_vjp"] = to_np(plan.vjp(torch.from_numpy(g).cuda()))
            # passive particles: every other one
            active = torch.zeros(len(pos), dtype=torch.bool, device="cuda")
            active[::2] = True
            plan.bin(x, active=active)
            plan.set_variant(0)
            acc = torch.zeros((len(pos), 4), dtype=torch.float32, device="cuda")
            res[key + "_active"] = to_np(plan.force(acc))
            plan.status()                              # raises on a failed bounds check
            plan.close()
    pos, lab, sizes = gen.nfw_clustered(8192, 20.0, 1002, m_lo=40.0, m_hi=1500.0)
    c = Centers(len(pos), len(sizes))
    phi, cen, _ = c.run(torch.from_numpy(pos).cuda(), torch.from_numpy(lab.astype(np.int32)).cuda(),
                        len(sizes), 20.0, 0.05)
    res["centers_phi"] = phi.cpu().numpy()
    res["centers_check"] = np.array([c.info()["check_code"]])
    c.close()
    # the self-test: a check whose condition is false, no access behind it
    w = wc.make_workload(wc.small_variant("uniform4k"))
    plan = make_plan(w["volumes"], w["params"])
    plan.bin(torch.from_numpy(w["volumes"][0][0]).cuda())
    rc = lib.sr_check_selftest(plan._h, None)
    res["selftest_rc"] = np.array([rc])
    res["selftest_status"] = np.array([lib.sr_plan_status(plan._h, None)])
    res["selftest_msg"] = np.array([lib.sr_last_error().decode()])
    res["after_status"] = np.array([lib.sr_plan_status(plan._h, None)])     # the report clears the word
    plan.close()
    np.savez(out_path, **res)


def _run(tmp_path, checked):
    out = str(tmp_path / ("checked.npz" if checked else "release.npz"))
    env = dict(os.environ, SR_B300_CHECKED="1" if checked else "0")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), out], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return dict(np.load(out))


def test_checked_build_matches_release_and_reports(tmp_path):
    chk = _run(tmp_path, True)
    rel = _run(tmp_path, False)
    assert chk["checked"][0] == 1 and rel["checked"][0] == 0
    assert set(chk) == set(rel)
    for k in chk:
        if k.startswith(("checked", "selftest", "after")):
            continue
        assert chk[k].tobytes() == rel[k].tobytes(), k
    assert chk["centers_check"][0] == 0
    assert chk["selftest_rc"][0] == 0 and rel["selftest_rc"][0] == 0
    assert chk["selftest_status"][0] == 7 and "bounds check 99" in str(chk["selftest_msg"][0])
    assert rel["selftest_status"][0] == 0
    assert chk["after_status"][0] == 0


if __name__ == "__main__":
    _child(sys.argv[1])
