"""The C-ABI library builds, loads without a GPU, and exports every entry
point the headers under include/ declare; host-only entry points and the
argument checks that precede any device work behave on the CPU."""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest

from oracle import fit as ofit

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    from paper_1411_3396_b300 import build
    path = build()
    return ctypes.CDLL(str(path))


def declared_functions():
    text = "\n".join(p.read_text() for p in sorted((ROOT / "include").glob("*.h")))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(sr_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sr_bin", "sr_force", "sr_kick", "sr_force_vjp", "sr_fit_poly",
                 "sr_plan_create", "sr_plan_batch", "sr_plan_destroy", "sr_last_error",
                 "sr_centers_create", "sr_centers_run", "sr_centers_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_checked_build_exports_the_same_boundary(lib):
    # the bounds-checked build (-DSR_CHECK) is the same library with the
    # index checks compiled in
    from paper_1411_3396_b300.build import LIB_CHECKED
    chk = ctypes.CDLL(str(LIB_CHECKED))
    for name in declared_functions():
        assert hasattr(chk, name), name
    assert chk.sr_build_checked() == 1 and lib.sr_build_checked() == 0


@pytest.mark.parametrize("mode,mname", [(0, "constrained"), (1, "unconstrained")])
@pytest.mark.parametrize("rc,sigma,eps", [(3.0, 0.8, 0.1), (3.0, 0.8, 0.05), (2.5, 0.6, 0.02)])
def test_library_fit_matches_oracle(lib, mode, mname, rc, sigma, eps):
    f = lib.sr_fit_poly
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    out = (ctypes.c_double * 6)()
    assert f(rc, sigma, eps, mode, out) == 0
    got = np.array(out[:]) * (rc * rc) ** np.arange(6)
    ref = ofit.fit_poly(rc, sigma, eps, mname) * (rc * rc) ** np.arange(6)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_fit_rejects_bad_arguments(lib):
    f = lib.sr_fit_poly
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    out = (ctypes.c_double * 6)()
    assert f(-1.0, 0.8, 0.1, 0, out) == 1
    assert f(3.0, 0.0, 0.1, 0, out) == 1
    assert f(3.0, 0.8, 0.1, 7, out) == 1
    lib.sr_last_error.restype = ctypes.c_char_p
    assert b"bad" in lib.sr_last_error()


def test_product_path_does_not_reference_the_oracle():
    pkg = ROOT / "paper_1411_3396_b300"
    for p in list(pkg.rglob("*.py")) + list(pkg.rglob("*.cu")) + list(pkg.rglob("*.cpp")) + \
            list(pkg.rglob("*.h")):
        assert "oracle" not in p.read_text(), p


def test_centers_argument_checks_need_no_device(lib):
    v = ctypes.c_void_p
    create = lib.sr_centers_create
    create.restype = ctypes.c_int
    create.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(v)]
    h = v()
    assert create(0, 10, ctypes.byref(h)) == 1 and not h.value
    assert create(100, 0, ctypes.byref(h)) == 1
    assert create(1 << 31, 10, ctypes.byref(h)) == 1
    assert create(100, 10, None) == 1
    run = lib.sr_centers_run
    run.restype = ctypes.c_int
    run.argtypes = [v, v, v, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                    v, v, v, v]
    assert run(None, None, None, 0, 0, 1.0, 0.1, None, None, None, None) == 1
    lib.sr_centers_set_variant.restype = ctypes.c_int
    lib.sr_centers_set_variant.argtypes = [v, ctypes.c_int]
    assert lib.sr_centers_set_variant(None, 0) == 1
    lib.sr_centers_get_info.restype = ctypes.c_int
    lib.sr_centers_get_info.argtypes = [v, v]
    assert lib.sr_centers_get_info(None, None) == 1
    lib.sr_centers_destroy.restype = ctypes.c_int
    lib.sr_centers_destroy.argtypes = [v]
    assert lib.sr_centers_destroy(None) == 0


def test_pm_argument_checks_need_no_device(lib):
    v = ctypes.c_void_p
    create = lib.sr_pm_create
    create.restype = ctypes.c_int
    create.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.POINTER(v)]
    h = v()
    assert create(100, 10.0, 0.8, 10, ctypes.byref(h)) == 1 and not h.value    # not a power of two
    assert create(8, 10.0, 0.8, 10, ctypes.byref(h)) == 1                      # too small
    assert create(2048, 10.0, 0.8, 10, ctypes.byref(h)) == 1                   # too large
    assert create(64, -1.0, 0.8, 10, ctypes.byref(h)) == 1
    assert create(64, 10.0, -0.5, 10, ctypes.byref(h)) == 1
    assert create(64, 10.0, 0.8, 0, ctypes.byref(h)) == 1
    for name, nargs in (("sr_pm_deposit", 4), ("sr_pm_transform", 2), ("sr_pm_power", 5), ("sr_pm_fft", 4),
                        ("sr_pm_copy", 4)):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        assert f(*([None] * nargs)) == 1, name
    lib.sr_pm_force.restype = ctypes.c_int
    assert lib.sr_pm_force(None, None, ctypes.c_int64(0), None, 0, None) == 1
    lib.sr_pm_destroy.restype = ctypes.c_int
    assert lib.sr_pm_destroy(None) == 0


def test_fof_argument_checks_need_no_device(lib):
    v = ctypes.c_void_p
    create = lib.sr_fof_create
    create.restype = ctypes.c_int
    create.argtypes = [ctypes.c_int64, ctypes.POINTER(v)]
    h = v()
    assert create(0, ctypes.byref(h)) == 1 and not h.value
    assert create(1 << 31, ctypes.byref(h)) == 1
    run = lib.sr_fof_run
    run.restype = ctypes.c_int
    run.argtypes = [v, v, v, ctypes.c_int64, ctypes.c_double, ctypes.c_int, v, v, v]
    assert run(None, None, None, 0, 0.2, 40, None, None, None) == 1
    lib.sr_fof_get_info.restype = ctypes.c_int
    assert lib.sr_fof_get_info(None, None) == 1
    lib.sr_fof_set_iteration_limit.restype = ctypes.c_int
    lib.sr_fof_set_iteration_limit.argtypes = [v, ctypes.c_int64]
    assert lib.sr_fof_set_iteration_limit(None, 5) == 1
    lib.sr_fof_destroy.restype = ctypes.c_int
    assert lib.sr_fof_destroy(None) == 0


def test_trajectory_plan_list_checks_need_no_device():
    # one plan per substep: the list must hold exactly `steps` plans
    from paper_1411_3396_b300.autograd import _plans
    with pytest.raises(ValueError):
        _plans([object(), object()], 2)
    with pytest.raises(ValueError):
        _plans([], 3)
    with pytest.raises(ValueError):
        _plans(None, 1)
    # the same plan object twice would keep only its last substep's binning
    from paper_1411_3396_b300.api import Plan
    p, q = Plan.__new__(Plan), Plan.__new__(Plan)
    with pytest.raises(ValueError):
        _plans([p] * 3, 3)
    with pytest.raises(ValueError):
        _plans([p, q, p], 3)
    assert _plans([p, q], 2) == (p, q)
    assert _plans(p, 5) == (p,)
