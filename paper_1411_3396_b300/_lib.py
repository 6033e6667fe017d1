"""ctypes declarations of the C ABI in include/sr.h, include/sr_centers.h,
include/sr_pm.h and include/sr_fof.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
from ctypes import POINTER, c_double, c_float, c_int, c_int64, c_uint64, c_void_p, c_char_p

import os

from .build import LIB, LIB_CHECKED

SR_OK, SR_ERR_ARG, SR_ERR_CUDA, SR_ERR_CAPACITY, SR_ERR_STATE, SR_ERR_RANGE, SR_ERR_TIMEOUT, SR_ERR_CHECK = range(8)
FIT_MODES = {"constrained": 0, "unconstrained": 1}
EXPORTS = {
    "perm": 0, "cell_start": 1, "cell_chunk_start": 2, "slot_pos": 3, "slot_idx": 4,
    "chunk_meta": 5, "chunk_lo": 6, "chunk_hi": 7, "order": 8, "cost": 9, "counters": 10,
}


class SrParams(ctypes.Structure):
    _fields_ = [("box", c_double), ("r_c", c_double), ("eps", c_double), ("sigma", c_double),
                ("fit_mode", c_int), ("n_cells", c_int), ("sub_bits", c_int), ("chunk_size", c_int)]


class SrPlanInfo(ctypes.Structure):
    _fields_ = [("n_particles", c_int64), ("capacity", c_int64), ("n_volumes", c_int64),
                ("total_cells", c_int64), ("max_chunks", c_int64), ("n_chunks", c_int64),
                ("sub_bits", ctypes.c_int32), ("key_bits", ctypes.c_int32),
                ("workers", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("chunk_size", ctypes.c_int32),
                ("coef", c_double * 6)]


class SrTuneEntry(ctypes.Structure):
    _fields_ = [("chunk_size", ctypes.c_int32), ("n_cells", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("ms", c_float)]


class SrCentersInfo(ctypes.Structure):
    _fields_ = [("n_particles", c_int64), ("n_members", c_int64), ("n_halos", c_int64),
                ("max_members", c_int64), ("pairs", c_int64), ("items", c_int64),
                ("evaluated", c_int64), ("fixed_shift", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("bad_labels", c_int64), ("wide_members", c_int64), ("check_code", c_int64)]


class SrFofInfo(ctypes.Structure):
    _fields_ = [("n_particles", c_int64), ("n_halos", c_int64), ("n_members", c_int64),
                ("max_members", c_int64), ("links", c_int64), ("band_checks", c_int64), ("tests", c_int64),
                ("error", c_int64)]


class SrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sr error {code}: {msg}")
        self.code = code


SIGNATURES = {
    "sr_fit_poly": (c_int, [c_double, c_double, c_double, c_int, POINTER(c_double)]),
    "sr_plan_create": (c_int, [POINTER(SrParams), c_int64, POINTER(c_void_p)]),
    "sr_plan_batch": (c_int, [POINTER(SrParams), POINTER(c_int64), c_int, POINTER(c_void_p)]),
    "sr_plan_destroy": (c_int, [c_void_p]),
    "sr_plan_get_info": (c_int, [c_void_p, POINTER(SrPlanInfo)]),
    "sr_plan_volume_info": (c_int, [c_void_p, c_int, POINTER(c_int64), POINTER(c_double),
                                    POINTER(c_int), POINTER(c_double)]),
    "sr_bin": (c_int, [c_void_p, c_void_p, c_int64, c_void_p]),
    "sr_force": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sr_force_plain": (c_int, [c_void_p, c_void_p, c_void_p]),
    "sr_force_kick": (c_int, [c_void_p, c_void_p, c_void_p, c_float, c_void_p]),
    "sr_leapfrog": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_int, c_int64, c_void_p]),
    "sr_force_vjp": (c_int, [c_void_p, c_void_p, c_void_p, c_float, c_int, c_void_p]),
    "sr_kick": (c_int, [c_int64, c_void_p, c_void_p, c_float, c_void_p]),
    "sr_drift": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int64, c_void_p]),
    "sr_invariants": (c_int, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sr_invariants_noalloc": (c_int, [c_int64, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sr_plan_status": (c_int, [c_void_p, c_void_p]),
    "sr_plan_copy": (c_int, [c_void_p, c_int, c_void_p, c_int64, c_void_p]),
    "sr_step_host": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_int64, c_void_p]),
    "sr_step_host_submit": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_int64, c_void_p]),
    "sr_step_host_wait": (c_int, [c_void_p]),
    "sr_plan_set_variant": (c_int, [c_void_p, c_int]),
    "sr_autotune": (c_int, [c_void_p, c_void_p, c_int, POINTER(c_float), c_void_p]),
    "sr_bin_active": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p]),
    "sr_variant_count": (c_int, []),
    "sr_plan_tune": (c_int, [POINTER(SrParams), c_int64, c_void_p, c_int64, c_int, POINTER(c_void_p),
                             POINTER(SrTuneEntry), POINTER(c_int), c_void_p]),
    "sr_build_checked": (c_int, []),
    "sr_check_selftest": (c_int, [c_void_p, c_void_p]),
    "sr_graph_capture": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_int64, c_void_p]),
    "sr_graph_launch": (c_int, [c_void_p, c_void_p]),
    "sr_centers_create": (c_int, [c_int64, ctypes.c_int32, POINTER(c_void_p)]),
    "sr_centers_destroy": (c_int, [c_void_p]),
    "sr_centers_set_variant": (c_int, [c_void_p, c_int]),
    "sr_centers_run": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, ctypes.c_int32, c_double, c_double,
                               c_void_p, c_void_p, c_void_p, c_void_p]),
    "sr_centers_prepare": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, ctypes.c_int32, c_double,
                                   c_double, c_void_p]),
    "sr_centers_potential": (c_int, [c_void_p, c_void_p]),
    "sr_centers_finish": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sr_centers_get_info": (c_int, [c_void_p, POINTER(SrCentersInfo)]),
    "sr_pm_create": (c_int, [c_int, c_double, c_double, c_int64, POINTER(c_void_p)]),
    "sr_pm_destroy": (c_int, [c_void_p]),
    "sr_pm_deposit": (c_int, [c_void_p, c_void_p, c_int64, c_void_p]),
    "sr_pm_deposit_binned": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p]),
    "sr_pm_transform": (c_int, [c_void_p, c_void_p]),
    "sr_pm_power": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sr_pm_force": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_int, c_void_p]),
    "sr_pm_fft": (c_int, [c_void_p, c_void_p, c_int, c_void_p]),
    "sr_pm_copy": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "sr_fof_create": (c_int, [c_int64, POINTER(c_void_p)]),
    "sr_fof_destroy": (c_int, [c_void_p]),
    "sr_fof_run": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_double, c_int, c_void_p, c_void_p, c_void_p]),
    "sr_fof_get_info": (c_int, [c_void_p, POINTER(SrFofInfo)]),
    "sr_fof_set_iteration_limit": (c_int, [c_void_p, c_int64]),
    "sr_last_error": (c_char_p, []),
    "sr_launch_count": (c_int64, []),
}

_lib = None


def load():
    """Load libsr_b300.so (built in-tree by __graft_entry__.build()), or the
    bounds-checked libsr_b300_check.so when SR_B300_CHECKED=1 is set in the
    environment of the process before the first call."""
    global _lib
    if _lib is None:
        path = LIB_CHECKED if os.environ.get("SR_B300_CHECKED") == "1" else LIB
        if not path.exists():
            raise RuntimeError(f"{path.name} is not built; run __graft_entry__.build() first")
        lib = ctypes.CDLL(str(path))
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(code: int):
    if code != SR_OK:
        msg = load().sr_last_error().decode(errors="replace")
        raise SrError(code, msg)
