"""Python face of the library: tensors in, C ABI calls, tensors out.

PyTorch only supplies device memory and the current CUDA stream; every step
of the short-range path (binning, sorting, pair sums, kick, drift, VJP,
invariants) runs in the library's own kernels.  There is no CPU fallback:
without the native library or a CUDA device these calls raise.
"""
from __future__ import annotations

import ctypes
from ctypes import byref, c_double, c_int, c_int64, c_void_p

import torch

from . import _lib
from ._lib import EXPORTS, FIT_MODES, SrParams, SrPlanInfo, check, load


def _stream():
    return c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor | None):
    return c_void_p(t.data_ptr()) if t is not None else c_void_p(0)


def _need(t: torch.Tensor, dtype, cols: int, name: str, n: int | None = None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.dim() != 2 or t.shape[1] != cols or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous (n, {cols}) tensor")
    if n is not None and t.shape[0] != n:
        raise ValueError(f"{name} must have {n} rows, got {t.shape[0]}")


def fit_poly(r_c: float, sigma: float, eps: float, mode: str = "constrained"):
    """Binary64 coefficients c[0..5] of p(s) (host computation in the library)."""
    out = (c_double * 6)()
    check(load().sr_fit_poly(r_c, sigma, eps, FIT_MODES[mode], out))
    return list(out)


def launch_count() -> int:
    return int(load().sr_launch_count())


def kick(acc: torch.Tensor, vel: torch.Tensor, dt: float):
    """vel[:, :3] += acc[:, :3] * dt (float4 rows)."""
    _need(acc, torch.float32, 4, "acc")
    _need(vel, torch.float32, 4, "vel", acc.shape[0])
    check(load().sr_kick(acc.shape[0], _ptr(acc), _ptr(vel), float(dt), _stream()))
    return vel


def _params(box, r_c, eps, sigma, fit_mode, n_cells, sub_bits, chunk_size):
    return SrParams(float(box), float(r_c), float(eps), float(sigma), FIT_MODES[fit_mode],
                    int(n_cells), int(sub_bits), int(chunk_size))


class Plan:
    """A binning + force plan for one periodic volume, or a batch of them."""

    def __init__(self, box: float, r_c: float, eps: float, sigma: float, n_max: int,
                 fit_mode: str = "constrained", n_cells: int = 0, sub_bits: int = 0,
                 chunk_size: int = 0, _batch=None):
        lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        handle = c_void_p()
        if _batch is None:
            prm = _params(box, r_c, eps, sigma, fit_mode, n_cells, sub_bits, chunk_size)
            check(lib.sr_plan_create(byref(prm), int(n_max), byref(handle)))
            self.volume_counts = [int(n_max)]
        else:
            boxes, counts, cells = _batch
            arr = (SrParams * len(boxes))(*[_params(b, r_c, eps, sigma, fit_mode, nc, sub_bits, chunk_size)
                                            for b, nc in zip(boxes, cells)])
            ns = (c_int64 * len(counts))(*[int(c) for c in counts])
            check(lib.sr_plan_batch(arr, ns, len(boxes), byref(handle)))
            self.volume_counts = [int(c) for c in counts]
        self._h = handle
        self.r_c, self.eps, self.sigma = float(r_c), float(eps), float(sigma)
        self.capacity = sum(self.volume_counts) if _batch is not None else int(n_max)
        self.n = None
        self.binnings = 0           # calls that replaced the plan's binning

    @classmethod
    def tune(cls, box: float, r_c: float, eps: float, sigma: float, pos: torch.Tensor, n_max: int | None = None,
             reps: int = 1, fit_mode: str = "constrained", sub_bits: int = 0):
        """A plan whose chunk size, cell count and kernel variant are chosen by
        timing on pos (sr_plan_tune); returns (plan, candidates), each
        candidate a dict of chunk_size, n_cells, variant, ms.  The plan is
        binned on pos."""
        lib = load()
        _need(pos, torch.float64, 3, "pos")
        n = pos.shape[0]
        n_max = int(n_max or n)
        prm = _params(box, r_c, eps, sigma, fit_mode, 0, sub_bits, 0)
        ents = (_lib.SrTuneEntry * 8)()
        cnt = c_int(0)
        handle = c_void_p()
        check(lib.sr_plan_tune(byref(prm), n_max, _ptr(pos), n, int(reps), byref(handle), ents, byref(cnt),
                               _stream()))
        plan = cls.__new__(cls)
        plan._h = handle
        plan.volume_counts = [n_max]
        plan.r_c, plan.eps, plan.sigma = float(r_c), float(eps), float(sigma)
        plan.capacity = n_max
        plan.n = n
        plan.binnings = 1
        cands = [{k: getattr(ents[i], k) for k, _ in _lib.SrTuneEntry._fields_} for i in range(cnt.value)]
        return plan, cands

    @classmethod
    def batch(cls, boxes, counts, r_c, eps, sigma, fit_mode="constrained", n_cells=None,
              sub_bits=0, chunk_size=0):
        cells = n_cells if n_cells is not None else [0] * len(boxes)
        return cls(0.0, r_c, eps, sigma, 0, fit_mode, 0, sub_bits, chunk_size, _batch=(boxes, counts, cells))

    # -- lifecycle -----------------------------------------------------------
    def close(self):
        if self._h:
            load().sr_plan_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        inf = SrPlanInfo()
        check(load().sr_plan_get_info(self._h, byref(inf)))
        d = {k: getattr(inf, k) for k, _ in SrPlanInfo._fields_ if k != "coef"}
        d["coef"] = list(inf.coef)
        return d

    def volume(self, v: int) -> dict:
        n, box, nc, h = c_int64(), c_double(), c_int(), c_double()
        check(load().sr_plan_volume_info(self._h, int(v), byref(n), byref(box), byref(nc), byref(h)))
        return dict(n=n.value, box=box.value, n_cells=nc.value, h=h.value)

    # -- hot path ------------------------------------------------------------
    def bin(self, pos: torch.Tensor, active: torch.Tensor | None = None):
        """Bin pos (n, 3) binary64.  active: optional (n,) bool or uint8 mask
        of the particles whose forces are wanted (sr_bin_active); the others
        are neighbours only, and their output rows are left untouched."""
        _need(pos, torch.float64, 3, "pos")
        if active is None:
            check(load().sr_bin(self._h, _ptr(pos), pos.shape[0], _stream()))
        else:
            if active.dtype not in (torch.bool, torch.uint8) or active.shape != (pos.shape[0],) \
                    or not active.is_cuda or not active.is_contiguous():
                raise ValueError("active must be a contiguous CUDA bool/uint8 tensor of shape (n,)")
            check(load().sr_bin_active(self._h, _ptr(pos), _ptr(active), pos.shape[0], _stream()))
        self.n = pos.shape[0]
        self.binnings += 1
        return self

    def force(self, acc: torch.Tensor | None = None, count: bool = False, per_particle=False):
        """Accelerations (n, 4) float32; with count/per_particle also the
        in-range pair total (uint64 device scalar) / per-particle counts
        (per_particle: True, or an (n,) int32 CUDA tensor to write into)."""
        n = self._need_binned()
        if acc is None:
            acc = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        _need(acc, torch.float32, 4, "acc", n)
        pairs = torch.zeros(1, dtype=torch.int64, device="cuda") if count else None
        if isinstance(per_particle, torch.Tensor):
            if per_particle.dtype != torch.int32 or per_particle.shape != (n,) or not per_particle.is_cuda \
                    or not per_particle.is_contiguous():
                raise ValueError("per_particle must be a contiguous CUDA int32 tensor of shape (n,)")
            pp = per_particle
        else:
            pp = torch.empty(n, dtype=torch.int32, device="cuda") if per_particle else None
        check(load().sr_force(self._h, _ptr(acc), _ptr(pairs), _ptr(pp), _stream()))
        if count or per_particle:
            return acc, pairs, pp
        return acc

    def force_kick(self, acc: torch.Tensor, vel: torch.Tensor, dt: float):
        """Accelerations with the kick fused into the epilogue (vel updated)."""
        n = self._need_binned()
        _need(acc, torch.float32, 4, "acc", n)
        _need(vel, torch.float32, 4, "vel", n)
        check(load().sr_force_kick(self._h, _ptr(acc), _ptr(vel), float(dt), _stream()))
        return acc

    def leapfrog(self, pos: torch.Tensor, vel: torch.Tensor, acc: torch.Tensor, dt: float, steps: int):
        """KDK leapfrog steps in place; acc must hold a(pos) on entry."""
        _need(pos, torch.float64, 3, "pos")
        n = pos.shape[0]
        _need(vel, torch.float32, 4, "vel", n)
        _need(acc, torch.float32, 4, "acc", n)
        check(load().sr_leapfrog(self._h, _ptr(pos), _ptr(vel), _ptr(acc), float(dt), int(steps), n, _stream()))
        self.n = n
        self.binnings += 1
        return pos, vel, acc

    def force_plain(self, acc: torch.Tensor | None = None):
        n = self._need_binned()
        if acc is None:
            acc = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        _need(acc, torch.float32, 4, "acc", n)
        check(load().sr_force_plain(self._h, _ptr(acc), _stream()))
        return acc

    def vjp(self, g_acc: torch.Tensor, g_pos: torch.Tensor | None = None, g_scale: float = 1.0,
            accumulate: bool = False):
        n = self._need_binned()
        _need(g_acc, torch.float32, 4, "g_acc", n)
        if g_pos is None:
            g_pos = torch.empty((n, 4), dtype=torch.float32, device="cuda")
            accumulate = False
        _need(g_pos, torch.float32, 4, "g_pos", n)
        check(load().sr_force_vjp(self._h, _ptr(g_acc), _ptr(g_pos), float(g_scale),
                                  1 if accumulate else 0, _stream()))
        return g_pos

    def drift(self, pos: torch.Tensor, vel: torch.Tensor, dt: float):
        _need(pos, torch.float64, 3, "pos")
        _need(vel, torch.float32, 4, "vel", pos.shape[0])
        check(load().sr_drift(self._h, _ptr(pos), _ptr(vel), float(dt), pos.shape[0], _stream()))
        return pos

    def invariants(self, vel: torch.Tensor | None, acc: torch.Tensor | None, out=None):
        n = (vel if vel is not None else acc).shape[0]
        if vel is not None:
            _need(vel, torch.float32, 4, "vel", n)
        if acc is not None:
            _need(acc, torch.float32, 4, "acc", n)
        if out is None:
            out = torch.empty(7, dtype=torch.float64, device="cuda")
        check(load().sr_invariants(self._h, n, _ptr(vel), _ptr(acc), _ptr(out), _stream()))
        return out

    def set_variant(self, v: int):
        check(load().sr_plan_set_variant(self._h, int(v)))

    def autotune(self, reps: int = 2):
        """Time the pair-kernel variants on the current binning; keeps the
        fastest and returns the per-variant mean times (ms)."""
        n = self._need_binned()
        acc = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        ms = (ctypes.c_float * load().sr_variant_count())()
        check(load().sr_autotune(self._h, _ptr(acc), int(reps), ms, _stream()))
        return list(ms)

    def graph_capture(self, pos: torch.Tensor, vel: torch.Tensor, acc: torch.Tensor, dt: float):
        """Capture bin + force + kick on the current (non-default) stream into
        a plan-owned CUDA graph; replay with graph_launch()."""
        _need(pos, torch.float64, 3, "pos")
        _need(vel, torch.float32, 4, "vel", pos.shape[0])
        _need(acc, torch.float32, 4, "acc", pos.shape[0])
        check(load().sr_graph_capture(self._h, _ptr(pos), _ptr(vel), _ptr(acc), float(dt), pos.shape[0],
                                      _stream()))
        self.n = pos.shape[0]
        self.binnings += 1

    def graph_launch(self):
        check(load().sr_graph_launch(self._h, _stream()))
        self.binnings += 1

    def status(self):
        check(load().sr_plan_status(self._h, _stream()))

    def export(self, name: str) -> torch.Tensor:
        """Copy an internal array of the last bin to a new device tensor."""
        inf = self.info()
        n, nch, cells = inf["n_particles"], inf["n_chunks"], inf["total_cells"]
        spec = {
            "perm": (torch.int32, (n,)), "cell_start": (torch.int32, (cells + 1,)),
            "cell_chunk_start": (torch.int32, (cells + 1,)),
            "slot_pos": (torch.float32, (nch * inf["chunk_size"], 4)),
            "slot_idx": (torch.int32, (nch * inf["chunk_size"],)),
            "chunk_meta": (torch.int32, (nch, 4)), "chunk_lo": (torch.float32, (nch, 4)),
            "chunk_hi": (torch.float32, (nch, 4)), "order": (torch.int32, (nch,)),
            "cost": (torch.int32, (nch,)), "counters": (torch.int64, (8,)),
        }[name]
        out = torch.empty(spec[1], dtype=spec[0], device="cuda")
        check(load().sr_plan_copy(self._h, EXPORTS[name], _ptr(out), out.numel() * out.element_size(),
                                  _stream()))
        return out

    def step_host(self, pos, vel, acc, dt: float):
        """Whole step from host (numpy/torch CPU) buffers: H2D, bin, force,
        kick, D2H.  pos (n,3) float64, vel (n,4) float32 updated in place,
        acc (n,4) float32 written (or None)."""
        n = pos.shape[0]
        check(load().sr_step_host(self._h, c_void_p(pos.data_ptr()), c_void_p(vel.data_ptr()),
                                  c_void_p(acc.data_ptr()) if acc is not None else c_void_p(0),
                                  float(dt), n, _stream()))
        self.n = n
        self.binnings += 1

    def step_host_submit(self, pos, vel, acc, dt: float):
        """step_host for a stream of independent inputs, without waiting:
        the uploads of this step overlap the step before it, its read-back
        the step after it.  pos, vel and acc (or None) are page-locked CPU
        tensors that must stay untouched until step_host_wait() returns (or
        two submits later); vel is overwritten with the kicked velocities."""
        n = pos.shape[0]
        check(load().sr_step_host_submit(self._h, c_void_p(pos.data_ptr()), c_void_p(vel.data_ptr()),
                                         c_void_p(acc.data_ptr()) if acc is not None else c_void_p(0),
                                         float(dt), n, _stream()))
        self.n = n
        self.binnings += 1

    def step_host_wait(self):
        """Block until every submitted step's results are in host memory."""
        check(load().sr_step_host_wait(self._h))

    def _need_binned(self) -> int:
        if self.n is None:
            raise RuntimeError("bin() must be called first")
        return self.n
