"""Python face of the long-range side (include/sr_pm.h): CIC deposit, 3-d
FFT, CIC-compensated power spectrum and the Gaussian-filtered PM
acceleration, computed by the library's kernels.  Argument marshalling only."""
from __future__ import annotations

from ctypes import byref, c_void_p

import torch

from ._lib import check, load
from .api import _ptr, _stream

EXPORTS = {"counts": 0, "delta_k": 1, "accel": 2}


def _check_pos(pos):
    if not (isinstance(pos, torch.Tensor) and pos.is_cuda and pos.dtype == torch.float64 and pos.dim() == 2
            and pos.shape[1] == 3 and pos.is_contiguous()):
        raise TypeError("pos must be a contiguous CUDA float64 (n, 3) tensor")


class PM:
    """Workspace for an n_grid^3 mesh of a periodic box (split scale sigma)."""

    def __init__(self, n_grid: int, box: float, sigma: float, n_max: int):
        lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        h = c_void_p()
        check(lib.sr_pm_create(int(n_grid), float(box), float(sigma), int(n_max), byref(h)))
        self._h = h
        self.n_grid, self.box, self.sigma = int(n_grid), float(box), float(sigma)

    def close(self):
        if self._h:
            load().sr_pm_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def deposit(self, pos: torch.Tensor, transform: bool = True, plan=None):
        """CIC counts of pos; with transform, also delta and its FFT (the
        input of power() and force()).  With plan (a one-volume Plan that
        binned these positions, same box), the deposit runs over the plan's
        cell order with on-chip tiles (sr_pm_deposit_binned): the same bits."""
        _check_pos(pos)
        if plan is None:
            check(load().sr_pm_deposit(self._h, _ptr(pos), int(pos.shape[0]), _stream()))
        else:
            check(load().sr_pm_deposit_binned(self._h, plan._h, _ptr(pos), int(pos.shape[0]), _stream()))
        if transform:
            self.transform()

    def transform(self):
        check(load().sr_pm_transform(self._h, _stream()))

    def power(self):
        """(k_mean, P, modes) per shell b = 1 .. n_grid/2 (device tensors)."""
        nb = self.n_grid // 2
        dev = torch.device("cuda", torch.cuda.current_device())
        k = torch.empty(nb, dtype=torch.float64, device=dev)
        p = torch.empty(nb, dtype=torch.float64, device=dev)
        m = torch.empty(nb, dtype=torch.int64, device=dev)
        check(load().sr_pm_power(self._h, _ptr(k), _ptr(p), _ptr(m), _stream()))
        return k, p, m

    def force(self, pos: torch.Tensor, acc: torch.Tensor | None = None, accumulate: bool = False):
        _check_pos(pos)
        n = pos.shape[0]
        if acc is None:
            acc = torch.zeros((n, 4), dtype=torch.float32, device=pos.device)
        if not (acc.is_cuda and acc.dtype == torch.float32 and acc.shape == (n, 4) and acc.is_contiguous()):
            raise TypeError("acc must be a contiguous CUDA float32 (n, 4) tensor")
        check(load().sr_pm_force(self._h, _ptr(pos), int(n), _ptr(acc), int(bool(accumulate)), _stream()))
        return acc

    def fft(self, data: torch.Tensor, inverse: bool = False):
        """In-place 3-d FFT of a complex64 (n, n, n) CUDA tensor."""
        g = self.n_grid
        if not (data.is_cuda and data.dtype == torch.complex64 and data.shape == (g, g, g) and data.is_contiguous()):
            raise TypeError(f"data must be a contiguous CUDA complex64 ({g}, {g}, {g}) tensor")
        check(load().sr_pm_fft(self._h, _ptr(data), int(bool(inverse)), _stream()))
        return data

    def export(self, name: str) -> torch.Tensor:
        g = self.n_grid
        dev = torch.device("cuda", torch.cuda.current_device())
        if name == "counts":
            out = torch.empty((g, g, g), dtype=torch.float64, device=dev)
        elif name == "delta_k":
            out = torch.empty((g, g, g), dtype=torch.complex64, device=dev)
        else:
            out = torch.empty((g, g, g, 4), dtype=torch.float32, device=dev)
        check(load().sr_pm_copy(self._h, EXPORTS[name], _ptr(out), _stream()))
        return out
