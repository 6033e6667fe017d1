"""Python face of the friends-of-friends halo finder (include/sr_fof.h),
computed by the library's kernels on a binned plan.  Argument marshalling
only."""
from __future__ import annotations

from ctypes import byref, c_void_p

import torch

from ._lib import SrFofInfo, check, load
from .api import _ptr, _stream


class FOF:
    """Workspace for friends-of-friends on up to n_max particles."""

    def __init__(self, n_max: int):
        lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        h = c_void_p()
        check(lib.sr_fof_create(int(n_max), byref(h)))
        self._h = h

    def close(self):
        if self._h:
            load().sr_fof_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, plan, pos: torch.Tensor, link: float, min_members: int = 40,
            labels: torch.Tensor | None = None, halo_sizes: torch.Tensor | None = None):
        """Labels (int32, caller order, -1 outside halos) and the per-halo
        sizes buffer (int32, entries < n_halos valid) of the particles the
        plan was last binned with."""
        if not (pos.is_cuda and pos.dtype == torch.float64 and pos.dim() == 2 and pos.shape[1] == 3
                and pos.is_contiguous()):
            raise TypeError("pos must be a contiguous CUDA float64 (n, 3) tensor")
        n = pos.shape[0]
        if labels is None:
            labels = torch.empty(n, dtype=torch.int32, device=pos.device)
        if halo_sizes is None:
            halo_sizes = torch.empty(max(n, 1), dtype=torch.int32, device=pos.device)
        check(load().sr_fof_run(self._h, plan._h, _ptr(pos), int(n), float(link), int(min_members),
                                _ptr(labels), _ptr(halo_sizes), _stream()))
        return labels, halo_sizes

    def set_iteration_limit(self, max_iter: int = 0):
        """Bound of the union-find loops (0 = default); a tiny bound makes
        them run out, which get_info reports as SR_ERR_TIMEOUT."""
        check(load().sr_fof_set_iteration_limit(self._h, int(max_iter)))

    def info(self) -> dict:
        """Counts of the last run; raises SrError (SR_ERR_TIMEOUT) if a
        union-find loop ran out of iterations."""
        inf = SrFofInfo()
        check(load().sr_fof_get_info(self._h, byref(inf)))
        return {k: getattr(inf, k) for k, _ in SrFofInfo._fields_}
