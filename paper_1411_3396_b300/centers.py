"""Python face of the halo center finder (include/sr_centers.h): the
potential of every halo member and each halo's most bound particle (Sec. 2.2),
computed by the library's kernels.  Argument marshalling only."""
from __future__ import annotations

from ctypes import byref, c_void_p

import torch

from ._lib import SrCentersInfo, check, load
from .api import _ptr, _stream

VARIANTS = {"symmetric": 0, "plain": 1}


def _check_inputs(pos, labels):
    if not (pos.is_cuda and pos.dtype == torch.float64 and pos.dim() == 2 and pos.shape[1] == 3
            and pos.is_contiguous()):
        raise TypeError("pos must be a contiguous CUDA float64 (n, 3) tensor")
    if not (labels.is_cuda and labels.dtype == torch.int32 and labels.shape == (pos.shape[0],)
            and labels.is_contiguous()):
        raise TypeError("labels must be a contiguous CUDA int32 (n,) tensor")


class Centers:
    """Workspace for up to n_max particles in up to n_halos_max halos."""

    def __init__(self, n_max: int, n_halos_max: int, variant: str = "symmetric"):
        lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        h = c_void_p()
        check(lib.sr_centers_create(int(n_max), int(n_halos_max), byref(h)))
        self._h = h
        self.set_variant(variant)

    def close(self):
        if self._h:
            load().sr_centers_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_variant(self, variant: str):
        check(load().sr_centers_set_variant(self._h, VARIANTS[variant]))
        self.variant = variant

    def run(self, pos: torch.Tensor, labels: torch.Tensor, n_halos: int, box: float, eps: float,
            phi: torch.Tensor | None = None, center: torch.Tensor | None = None,
            center_phi: torch.Tensor | None = None, want_phi: bool = True):
        """Returns (phi (n,) float64 or None, center (n_halos,) int64, center_phi (n_halos,) float64)."""
        _check_inputs(pos, labels)
        n = pos.shape[0]
        dev = pos.device
        if phi is None and want_phi:
            phi = torch.empty(n, dtype=torch.float64, device=dev)
        if center is None:
            center = torch.empty(int(n_halos), dtype=torch.int64, device=dev)
        if center_phi is None:
            center_phi = torch.empty(int(n_halos), dtype=torch.float64, device=dev)
        check(load().sr_centers_run(self._h, _ptr(pos), _ptr(labels), int(n), int(n_halos), float(box),
                                    float(eps), _ptr(phi), _ptr(center), _ptr(center_phi), _stream()))
        return phi, center, center_phi

    def prepare(self, pos: torch.Tensor, labels: torch.Tensor, n_halos: int, box: float, eps: float):
        _check_inputs(pos, labels)
        check(load().sr_centers_prepare(self._h, _ptr(pos), _ptr(labels), int(pos.shape[0]), int(n_halos),
                                        float(box), float(eps), _stream()))
        self.n, self.n_halos = int(pos.shape[0]), int(n_halos)

    def potential(self):
        check(load().sr_centers_potential(self._h, _stream()))

    def finish(self, phi=None, center=None, center_phi=None):
        check(load().sr_centers_finish(self._h, _ptr(phi), _ptr(center), _ptr(center_phi), _stream()))
        return phi, center, center_phi

    def info(self) -> dict:
        inf = SrCentersInfo()
        check(load().sr_centers_get_info(self._h, byref(inf)))
        return {k: getattr(inf, k) for k, _ in SrCentersInfo._fields_}
