"""B300 short-range particle-particle force library (Q Continuum / HACC method).

The hot path -- cell binning, stable counting sort, the persistent pair
kernel with compensated accumulation, the kick, the drift and the force
VJP -- the friends-of-friends halo finder, the halo center finder and the
long-range PM / power-spectrum side run in the CUDA kernels of
``libsr_b300.so`` (sources in ``csrc/``, C ABI in ``include/sr.h``,
``include/sr_fof.h``, ``include/sr_centers.h`` and ``include/sr_pm.h``).
This package only marshals tensors; ``decomp`` adds the overload slab
decomposition of one volume over ranks (selection and exchange in
PyTorch / torch.distributed around those kernels).
"""
from .api import Plan, fit_poly, kick, launch_count  # noqa: F401
from .centers import Centers  # noqa: F401
from .pm import PM  # noqa: F401
from .fof import FOF  # noqa: F401
from .decomp import Slabs, slab_bounds  # noqa: F401
from .autograd import TrajectoryGraph, trajectory  # noqa: F401
from ._lib import SrError  # noqa: F401
from .build import LIB, build  # noqa: F401
