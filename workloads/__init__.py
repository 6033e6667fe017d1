"""Seeded synthetic particle sets shared by the oracle side and the CUDA side.

This package generates inputs only: positions, velocities, cotangents and
the physics parameters of each named workload.  It holds none of the
short-range force method's arithmetic (no binning, no pair sums, no
polynomial fit), so both the FP64 oracle and the GPU path may import it
without sharing any of the method with each other.
"""
from .generators import (  # noqa: F401
    uniform_box,
    lattice,
    zeldovich,
    nfw_clustered,
    batch_volumes,
    two_body,
    random_directions,
)
from .configs import CONFIGS, make_workload, small_variant  # noqa: F401
