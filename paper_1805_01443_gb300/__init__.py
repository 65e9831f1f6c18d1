"""GB300-native (sm_103a) discontinuous-Galerkin operator of arXiv:1805.01443.

The hot path -- the per-stage DG spatial operator for the 2D Euler equations
with star + planet gravity on a Cartesian mesh, tensor-product Legendre modal
basis up to p = 4, SSP-RK stage update, damping zones and the planet torque --
is hand-written CUDA behind the C ABI of include/dg.h (libdg.so).  `dg` is the
ctypes binding; `inputs` holds the seeded synthetic workloads.
"""
from . import inputs  # noqa: F401
