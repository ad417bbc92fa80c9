"""GB300-native (sm_103a) bonded-particle model for magneto-elastic rods.

One timestep of the model of arXiv 2603.27279 -- co-rotational bond forces
and torques, Zeeman and all-pairs dipole-dipole interactions, velocity
Verlet with the Richardson quaternion update -- as hand-written CUDA kernels
behind the C ABI of include/bpm.h.  ``bpm`` is the Python binding,
``workloads`` the seeded synthetic systems.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "bpm", "build", "adjoint"]
