"""GB300 (sm_103a) point-based ray tracing of 3D Gaussians: LBVH build,
visibility trace, adjoint, learned visibility surrogate and batched launches
behind the C ABI of include/rt3dg.h.  ``rt`` holds the ctypes binding."""
from . import rt  # noqa: F401

__all__ = ["rt"]
