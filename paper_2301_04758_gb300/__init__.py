"""GB300 (sm_103a) DG S_N transport sweep and VEF closure pass.

Data-parallel hot path of the VEF method of Olivier & Haut (high-order mixed finite
element Variable Eddington Factor methods): the upwind DG discrete-ordinates sweep on
curved quadrilaterals, the angular moments and closures (phi, J, E, E_b, J_in), source
iteration and an adjoint sweep, all in hand-written CUDA behind the C ABI of
include/vef.h (libvef.so).  Python here only marshals arguments.
"""
from . import _lib  # noqa: F401

__all__ = ["_lib"]
