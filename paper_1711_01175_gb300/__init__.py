"""GB300-native hot path of the upwind DG/HDG velocity-stress elastic-wave operator.

``libdgw.so`` (CUDA, sm_103a) computes the per-stage semi-discrete right-hand
side -- split-form volume term on curvilinear hexahedra, face gather with the
upwind HDG flux, diagonal GLL lift, Q^{-1} -- fused with the low-storage
Runge-Kutta stage update, plus the discrete energy.  ``capi`` is the ctypes
binding of its C ABI (include/dgw.h); ``Solver`` marshals torch tensors or
numpy arrays to it.
"""
from .capi import DGWError, load
from .solver import Solver, reference_nodes

__all__ = ["DGWError", "Solver", "load", "reference_nodes"]
