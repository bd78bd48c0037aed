"""CPU oracle (test infrastructure only).

Plain FP64 implementations that the CUDA library is checked against.  Only the
test suite, the smoke check and the benchmark's CPU-baseline leg use it; the
library never imports it.
"""
from .dg_elastic import (ElasticDG, gll, lagrange_derivative_matrix, legendre, A_of, B_of, abs_A, abs_A_Q,
                         Q_of, stiffness_voigt, weighted_trace, hdg_flux, LSRK_A, LSRK_B, LSRK_C,
                         cfl_dt, cfl_number, face_node_indices, neighbour_face_position,
                         h_min_corner_edges, ricker, lagrange_values)
from .dg_friedrichs import FriedrichsSystem, FriedrichsDG, transport, shallow_water
