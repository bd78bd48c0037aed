"""Seeded synthetic inputs for the DG elastic-wave hot path.

This package is the one piece of code that both the CUDA library's tests/bench
and the CPU oracle use.  It holds no arithmetic of the discretisation itself:
it builds mesh topology, node coordinates at caller-supplied reference nodes,
material fields and initial data.  The paper's workloads are structured
hexahedral meshes of the unit cube with smooth exact solutions (Section 6,
numerical results); these generators make inputs of that shape.
"""
from .mesh import (Mesh, structured_hex_mesh, warped_node_coords, BC_INTERIOR,
                   BC_FREE_SURFACE, BC_ABSORBING, BC_WALL, rotate_elements)
from .material import smooth_random_material, homogeneous_material
from .fields import (plane_p_wave, gaussian_stress_pulse, random_state, transport_periodic, transport_gaussian,
                     shallow_water_standing_wave, random_fields)
from .configs import parity_config, large_config, precision_config
from .serving import Request, make_requests

__all__ = [
    "Mesh", "structured_hex_mesh", "warped_node_coords", "rotate_elements",
    "BC_INTERIOR", "BC_FREE_SURFACE", "BC_ABSORBING", "BC_WALL",
    "smooth_random_material", "homogeneous_material",
    "plane_p_wave", "gaussian_stress_pulse", "random_state", "transport_periodic", "transport_gaussian",
    "shallow_water_standing_wave", "random_fields",
    "parity_config", "large_config", "precision_config", "Request", "make_requests",
]
