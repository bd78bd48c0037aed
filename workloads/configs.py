"""Named workloads (sizes, boundary tags, material and initial data recipes).

* parity:    4^3 periodic cube, N=3, warp amplitude 0.05, homogeneous
             rho=1, lambda=2, mu=1, plane P-wave along (1,1,0), upwind flux,
             CFL 0.5, 100 steps.
* large:     64^3 cube, N=4, warp amplitude 0.1, smooth random medium
             (seed 1), Gaussian stress pulse, x/y periodic, z=0 absorbing,
             z=1 free surface, CFL 0.5, 1000 steps.  Elements in Morton order.
* precision: 48^3 cube, N=7, same recipe with material seed 2, to T = 1.
Smaller cuts of ``large`` (same recipe, fewer elements) serve as parity cases.
"""
from __future__ import annotations

from dataclasses import dataclass, field

from .mesh import (structured_hex_mesh, warped_node_coords, BC_ABSORBING, BC_FREE_SURFACE)
from .material import smooth_random_material, homogeneous_material
from .fields import plane_p_wave, gaussian_stress_pulse


@dataclass(frozen=True)
class Workload:
    name: str
    E: int
    N: int
    amplitude: float
    periodic: tuple
    boundary: dict = field(default_factory=dict)
    material: str = "homogeneous"        # or "random"
    material_seed: int = 0
    initial: str = "plane_p_wave"        # or "gaussian_pulse"
    tau: int = 1                         # 1 upwind, 0 central
    cfl: float = 0.5
    steps: int = 100
    order: str = "lex"

    def build(self, r1d):
        """Arrays for this workload at the 1-D reference nodes ``r1d`` (length N+1)."""
        if len(r1d) != self.N + 1:
            raise ValueError("reference nodes must have N+1 entries")
        mesh = structured_hex_mesh(self.E, self.periodic, self.boundary, self.order)
        x = warped_node_coords(mesh, r1d, self.amplitude)
        if self.material == "homogeneous":
            rho, lam, mu = homogeneous_material(mesh.nel, 1.0, 2.0, 1.0)
        else:
            rho, lam, mu = smooth_random_material(mesh, self.material_seed)
        if self.initial == "plane_p_wave":
            u0 = plane_p_wave(x, 1.0, 2.0, 1.0)
        else:
            u0 = gaussian_stress_pulse(x)
        return dict(mesh=mesh, x=x, rho=rho, lam=lam, mu=mu, u0=u0)


def parity_config() -> Workload:
    return Workload("parity-4^3-N3", 4, 3, 0.05, (True, True, True))


def large_config(E: int = 64, N: int = 4, steps: int = 1000) -> Workload:
    return Workload(f"large-{E}^3-N{N}", E, N, 0.1, (True, True, False),
                    {4: BC_ABSORBING, 5: BC_FREE_SURFACE}, "random", 1,
                    "gaussian_pulse", 1, 0.5, steps, "morton")


def precision_config(E: int = 48, N: int = 7) -> Workload:
    return Workload(f"precision-{E}^3-N{N}", E, N, 0.1, (True, True, False),
                    {4: BC_ABSORBING, 5: BC_FREE_SURFACE}, "random", 2,
                    "gaussian_pulse", 1, 0.5, 0, "morton")
