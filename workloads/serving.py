"""Seeded request streams for the serving loop.

Each request is a separate wave solve: a structured cube mesh of E^3
elements (E log-uniform in a range), degree N, its own smooth random medium,
a Ricker point force at a reference point of the centre element, zero initial
state, and a number of LSRK steps (even: the batch advances step pairs).
Arrivals form a Poisson process.  The point force's peak frequency gives five
S-wavelengths across the unit domain at the medium's mean shear speed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .mesh import structured_hex_mesh, warped_node_coords, BC_ABSORBING, BC_FREE_SURFACE
from .material import smooth_random_material


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    E: int
    N: int
    steps: int              # even
    material_seed: int
    xi: tuple
    force: tuple
    payload: dict = field(default_factory=dict, repr=False)

    def build(self, r1d):
        """Mesh, node coordinates (at the reference nodes r1d), medium and point force."""
        mesh = structured_hex_mesh(self.E, (True, True, False), {4: BC_ABSORBING, 5: BC_FREE_SURFACE}, "morton")
        x = warped_node_coords(mesh, r1d, 0.1)
        rho, lam, mu = smooth_random_material(mesh, self.material_seed)
        cs_mean = float(np.mean(np.sqrt(mu / rho)))
        f0 = 5.0 * cs_mean
        centre = np.nonzero(np.all(mesh.cell == self.E // 2, axis=1))[0][0]
        src = dict(element=int(centre), xi=list(self.xi), force=list(self.force), f0=f0, t0=1.2 / f0)
        return dict(mesh=mesh, x=x, rho=rho, lam=lam, mu=mu, source=src)


def make_requests(count, seed, rate, E_range=(8, 48), N_choices=(3, 4, 5), steps_range=(200, 2000)):
    """`count` requests with Poisson arrivals of `rate` per second."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        E = int(round(np.exp(rng.uniform(np.log(E_range[0]), np.log(E_range[1])))))
        N = int(rng.choice(N_choices))
        steps = 2 * int(rng.integers(steps_range[0] // 2, steps_range[1] // 2 + 1))
        xi = tuple(float(v) for v in rng.uniform(-0.5, 0.5, 3))
        d = rng.standard_normal(3)
        force = tuple(float(v) for v in d / np.linalg.norm(d))
        out.append(Request(i, t, E, N, steps, int(rng.integers(1, 2**31 - 1)), xi, force))
    return out
