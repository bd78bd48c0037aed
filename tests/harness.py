"""Shared set-up for the GPU tests: the same seeded workload built twice, once at
the library's reference nodes (for the CUDA path) and once at the oracle's own
GLL nodes (for the oracle).  The two paths share only the input generators."""
from __future__ import annotations

import numpy as np

import oracle
import workloads as wl


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


class Case:
    """One mesh + medium + initial state, on both sides."""

    def __init__(self, E, N, amplitude=0.1, periodic=(True, True, True), boundary=None, order="lex",
                 material=None, rotate=None, tau=1, precision="fp64", initial="random", seed=0):
        from paper_1711_01175_gb300 import Solver, reference_nodes
        self.N, self.tau = N, tau
        mesh = wl.structured_hex_mesh(E, periodic, boundary, order)
        if rotate is not None:
            mesh = wl.rotate_elements(mesh, rotate)
        self.mesh = mesh
        if material is None:
            rho, lam, mu = wl.homogeneous_material(mesh.nel)
        else:
            rho, lam, mu = wl.smooth_random_material(mesh, material)
        self.rho, self.lam, self.mu = rho, lam, mu
        r_lib, _ = reference_nodes(N)
        r_or, _ = oracle.gll(N)
        self.x_lib = wl.warped_node_coords(mesh, r_lib, amplitude)
        self.x_or = wl.warped_node_coords(mesh, r_or, amplitude)
        Np = (N + 1) ** 3
        if initial == "random":
            self.u0 = wl.random_state(mesh.nel, Np, seed)
        elif initial == "gaussian_pulse":
            self.u0 = wl.gaussian_stress_pulse(self.x_or)
        else:
            self.u0 = wl.plane_p_wave(self.x_or, 1.0, 2.0, 1.0)
        self.solver = Solver(N, tau=tau, precision=precision)
        self.solver.upload_mesh(self.x_lib, mesh.etoe, mesh.etof, mesh.orient, mesh.bc)
        self.solver.upload_material(rho, lam, mu)
        self._op = None

    @property
    def op(self):
        if self._op is None:
            m = self.mesh
            self._op = oracle.ElasticDG(self.N, self.x_or, m.etoe, m.etof, m.orient, m.bc,
                                        self.rho, self.lam, self.mu, self.tau)
        return self._op

    def gpu_rhs(self, u):
        import torch
        ud = torch.from_numpy(np.ascontiguousarray(u)).cuda()
        out = torch.empty_like(ud)
        self.solver.rhs(ud, out)
        return out.cpu().numpy()
