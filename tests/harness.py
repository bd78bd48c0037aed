"""Shared set-up for the GPU tests: the same seeded workload built twice, once at
the library's reference nodes (for the CUDA path) and once at the oracle's own
GLL nodes (for the oracle).  The two paths share only the input generators."""
from __future__ import annotations

import numpy as np

import oracle
import workloads as wl

# Parity bounds of the CUDA path against the oracle.
FP64_TOL = 1e-12
# FP32 volume/flux arithmetic on FP32 geometry: unit round-off 6e-8 times the
# O(N^2) amplification of the derivative and lift operators on rough data.
# Measured: 1.3e-7 (48^3, N=7, sampled elements), 8.5e-8 (smoke), 3.4e-7
# (8^3 Gaussian pulse; element max 6.4e-7); the bound is a few times the
# largest.  The tensor-core FP16 form (hi/lo split of 11-bit
# halves with a power-of-two scale per line group: about 22 bits per operand,
# products exact, FP32 sums) is held to the same bound.
MIXED_RHS_TOL = 1e-6
# BF16 hi/lo keeps 16 of FP32's 24 mantissa bits per operand: the dropped
# lo*lo product and the rounding of lo leave about 2^-17 relative per term.
BF16_RHS_TOL = 5e-5
TC_TOL = {"mixed": MIXED_RHS_TOL, "mixed_tc": MIXED_RHS_TOL, "mixed_tc_bf16": BF16_RHS_TOL}
# Ten LSRK steps of the parity workload (50 stages) against the oracle.
# Measured (rel L2 / element max): mixed 8.1e-8 / 3.2e-7, mixed_tc 4.7e-8 /
# 1.0e-7, mixed_tc_bf16 6.7e-6 / 1.3e-5.
STEP10_TOL = {"mixed": 1e-6, "mixed_tc": 1e-6, "mixed_tc_bf16": 2e-5}


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def elem_max_rel(a, b):
    """Largest per-element error: max over elements e of max |a_e - b_e| (all
    fields and nodes of e), relative to max |b| over the whole array.  Arrays
    are [m][nel][Np] (or a sample of elements on the middle axis).  One wrong
    node shows here at its own size, where a global L2 norm dilutes it."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max(axis=(0, 2)).max() / np.abs(b).max())


def assert_parity(got, want, tol, tol_elem=None, label=""):
    """Global relative L2 <= tol and per-element maximum error <= tol_elem
    (default: tol); returns both measures."""
    e2, em = rel_l2(got, want), elem_max_rel(got, want)
    te = tol if tol_elem is None else tol_elem
    if label:
        print(f"{label}: rel L2 {e2:.3e}, element max {em:.3e}")
    assert e2 < tol and em < te, f"{label} rel L2 {e2:.3e} (bound {tol:.1e}), element max {em:.3e} (bound {te:.1e})"
    return e2, em


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


def graph_distance(etoe, sources, maxd):
    """Face-neighbour graph distance from the `sources` elements, up to maxd
    (larger distances stay at maxd + 1)."""
    d = np.full(etoe.shape[0], maxd + 1, dtype=np.int64)
    frontier = np.unique(np.asarray(sources, dtype=np.int64))
    d[frontier] = 0
    for k in range(1, maxd + 1):
        nb = etoe[frontier].ravel()
        nb = np.unique(nb[nb >= 0])
        frontier = nb[d[nb] > k]
        d[frontier] = k
    return d


def oracle_sampled_steps(op, u0, res0, dt, nsteps, sample, t0=0.0):
    """The oracle's nsteps LSRK steps, exact on the `sample` elements without a
    full-mesh run: a stage reads face neighbours only, so stage k (of S = 5 nsteps)
    is evaluated on the elements within graph distance S - k of the sample, whose
    neighbours the previous stage has updated.  Returns (u, res) on the sample."""
    S = 5 * nsteps
    dist = graph_distance(op.etoe, sample, S)
    u, res = u0.copy(), res0.copy()
    k = 0
    for step in range(nsteps):
        for s in range(5):
            k += 1
            region = np.nonzero(dist <= S - k)[0]
            un, rn = op.lsrk_stage(u, res, s, dt, region, t=t0 + step * dt)
            u[:, region] = un
            res[:, region] = rn
            for c in (op._geo_cache, op._nbr_cache, op._abs_cache, op._qinv_cache):
                c.clear()
    sample = np.asarray(sample)
    return u[:, sample], res[:, sample]
