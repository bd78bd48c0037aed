"""Fully discrete stability of the upwind elastic operator with LSRK(5,4) at the
CFL convention dt = CFL h_min / (c_max N^2) (the convention of the paper's
transport experiments, Section 6.1), on the oracle alone.

With the upwind flux of Section 2 the semi-discrete operator loses energy
through the faces only (the semi-discrete energy identity that the oracle's
operator tests check), so at a stable step the energy of every step is at most
that of the step before.  The N^2 scaling understates the stiffness at low
degree: a rough state (random nodal values on 27 warped, rotated elements with
a smooth random medium and free-surface and absorbing boundaries) grows without
bound at CFL 0.5 for N = 1 and N = 2.  These are the limits that the library's dgw_dt_cfl documentation
states: N = 1 stable at 0.125 and unstable at 0.15, N = 2 stable at 0.45 and
unstable at 0.5, N = 3 stable at 0.5.
"""
import numpy as np
import pytest

import oracle
import workloads as wl


def _rough_case(N):
    mesh = wl.structured_hex_mesh(3, (True, False, False),
                                  {2: wl.BC_FREE_SURFACE, 3: wl.BC_ABSORBING, 4: wl.BC_ABSORBING,
                                   5: wl.BC_FREE_SURFACE}, "lex")
    mesh = wl.rotate_elements(mesh, 100 + N)
    rho, lam, mu = wl.smooth_random_material(mesh, N)
    r, _ = oracle.gll(N)
    x = wl.warped_node_coords(mesh, r, 0.08)
    op = oracle.ElasticDG(N, x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc, rho, lam, mu, 1)
    return op, wl.random_state(mesh.nel, (N + 1) ** 3, N), oracle.h_min_corner_edges(x, N)


def _energies(N, cfl, steps):
    op, u, h = _rough_case(N)
    dt = oracle.cfl_dt(cfl, h, op.c_max(), N)
    res = np.zeros_like(u)
    e = [op.energy(u)]
    for _ in range(steps):
        u, res = op.step(u, res, dt)
        e.append(op.energy(u))
    return np.array(e) / e[0]


@pytest.mark.parametrize("N,cfl,steps", [(1, 0.125, 40), (2, 0.45, 60), (3, 0.5, 40)])
def test_energy_decays_at_stable_cfl(N, cfl, steps):
    e = _energies(N, cfl, steps)
    assert np.all(e[1:] <= e[:-1] * (1 + 1e-12))
    assert e[-1] < 0.5


@pytest.mark.parametrize("N,cfl,steps", [(1, 0.15, 40), (2, 0.5, 40)])
def test_energy_grows_beyond_low_degree_limit(N, cfl, steps):
    e = _energies(N, cfl, steps)
    assert e[-1] > 1e6
