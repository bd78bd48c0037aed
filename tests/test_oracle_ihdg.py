"""Pins of the iHDG-II oracle (Section 3, Algorithm "The iHDG-II approach").

* the local blocks: L_K^self from the colouring equals the element-by-element
  definition, and L_K^self u_K + L_K^nbr(u) = L(u)_K;
* a fixed point of the iteration solves sigma u - L(u) = b (direct solve);
* finite convergence for upwind transport (Theorem DDMConvergence): with
  beta > 0 componentwise on an E^3 structured mesh the iterate equals the
  direct solution after exactly 3E - 2 iterations (one per diagonal layer of
  elements, counted from the inflow corner), independent of the degree;
* the iteration counts of the paper's table (golden fixture), with its
  stopping criterion (eq. tolerancecriteria): within one iteration, and the
  asymptotics d N_el^(1/d);
* the locally implicit use (Section 4.3): one implicit Euler step solved by
  iHDG-II equals the direct implicit step.
"""
import os

import numpy as np
import pytest

import oracle
import workloads as wl
from oracle.ihdg import IHDGTransport, element_coloring

BETA = np.array([1.0, 0.7, 0.4])
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ihdg_transport_iterations.txt")


def _op(E, N, a=0.0, periodic=False, beta=BETA):
    mesh = wl.structured_hex_mesh(E, (periodic,) * 3)
    r, _ = oracle.gll(N)
    x = wl.warped_node_coords(mesh, r, a)
    return oracle.FriedrichsDG(N, x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc, oracle.transport(beta)), x


def _manufactured(x, beta=BETA):
    """u^e = prod sin(pi x_i) (zero on every boundary face, so the zero exterior
    state is the exact inflow data) and f = beta . grad u^e at the nodes."""
    X = np.pi * x
    s, c = np.sin(X), np.cos(X)
    ue = np.prod(s, axis=-1)
    grad = np.pi * np.stack([c[..., 0] * s[..., 1] * s[..., 2], s[..., 0] * c[..., 1] * s[..., 2],
                             s[..., 0] * s[..., 1] * c[..., 2]], axis=-1)
    return ue[None], (grad @ beta)[None]


def test_self_blocks_and_splitting():
    op, _ = _op(3, 2, a=0.05)
    ih = IHDGTransport(op, 0.0)
    color = element_coloring(op.etoe)
    for e in range(op.nel):
        assert all(color[n] != color[e] for n in op.etoe[e] if n >= 0)
    K = 13
    for j in (0, 5, 26):
        u = np.zeros((1, op.nel, op.Np))
        u[0, K, j] = 1.0
        assert np.allclose(ih.Lself[K][:, j], op.rhs(u)[0, K], atol=1e-13)
    u = wl.random_fields(1, op.nel, op.Np, 3)
    lhs = np.einsum("eij,ej->ei", ih.Lself, u[0])[None] + ih.neighbour_term(u)
    assert np.allclose(lhs, op.rhs(u), atol=1e-12)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_finite_convergence_after_one_iteration_per_layer(N):
    E = 3
    op, x = _op(E, N)
    ih = IHDGTransport(op, 0.0)
    _, f = _manufactured(x)
    ud = ih.direct(f)
    u = np.zeros_like(f)
    for k in range(1, 3 * E - 2):
        u = ih.iterate(f, u)
        assert ih.norm(u - ud) > 1e-6 * ih.norm(ud), k
    u = ih.iterate(f, u)                       # iteration 3E - 2
    assert ih.norm(u - ud) < 1e-12 * ih.norm(ud)


def _golden():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    return {(int(E), int(p)): int(k) for E, p, k in rows}


@pytest.mark.parametrize("E,N", [(2, 1), (4, 1), (8, 1), (2, 2), (4, 2), (2, 3), (2, 4)])
def test_iteration_counts_of_the_paper(E, N):
    op, x = _op(E, N)
    ih = IHDGTransport(op, 0.0)
    ue, f = _manufactured(x)
    u, its, _ = ih.solve(f, np.zeros_like(f), tol=1e-10, exact=ue)
    paper = _golden()[(E, N)]
    assert its == 3 * E - 1                    # 3E - 2 layers, then one iteration without change
    # The paper's counts are 3E - 1 from 8^3 on and one or two more on 2^3 and 4^3,
    # where they also vary with p (6 or 7 on 2^3) although its theorem makes them
    # p-independent; its velocity and exact solution are not printed.
    assert abs(its - paper) <= (1 if E >= 4 else 2)
    assert abs(its - 3 * E) <= 1               # d N_el^(1/d)
    if op.nel * op.Np <= 2000:                 # the converged iterate is the HDG solution
        ud = ih.direct(f)
        assert ih.norm(u - ud) < 1e-10 * ih.norm(ud)


def test_locally_implicit_step_equals_the_direct_implicit_step():
    op, x = _op(3, 3, a=0.05, periodic=True, beta=np.array([0.2, 0.3, -0.1]))
    dt = 2.0 * oracle.cfl_dt(1.0, 1.0 / 3, op.c_max(), 3)         # CFL 2
    ih = IHDGTransport(op, 1.0 / dt)
    um = wl.transport_periodic(x, (0.2, 0.3, -0.1))
    b = um / dt
    ud = ih.direct(b)
    u, its, hist = ih.solve(b, um, tol=1e-12)
    assert its < 40 and hist[-1] < 1e-12
    assert ih.norm(u - ud) < 1e-10 * ih.norm(ud)


# ---- the linearized shallow-water system, Crank-Nicolson (Section 6.2) -------

SW_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ihdg_shallow_water_iterations.txt")


def _sw_golden():
    rows = [l.split() for l in open(SW_GOLDEN) if l.strip() and not l.startswith("#")]
    return {(int(n), int(p)): (int(a), int(b)) for n, p, a, b in rows}


def _sw_op(E, N):
    mesh = wl.structured_hex_mesh((E, E, 1), (False, False, True), {0: wl.BC_WALL, 1: wl.BC_WALL,
                                                                     2: wl.BC_WALL, 3: wl.BC_WALL})
    r, _ = oracle.gll(N)
    x = wl.warped_node_coords(mesh, r, 0.0)
    return oracle.FriedrichsDG(N, x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc, oracle.shallow_water()), x


def _cn_step(op, x, dt):
    """sigma = 2/dt, b = sigma u^m + L(u^m) from the standing wave at t = 0."""
    from oracle.ihdg import IHDG
    ih = IHDG(op, 2.0 / dt)
    um = wl.shallow_water_standing_wave(x)
    return ih, um, ih.sigma * um + op.rhs(um)


def test_shallow_water_cn_step_converges_to_the_direct_step():
    op, x = _sw_op(3, 2)
    ih, um, b = _cn_step(op, x, 0.1)
    u, its, hist = ih.solve(b, um, tol=1e-12)
    assert hist[-1] < 1e-12
    ud = ih.direct(b)
    assert ih.norm(u - ud) < 1e-10 * ih.norm(ud)
    # the Crank-Nicolson step approximates the standing wave at t = dt (coarse mesh: a sanity bound)
    assert ih.norm(ud - wl.shallow_water_standing_wave(x, 0.1)) < 0.05 * ih.norm(ud)


@pytest.mark.parametrize("E,N", [(4, 1), (8, 1), (16, 1), (4, 2), (8, 2), (4, 3)])
def test_shallow_water_iteration_counts_of_the_paper(E, N):
    """The paper's iHDG-II counts (golden table), with eq. tolerancecriteriarelerror
    on the first Crank-Nicolson step: within 3 for both time steps; more
    iterations for the larger step (the count grows with dt)."""
    op, x = _sw_op(E, N)
    paper = _sw_golden()[(E * E, N)]
    counts = []
    for dt in (0.1, 0.01):
        ih, um, b = _cn_step(op, x, dt)
        _, its, _ = ih.solve(b, um, tol=1e-10)
        counts.append(its)
    assert abs(counts[0] - paper[0]) <= 3 and abs(counts[1] - paper[1]) <= 3, (counts, paper)
    assert counts[0] > counts[1]


# ---- the elastic system (velocity-stress, heterogeneous, curvilinear) --------
#
# The paper builds iHDG-II on the upwind HDG discretisation of a Friedrichs
# system; the elastic operator is one (with Q), taken here with the upwind
# flux.  Pins: the self-only operator is the operator of one element alone; a
# fixed point solves the implicit step; and the implicit steps obey the exact
# energy identities of a linear operator L in the Q inner product, with
# rate(w) = <w, L w>_Q (the oracle's energy_rate, computed independently):
#   implicit Euler   E(u^0) = E(u^1) + E(u^1 - u^0) - dt rate(u^1),
#   Crank-Nicolson   E(u^1) - E(u^0) = dt/4 rate(u^1 + u^0).
# A wrong local block or neighbour term leaves the step unsolved and breaks them.


def _el_op(tau=1, E=(3, 3, 2), N=1, seed=3):
    mesh = wl.structured_hex_mesh(E, (True, True, False), {4: wl.BC_FREE_SURFACE, 5: wl.BC_ABSORBING})
    r, _ = oracle.gll(N)
    x = wl.warped_node_coords(mesh, r, 0.05)
    rho, lam, mu = wl.smooth_random_material(mesh, seed)
    op = oracle.ElasticDG(N, x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc, rho, lam, mu, tau)
    dt = oracle.cfl_dt(0.5, oracle.h_min_corner_edges(x, N), op.c_max(), N)
    return op, x, dt


def test_elastic_self_blocks_are_the_operator_of_one_element():
    from oracle.ihdg import IHDG
    op, _, dt = _el_op()
    ih = IHDG(op, 1.0 / dt)
    for K in (0, 4, 17):            # free-surface bottom, absorbing top
        for qj in (0, 5, 3 * op.Np + 2, 8 * op.Np + 7):
            u = np.zeros((9, op.nel, op.Np))
            u[qj // op.Np, K, qj % op.Np] = 1.0
            col = op.rhs(u, source=False)[:, K].reshape(-1)
            assert np.allclose(ih.Lself[K][:, qj], col, atol=1e-12 * np.abs(col).max())


def test_elastic_implicit_euler_by_ihdg():
    """sigma = 1/dt (CFL 2), b = u^0/dt: the converged iterate is the direct
    implicit step and satisfies the implicit-Euler energy identity."""
    from oracle.ihdg import IHDG
    op, x, dt0 = _el_op()
    dt = 4.0 * dt0
    ih = IHDG(op, 1.0 / dt)
    u0 = wl.random_fields(9, op.nel, op.Np, 11)
    b = u0 / dt
    u, its, hist = ih.solve(b, u0, tol=1e-13, max_iter=400)
    assert hist[-1] < 1e-13
    ud = ih.direct(b)
    assert ih.norm(u - ud) < 1e-10 * ih.norm(ud)
    E0, E1, Ed = op.energy(u0), op.energy(u), op.energy(u - u0)
    rate = op.energy_rate(u)
    assert rate < 0 and E1 < E0
    assert abs(E0 - (E1 + Ed - dt * rate)) < 1e-11 * E0


def test_elastic_crank_nicolson_by_ihdg_energy_identity():
    from oracle.ihdg import IHDG
    op, x, dt0 = _el_op()
    dt = 4.0 * dt0
    ih = IHDG(op, 2.0 / dt)
    u0 = wl.random_fields(9, op.nel, op.Np, 12)
    b = ih.sigma * u0 + op.rhs(u0, source=False)
    u, its, hist = ih.solve(b, u0, tol=1e-13, max_iter=400)
    assert hist[-1] < 1e-13
    E0, E1 = op.energy(u0), op.energy(u)
    assert abs((E1 - E0) - 0.25 * dt * op.energy_rate(u + u0)) < 1e-11 * E0


def test_elastic_crank_nicolson_identity_at_degree_two():
    """The Crank-Nicolson energy identity at N = 2 (243-row local blocks), and
    the converged iterate equals the direct step."""
    from oracle.ihdg import IHDG
    op, x, dt0 = _el_op(E=(3, 2, 2), N=2, seed=5)
    dt = 4.0 * dt0
    ih = IHDG(op, 2.0 / dt)
    u0 = wl.random_fields(9, op.nel, op.Np, 13)
    b = ih.sigma * u0 + op.rhs(u0, source=False)
    u, its, hist = ih.solve(b, u0, tol=1e-13, max_iter=400)
    assert hist[-1] < 1e-13
    E0, E1 = op.energy(u0), op.energy(u)
    assert abs((E1 - E0) - 0.25 * dt * op.energy_rate(u + u0)) < 1e-11 * E0
    assert ih.norm(u - ih.direct(b)) < 1e-10 * ih.norm(u)
