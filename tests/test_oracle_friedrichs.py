"""Pins of the generic Friedrichs-system oracle (transport, linearized shallow water).

What fixes each part without a reference implementation:
* the flux: scalar upwinding by hand (transport) and the closed-form |A(n)| of
  the shallow-water flux matrix (eigenvalues 0, +-|n_xy|);
* volume term, metrics, lift: free-stream preservation on warped, rotated meshes;
* flux and boundary states: the semi-discrete energy identity (volume form ==
  face form), energy conservation of the central flux with periodic faces and
  with walls, brute-force skew-symmetry / dissipativity of the assembled operator;
* everything together: design-order convergence to the exact solutions of the
  paper's transport (periodic stand-in, Section 6.1) and shallow-water
  standing-wave (Section 6.2) tests.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

BETA = (0.2, 0.3, -0.1)


def _transport_op(E, N, a=0.1, tau=1, rotate=None, beta=BETA):
    mesh = wl.structured_hex_mesh(E)
    if rotate is not None:
        mesh = wl.rotate_elements(mesh, rotate)
    r, _ = oracle.gll(N)
    x = wl.warped_node_coords(mesh, r, a)
    return oracle.FriedrichsDG(N, x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc, oracle.transport(beta), tau), x


def _sw_op(E, N, a=0.05, tau=1, rotate=None):
    mesh = wl.structured_hex_mesh((E, E, 1), (False, False, True), {0: wl.BC_WALL, 1: wl.BC_WALL,
                                                                     2: wl.BC_WALL, 3: wl.BC_WALL})
    if rotate is not None:
        mesh = wl.rotate_elements(mesh, rotate)
    r, _ = oracle.gll(N)
    x = wl.warped_node_coords(mesh, r, a)
    return oracle.FriedrichsDG(N, x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc, oracle.shallow_water(), tau), x


def test_transport_flux_is_scalar_upwinding():
    sysm = oracle.transport(BETA)
    for n in ([1.0, 0.0, 0.0], [-0.6, 0.0, 0.8], [0.0, 0.6, 0.8]):
        n = np.asarray(n)
        bn = float(np.dot(BETA, n))
        An = sysm.A_of(n)
        stab = sysm.abs_A(n)
        assert np.isclose(stab[0, 0], abs(bn))
        um, up = np.array([1.7]), np.array([-0.4])
        fhat = oracle.hdg_flux(An, stab, um, oracle.weighted_trace(An, stab, um, up))
        assert np.isclose(fhat[0], bn * (um[0] if bn > 0 else up[0]))


def test_shallow_water_flux_matrix_and_closed_form_stabilisation():
    sysm = oracle.shallow_water()
    # eq. linearizedShallow with Phi = 1: phi_t + div(Phi u) = 0, (Phi u)_t + Phi grad phi = 0
    A = sysm.A_of([0.3, -0.5, 0.7])
    assert np.allclose(A, [[0, 0.3, -0.5], [0.3, 0, 0], [-0.5, 0, 0]])
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        nu = np.hypot(n[0], n[1])
        closed = np.array([[nu, 0, 0], [0, n[0] ** 2 / nu, n[0] * n[1] / nu], [0, n[0] * n[1] / nu, n[1] ** 2 / nu]])
        assert np.allclose(sysm.abs_A(n), closed, atol=1e-14)


def test_shallow_water_wall_reflects_normal_momentum():
    sysm = oracle.shallow_water()
    n = np.array([0.6, -0.8, 0.0])
    um = np.array([0.7, 0.2, 0.5])
    up = sysm.ghost(um, n, 1)
    assert up[0] == um[0]
    assert np.isclose(np.dot(up[1:3] + um[1:3], n[:2]), 0.0)          # mean normal momentum vanishes
    assert np.allclose((up[1:3] - um[1:3]) - np.dot(up[1:3] - um[1:3], n[:2]) * n[:2], 0.0)   # tangential kept


@pytest.mark.parametrize("rotate", [None, 5])
def test_free_stream_preservation(rotate):
    op, _ = _transport_op(3, 4, 0.1, rotate=rotate)
    assert np.max(np.abs(op.rhs(np.full((1, op.nel, op.Np), 2.5)))) < 1e-12
    sw, _ = _sw_op(3, 4, 0.05, rotate=rotate)
    u = np.zeros((3, sw.nel, sw.Np))
    u[0] = 1.3
    assert np.max(np.abs(sw.rhs(u))) < 1e-12


@pytest.mark.parametrize("tau", [0, 1])
def test_energy_identity(tau):
    op, _ = _transport_op(2, 3, 0.1, tau=tau, rotate=2)
    u = wl.random_fields(1, op.nel, op.Np, 4)
    a, b = op.energy_rate(u), op.energy_rate_from_faces(u)
    assert abs(a - b) <= 1e-12 * max(1.0, abs(a))
    if tau == 0:
        assert abs(a) < 1e-12
    else:
        assert a < 0
    sw, _ = _sw_op(3, 3, 0.05, tau=tau, rotate=4)
    u = wl.random_fields(3, sw.nel, sw.Np, 5)
    a, b = sw.energy_rate(u), sw.energy_rate_from_faces(u)
    assert abs(a - b) <= 1e-12 * max(1.0, abs(a))
    if tau == 0:
        assert abs(a) < 1e-12            # walls conserve energy with the central flux
    else:
        assert a < 0


def _assemble(op):
    m, nel, Np = op.m, op.nel, op.Np
    n = m * nel * Np
    L = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        L[:, j] = op.rhs(e.reshape(m, nel, Np)).ravel()
    _, J = op.geometry(np.arange(nel))
    M = np.tile((op.w_vol[None, :] * J).ravel(), m)
    return M[:, None] * L


@pytest.mark.parametrize("tau", [0, 1])
def test_bruteforce_operator_skew_and_dissipative(tau):
    for op in (_transport_op(2, 2, 0.1, tau=tau, rotate=3)[0], _sw_op(2, 2, 0.05, tau=tau, rotate=1)[0]):
        ML = _assemble(op)
        S = ML + ML.T
        scale = np.max(np.abs(ML))
        if tau == 0:
            assert np.max(np.abs(S)) < 1e-12 * scale
        else:
            assert np.max(np.linalg.eigvalsh(0.5 * S)) < 1e-12 * scale


def _run(op, u, dt, nsteps):
    res = np.zeros_like(u)
    for k in range(nsteps):
        u, res = op.step(u, res, dt, t=k * dt)
    return u


def _l2(op, d):
    _, J = op.geometry(np.arange(op.nel))
    return float(np.sqrt(np.sum(op.w_vol[None, None, :] * J[None] * d * d)))


@pytest.mark.parametrize("N,meshes,min_rate", [(2, (8, 16), 2.4), (4, (4, 8), 4.0)])
def test_transport_design_order(N, meshes, min_rate):
    """Rate of the L2 error at T on the warped periodic mesh (the 3-D product of
    sines is pre-asymptotic on coarse meshes; the bounds are N + 0.4 and N)."""
    T = 0.2
    errs = []
    for E in meshes:
        op, x = _transport_op(E, N, 0.05)
        dt = oracle.cfl_dt(0.5, 1.0 / E, op.c_max(), N)
        nsteps = int(np.ceil(T / dt))
        u = _run(op, wl.transport_periodic(x, BETA), T / nsteps, nsteps)
        errs.append(_l2(op, u - wl.transport_periodic(x, BETA, T)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > min_rate, (errs, rates)


@pytest.mark.parametrize("N,meshes,min_rate", [(2, (4, 8), 2.8), (3, (4, 8), 3.6)])
def test_shallow_water_standing_wave_design_order(N, meshes, min_rate):
    """The paper's standing wave with walls (Section 6.2): design rate N + 1."""
    T = 0.25
    errs = []
    for E in meshes:
        op, x = _sw_op(E, N, 0.0)
        dt = oracle.cfl_dt(0.5, 1.0 / E, op.c_max(), N)
        nsteps = int(np.ceil(T / dt))
        u = _run(op, wl.shallow_water_standing_wave(x), T / nsteps, nsteps)
        errs.append(_l2(op, u - wl.shallow_water_standing_wave(x, T)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > min_rate, (errs, rates)
