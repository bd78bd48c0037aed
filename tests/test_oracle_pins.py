"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test checks the oracle against a closed form, an exact invariant of the
scheme, brute force on a tiny mesh, a value printed in the paper, or a
convergence rate -- never against a retyped copy of its own formula.
"""
from fractions import Fraction
from math import sqrt
import os

import numpy as np
import pytest

import oracle
from oracle.dg_elastic import ElasticDG, A_of, abs_A, abs_A_Q, weighted_trace, hdg_flux
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- GLL, D, SBP
@pytest.mark.parametrize("N,nodes,weights", [
    (1, [-1, 1], [1, 1]),
    (2, [-1, 0, 1], [1 / 3, 4 / 3, 1 / 3]),
    (3, [-1, -1 / sqrt(5), 1 / sqrt(5), 1], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    (4, [-1, -sqrt(3 / 7), 0, sqrt(3 / 7), 1], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
])
def test_gll_closed_forms(N, nodes, weights):
    r, w = oracle.gll(N)
    np.testing.assert_allclose(r, nodes, atol=1e-15)
    np.testing.assert_allclose(w, weights, atol=1e-15)


@pytest.mark.parametrize("N", range(1, 9))
def test_gll_quadrature_degree(N):
    r, w = oracle.gll(N)
    for q in range(2 * N):
        exact = 0.0 if q % 2 else 2.0 / (q + 1)
        assert abs(np.sum(w * r ** q) - exact) < 1e-13
    # GLL is not exact at degree 2N (a discriminating check of the rule)
    assert abs(np.sum(w * r ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-6


@pytest.mark.parametrize("N", range(1, 9))
def test_derivative_matrix_exact_and_sbp(N):
    r, w = oracle.gll(N)
    D = oracle.lagrange_derivative_matrix(r)
    for q in range(N + 1):
        d_exact = q * r ** (q - 1) if q > 0 else np.zeros_like(r)
        np.testing.assert_allclose(D @ r ** q, d_exact, atol=1e-11)
    W = np.diag(w)
    Bnd = np.zeros((N + 1, N + 1))
    Bnd[0, 0], Bnd[-1, -1] = -1.0, 1.0
    np.testing.assert_allclose(W @ D + D.T @ W, Bnd, atol=1e-13)


# ------------------------------------------------------------ system and |A|
def test_A_is_elastodynamics():
    """A(n) u = -(sigma n, Voigt(sym(n (x) v))) for a random state and normal."""
    rng = np.random.default_rng(0)
    n = rng.standard_normal(3)
    v = rng.standard_normal(3)
    S = rng.standard_normal((3, 3))
    S = S + S.T
    s_voigt = np.array([S[0, 0], S[1, 1], S[2, 2], S[1, 2], S[0, 2], S[0, 1]])
    out = A_of(n) @ np.concatenate([v, s_voigt])
    np.testing.assert_allclose(out[:3], -S @ n, atol=1e-14)
    E = 0.5 * (np.outer(n, v) + np.outer(v, n))
    np.testing.assert_allclose(out[3:], -np.array([E[0, 0], E[1, 1], E[2, 2],
                                                   2 * E[1, 2], 2 * E[0, 2], 2 * E[0, 1]]), atol=1e-14)


def test_absA_axis_normal_by_hand():
    """n = e1: B^T B = I, so |A| = diag(I_3, B B^T) = diag(1,1,1, 1,0,0,0,1,1)."""
    expect = np.diag([1, 1, 1, 1, 0, 0, 0, 1, 1]).astype(float)
    np.testing.assert_allclose(abs_A(np.array([1.0, 0, 0])), expect, atol=1e-14)
    np.testing.assert_allclose(abs_A(np.array([-1.0, 0, 0])), expect, atol=1e-14)


def test_absA_invariants():
    rng = np.random.default_rng(1)
    for _ in range(20):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        A = A_of(n)
        M = abs_A(n)
        np.testing.assert_allclose(M @ M, A @ A, atol=1e-13)
        assert np.min(np.linalg.eigvalsh(M)) > -1e-13
        np.testing.assert_allclose(M, M.T, atol=1e-14)
        # three zero eigenvalues (rank-6 A), the rest in +- pairs
        ev = np.sort(np.linalg.eigvalsh(A))
        np.testing.assert_allclose(ev, -ev[::-1], atol=1e-13)
        assert np.sum(np.abs(ev) < 1e-12) == 3


def test_impedance_stabilisation_axis_normal_by_hand():
    """rho=1, lam=2, mu=1 (Zp = 2, Zs = 1), n = e1: the velocity block is
    diag(Zp, Zs, Zs); the stress block B diag(1/Zp, 1/Zs, 1/Zs) B^T acts on
    (s11, s13, s12) only."""
    expect = np.diag([2, 1, 1, 0.5, 0, 0, 0, 1, 1]).astype(float)
    np.testing.assert_allclose(abs_A_Q(np.array([1.0, 0, 0]), 1.0, 2.0, 1.0), expect, atol=1e-14)


def test_impedance_stabilisation_is_physical_upwinding():
    rng = np.random.default_rng(5)
    for _ in range(10):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        rho, cp = rng.uniform(1, 3), rng.uniform(2, 6)
        cs = cp / np.sqrt(3) * rng.uniform(0.9, 1.1)
        mu, lam = rho * cs * cs, rho * (cp * cp - 2 * cs * cs)
        A, S = A_of(n), abs_A_Q(n, rho, lam, mu)
        Q = oracle.Q_of(rho, lam, mu)
        Qi = np.linalg.inv(Q)
        np.testing.assert_allclose(S, S.T, atol=1e-12)
        assert np.min(np.linalg.eigvalsh(S)) > -1e-12
        np.testing.assert_allclose(S @ Qi @ S, A @ Qi @ A, atol=1e-10 * np.max(np.abs(A @ Qi @ A)))
        # |Q^{-1} A| has the physical speeds: cp twice, cs four times, three zeros
        sp = np.sort(np.linalg.eigvals(Qi @ S).real)
        np.testing.assert_allclose(sp, [0, 0, 0, cs, cs, cs, cs, cp, cp], atol=1e-10 * cp)
        # characteristic upwinding: outgoing waves (speed > 0 along n) need no
        # correction, incoming ones are replaced entirely by the exterior state
        lamv, R = np.linalg.eig(Qi @ A)
        for k in range(9):
            r = R[:, k].real
            corr = 0.5 * (A - S) @ r
            if lamv[k].real > 1e-8:
                assert np.max(np.abs(corr)) < 1e-10 * np.max(np.abs(A @ r) + 1)
            elif lamv[k].real < -1e-8:
                np.testing.assert_allclose(corr, A @ r, atol=1e-10 * np.max(np.abs(A @ r)))


def test_hdg_flux_conservation_and_scalar_upwind():
    """eq. HDGeqn: F_hat.n^- + F_hat.n^+ = 0 on a face; for m = 1 transport the
    flux is the textbook upwind value beta.n u_upwind."""
    rng = np.random.default_rng(2)
    n = rng.standard_normal(3)
    n /= np.linalg.norm(n)
    um, up = rng.standard_normal(9), rng.standard_normal(9)
    An, S = A_of(n), abs_A(n)
    f_minus = hdg_flux(An, S, um, weighted_trace(An, S, um, up))
    f_plus = hdg_flux(-An, S, up, weighted_trace(-An, S, up, um))
    np.testing.assert_allclose(f_minus + f_plus, 0.0, atol=1e-13)
    for b in (0.7, -0.3):
        a = np.array([[b]])
        s = np.array([[abs(b)]])
        ul, ur = np.array([1.3]), np.array([-0.4])
        f = hdg_flux(a, s, ul, weighted_trace(a, s, ul, ur))
        assert abs(f[0] - b * (ul[0] if b > 0 else ur[0])) < 1e-15


# ---------------------------------------------------------------- LSRK(5,4)
def _butcher_from_2n(A, B):
    s = len(A)
    # Track stage inputs Y_i and the register dU as coefficient vectors over k_j.
    U = [Fraction(0)] * s
    dU = [Fraction(0)] * s
    rows = []
    for i in range(s):
        rows.append(list(U))                       # Y_i = U (before stage i)
        dU = [A[i] * c for c in dU]
        dU[i] += 1
        U = [U[j] + B[i] * dU[j] for j in range(s)]
    return rows, U


def test_lsrk_order_conditions():
    a, b = _butcher_from_2n(oracle.LSRK_A, oracle.LSRK_B)
    s = len(b)
    c = [sum(row) for row in a]
    tol = Fraction(1, 10 ** 18)
    conds = [
        (sum(b), Fraction(1)),
        (sum(b[i] * c[i] for i in range(s)), Fraction(1, 2)),
        (sum(b[i] * c[i] ** 2 for i in range(s)), Fraction(1, 3)),
        (sum(b[i] * a[i][j] * c[j] for i in range(s) for j in range(s)), Fraction(1, 6)),
        (sum(b[i] * c[i] ** 3 for i in range(s)), Fraction(1, 4)),
        (sum(b[i] * c[i] * a[i][j] * c[j] for i in range(s) for j in range(s)), Fraction(1, 8)),
        (sum(b[i] * a[i][j] * c[j] ** 2 for i in range(s) for j in range(s)), Fraction(1, 12)),
        (sum(b[i] * a[i][j] * a[j][k] * c[k] for i in range(s) for j in range(s) for k in range(s)),
         Fraction(1, 24)),
    ]
    for got, want in conds:
        assert abs(got - want) < tol
    for ci, cc in zip(c, oracle.LSRK_C):
        assert abs(ci - cc) < tol
    # and it is not fifth order (discriminating)
    assert abs(sum(b[i] * c[i] ** 4 for i in range(s)) - Fraction(1, 5)) > Fraction(1, 10 ** 6)


def test_lsrk_temporal_order_four():
    lam = np.array([[-0.5, 2.0], [-2.0, -0.5]])       # damped rotation y' = lam y
    y0 = np.array([1.0, 0.0])
    exact_T = None
    errs = []
    for nsteps in (20, 40, 80):
        dt = 1.0 / nsteps
        y, res = y0.copy(), np.zeros(2)
        for _ in range(nsteps):
            for s in range(5):
                res = float(oracle.LSRK_A[s]) * res + dt * (lam @ y)
                y = y + float(oracle.LSRK_B[s]) * res
        w, V = np.linalg.eig(lam)
        exact_T = np.real(V @ np.diag(np.exp(w)) @ np.linalg.solve(V, y0))
        errs.append(np.linalg.norm(y - exact_T))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.8) and np.all(rates < 4.5)


# ------------------------------------------------------------------- CFL pin
def test_cfl_matches_paper_table():
    rows = np.loadtxt(os.path.join(GOLDEN, "cfl_time_dependent_transport.txt"))
    for cores, nel, printed in rows:
        E = round(nel ** (1 / 3))
        assert E ** 3 == nel
        cfl = oracle.cfl_number(0.01, 1.0 / E, 0.35, 4)
        assert abs(cfl - printed) <= 0.05 * printed + 1e-12
        assert abs(oracle.cfl_dt(cfl, 1.0 / E, 0.35, 4) - 0.01) < 1e-15


# -------------------------------------------------------------- geometry pins
def _operator(E, N, a, periodic=(True, True, True), boundary=None, tau=1, rotate=None, mat=None):
    r, _ = oracle.gll(N)
    mesh = wl.structured_hex_mesh(E, periodic, boundary)
    if rotate is not None:
        mesh = wl.rotate_elements(mesh, rotate)
    x = wl.warped_node_coords(mesh, r, a)
    if mat is None:
        rho, lam, mu = wl.homogeneous_material(mesh.nel)
    else:
        rho, lam, mu = wl.smooth_random_material(mesh, mat)
    op = ElasticDG(N, x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc, rho, lam, mu, tau)
    return op, mesh, x


def _analytic_metrics(X0, a):
    """Exact J a^i_k and J of the warp x -> X0 + a prod sin(2 pi X0), from the
    cofactors of its Jacobian matrix, for a cube element of edge h: X0 = c + (xi+1) h/2."""
    s = np.sin(2 * np.pi * X0)
    c = np.cos(2 * np.pi * X0)
    grad = np.stack([2 * np.pi * c[..., 0] * s[..., 1] * s[..., 2],
                     2 * np.pi * s[..., 0] * c[..., 1] * s[..., 2],
                     2 * np.pi * s[..., 0] * s[..., 1] * c[..., 2]], axis=-1)
    F = np.eye(3) + a * np.ones(3)[:, None] * grad[..., None, :]   # dx_i/dX0_j
    return F


@pytest.mark.parametrize("a", [0.05, 0.1])
def test_curl_metrics_match_cofactors(a):
    E, N = 2, 10
    op, mesh, x = _operator(E, N, a)
    elems = np.arange(op.nel)
    Ja, J = op.geometry(elems)
    r = op.r
    rho = wl.mesh.reference_grid(r)
    h = 1.0 / E
    X0 = (mesh.cell[:, None, :] + (rho[None] + 1) / 2) / E
    F = _analytic_metrics(X0, a) * (h / 2)                 # dx/dxi
    J_exact = np.linalg.det(F)
    cof = np.linalg.inv(F) * J_exact[..., None, None]      # J dxi_i/dx_k
    np.testing.assert_allclose(J, J_exact, rtol=0, atol=1e-5 * np.max(J_exact))
    for i in range(3):
        for k in range(3):
            np.testing.assert_allclose(Ja[i][k], cof[..., i, k], atol=1e-5 * (h / 2) ** 2)


def test_discrete_metric_identities_and_positive_J():
    op, mesh, x = _operator(3, 4, 0.1)
    elems = np.arange(op.nel)
    Ja, J = op.geometry(elems)
    assert np.all(J > 0)
    for k in range(3):
        div = sum(op.dref(Ja[i][k], i) for i in range(3))
        assert np.max(np.abs(div)) < 1e-13


def test_flat_boundary_face_area():
    """The warp vanishes on the cube's faces: the z=0 face has area exactly 1."""
    op, mesh, x = _operator(3, 4, 0.1, periodic=(True, True, False),
                            boundary={4: wl.BC_ABSORBING, 5: wl.BC_FREE_SURFACE})
    elems = np.nonzero(mesh.bc[:, 4] == wl.BC_ABSORBING)[0]
    Ja, J = op.geometry(elems)
    m = op.outward_scaled_normal(Ja, 4)
    sJ = np.linalg.norm(m, axis=-1)
    area = np.sum(op.w_face[None, :] * sJ)
    assert abs(area - 1.0) < 1e-12
    np.testing.assert_allclose(m[..., 2] / sJ, -1.0, atol=1e-12)


def test_matched_face_nodes_coincide():
    """Neighbour maps (including all eight permutation codes on a rotated mesh)
    pair physically coincident nodes (modulo the periodic shift)."""
    for rotate in (None, 7):
        op, mesh, x = _operator(3, 3, 0.1, rotate=rotate)
        flat = x.reshape(-1, 3)
        for f in range(6):
            nbr = op._neighbour_map(f)
            own = x[:, op.face_nodes[f]]                    # [nel, nf, 3]
            other = flat[nbr]
            d = own - other
            d -= np.round(d)                                 # periodic shift by whole cube
            assert np.max(np.abs(d)) < 1e-12
        if rotate is not None:
            assert len(set(mesh.orient.ravel().tolist())) == 8


# --------------------------------------------------- free stream / constants
@pytest.mark.parametrize("rotate", [None, 3])
def test_free_stream_preservation(rotate):
    op, mesh, x = _operator(3, 4, 0.1, rotate=rotate)
    u = np.ones((9, op.nel, op.Np)) * np.arange(1, 10)[:, None, None]
    L = op.rhs(u)
    assert np.max(np.abs(L)) < 1e-11 * np.max(np.abs(u)) * (op.N ** 2 * 3)


# ------------------------------------------------------------ energy identity
@pytest.mark.parametrize("tau", [0, 1])
def test_semidiscrete_energy_identity_periodic(tau):
    op, mesh, x = _operator(3, 3, 0.1, tau=tau, mat=4)
    u = wl.random_state(op.nel, op.Np, 11)
    rate = op.energy_rate(u)
    faces = op.energy_rate_from_faces(u)
    scale = op.energy(u) * op.N ** 2 * 3 / 0.2
    if tau == 0:
        assert abs(rate) < 1e-12 * scale
    else:
        assert faces < 0
    assert abs(rate - faces) < 1e-12 * scale


def test_semidiscrete_energy_identity_boundaries():
    op, mesh, x = _operator(3, 3, 0.1, periodic=(True, False, False),
                            boundary={2: wl.BC_FREE_SURFACE, 3: wl.BC_ABSORBING,
                                      4: wl.BC_ABSORBING, 5: wl.BC_FREE_SURFACE}, mat=5)
    u = wl.random_state(op.nel, op.Np, 12)
    rate = op.energy_rate(u)
    faces = op.energy_rate_from_faces(u)
    scale = op.energy(u) * op.N ** 2 * 3 / 0.2
    assert faces < 0
    assert abs(rate - faces) < 1e-12 * scale


def test_free_surface_central_conserves_energy():
    """With the central flux a traction-free surface neither adds nor removes energy."""
    op, mesh, x = _operator(2, 3, 0.05, periodic=(True, True, False),
                            boundary={4: wl.BC_FREE_SURFACE, 5: wl.BC_FREE_SURFACE}, tau=0, mat=6)
    u = wl.random_state(op.nel, op.Np, 13)
    scale = op.energy(u) * op.N ** 2 * 2 / 0.5
    assert abs(op.energy_rate(u)) < 1e-12 * scale


# --------------------------------------------------- brute-force operator
@pytest.mark.parametrize("E,N,tau", [(1, 2, 0), (1, 2, 1), (2, 1, 0), (2, 1, 1)])
def test_bruteforce_operator_skew_and_dissipative(E, N, tau):
    op, mesh, x = _operator(E, N, 0.08, tau=tau, mat=8)
    n = 9 * op.nel * op.Np
    L = np.zeros((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        L[:, c] = op.rhs(e.reshape(9, op.nel, op.Np)).ravel()
    _, J = op.geometry(np.arange(op.nel))
    MQ = np.zeros((n, n))
    for el in range(op.nel):
        Q = oracle.Q_of(op.rho[el], op.lam[el], op.mu[el])
        for p in range(9):
            for q in range(9):
                idx_p = p * op.nel * op.Np + el * op.Np + np.arange(op.Np)
                idx_q = q * op.nel * op.Np + el * op.Np + np.arange(op.Np)
                MQ[idx_p, idx_q] = Q[p, q] * op.w_vol * J[el]
    S = MQ @ L
    sym = S + S.T
    scale = np.max(np.abs(S))
    if tau == 0:
        assert np.max(np.abs(sym)) < 1e-12 * scale
    else:
        assert np.max(np.linalg.eigvalsh(0.5 * sym)) < 1e-12 * scale
        assert np.min(np.linalg.eigvalsh(0.5 * sym)) < -1e-3 * scale
    ev = np.linalg.eigvals(L)
    assert np.max(ev.real) < 1e-10 * np.max(np.abs(ev))


# --------------------------------------------------- plane wave: sign + order
def test_plane_wave_time_derivative():
    """The operator applied to the exact plane P-wave gives its time derivative."""
    op, mesh, x = _operator(2, 8, 0.05)
    u0 = wl.plane_p_wave(x, 1.0, 2.0, 1.0, t=0.0)
    dt = 1e-5
    dudt = (wl.plane_p_wave(x, 1.0, 2.0, 1.0, t=dt) - wl.plane_p_wave(x, 1.0, 2.0, 1.0, t=-dt)) / (2 * dt)
    L = op.rhs(u0)
    err = np.linalg.norm(L - dudt) / np.linalg.norm(dudt)
    assert err < 1e-3


def _l2_error(op, u, uex):
    _, J = op.geometry(np.arange(op.nel))
    d = u - uex
    return np.sqrt(np.sum(op.w_vol * J * np.sum(d * d, axis=0)))


@pytest.mark.parametrize("N,meshes,min_rate", [(2, (4, 8), 2.4), (4, (2, 4), 4.0)])
def test_plane_wave_design_order(N, meshes, min_rate):
    """L2 error at T of the plane P-wave on the warped periodic mesh falls at
    close to the design rate N+1 (pre-asymptotic meshes: the bound is N+0.4 / N)."""
    T = 0.05
    errs = []
    for E in meshes:
        op, mesh, x = _operator(E, N, 0.05)
        u = wl.plane_p_wave(x, 1.0, 2.0, 1.0, direction=(1, 0, 0))
        dt0 = oracle.cfl_dt(0.5, 1.0 / E, 2.0, N)
        nsteps = int(np.ceil(T / dt0))
        dt = T / nsteps
        res = np.zeros_like(u)
        for _ in range(nsteps):
            u, res = op.step(u, res, dt)
        errs.append(_l2_error(op, u, wl.plane_p_wave(x, 1.0, 2.0, 1.0, t=T, direction=(1, 0, 0))))
    rate = np.log2(errs[0] / errs[1])
    assert rate > min_rate, (errs, rate)


# ------------------------------------------------------- fully discrete energy
def test_energy_nonincreasing_parity_workload():
    cfg = wl.parity_config()
    r, _ = oracle.gll(cfg.N)
    d = cfg.build(r)
    m = d["mesh"]
    op = ElasticDG(cfg.N, d["x"], m.etoe, m.etof, m.orient, m.bc, d["rho"], d["lam"], d["mu"], cfg.tau)
    dt = oracle.cfl_dt(cfg.cfl, 1.0 / cfg.E, op.c_max(), cfg.N)
    assert abs(dt - 0.5 * 0.25 / (2.0 * 9)) < 1e-15
    u, res = d["u0"], np.zeros_like(d["u0"])
    E0 = op.energy(u)
    prev = E0
    for _ in range(20):
        u, res = op.step(u, res, dt)
        En = op.energy(u)
        assert En <= prev * (1 + 1e-13)
        prev = En
    assert prev > 0.5 * E0


def test_free_surface_numerical_traction_vanishes():
    """On a traction-free face the HDG flux carries no traction: the velocity rows
    of F_hat.n (= -sigma_hat n) are zero for any interior state."""
    op, mesh, x = _operator(2, 3, 0.1, periodic=(True, True, False),
                            boundary={4: wl.BC_ABSORBING, 5: wl.BC_FREE_SURFACE}, mat=9)
    u = wl.random_state(op.nel, op.Np, 14)
    elems = np.nonzero(mesh.bc[:, 5] == wl.BC_FREE_SURFACE)[0]
    Ja, J = op.geometry(elems)
    m = op.outward_scaled_normal(Ja, 5)
    nrm = m / np.linalg.norm(m, axis=-1)[..., None]
    um, up = op.exterior_state(u, elems, 5)
    um, up = np.moveaxis(um, 0, -1), np.moveaxis(up, 0, -1)
    An = np.einsum("...k,kij->...ij", nrm, oracle.dg_elastic.A_STACK)
    S = op._abs_A_cached(elems, 5, nrm)
    F = hdg_flux(An, S, um, weighted_trace(An, S, um, up))
    assert np.max(np.abs(F[..., :3])) < 1e-13
    assert np.max(np.abs(F[..., 3:])) > 1e-3


# ------------------------------------------------------------ point source
def test_ricker_closed_form_properties():
    f0, t0 = 7.0, 0.2
    t = np.linspace(t0 - 2.0, t0 + 2.0, 400001)
    R = oracle.ricker(t, f0, t0)
    assert abs(oracle.ricker(t0, f0, t0) - 1.0) < 1e-15
    assert abs(np.trapezoid(R, t)) < 1e-9                       # zero mean
    # zeros at t0 +- 1/(sqrt(2) pi f0)
    tz = t0 + 1.0 / (np.sqrt(2.0) * np.pi * f0)
    assert abs(oracle.ricker(tz, f0, t0)) < 1e-15


def test_point_source_total_force_and_location():
    """The projected source integrates to the force (partition of unity) and its
    first moment is the source location x_s = x(xi_s) (interpolated map)."""
    op, mesh, x = _operator(2, 4, 0.1)
    e, xi, F = 5, np.array([0.3, -0.55, 0.1]), np.array([0.2, -1.0, 0.5])
    op.set_point_force(e, xi, F, f0=6.0, t0=0.1)
    t = 0.13
    es, sn = op.source_nodal(t)
    _, J = op.geometry(np.array([e]))
    mass = op.w_vol * J[0]
    R = float(oracle.ricker(t, 6.0, 0.1))
    np.testing.assert_allclose(sn[:3] @ mass, F * R, rtol=1e-13)
    assert np.all(sn[3:] == 0)
    li = [oracle.lagrange_values(op.r, xi[a]) for a in range(3)]
    l3 = np.einsum("k,j,i->kji", li[2], li[1], li[0]).ravel()
    xs = l3 @ x[e]
    for c in range(3):
        np.testing.assert_allclose((sn[c] * mass) @ x[e], F[c] * R * xs, rtol=1e-12, atol=1e-15)
    # a source at a node puts the whole force on that node
    op.set_point_force(e, np.array([op.r[1], op.r[0], op.r[3]]), F, 6.0, 0.1)
    _, sn2 = op.source_nodal(t)
    node = 1 + 5 * (0 + 5 * 3)
    assert np.count_nonzero(np.abs(sn2[0]) > 1e-14) == 1 and sn2[0, node] != 0


# ------------------------------------------------------------------ adjoint
def _bc_operator(E, N, mat, rotate=None):
    return _operator(E, N, 0.08, periodic=(True, False, False),
                     boundary={2: wl.BC_FREE_SURFACE, 3: wl.BC_ABSORBING, 4: wl.BC_ABSORBING,
                               5: wl.BC_FREE_SURFACE}, mat=mat, rotate=rotate)


def test_adjoint_rhs_is_the_bruteforce_transpose():
    op, mesh, x = _bc_operator(1, 1, 21)
    n = 9 * op.nel * op.Np
    L = np.zeros((n, n))
    LT = np.zeros((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        L[:, c] = op.rhs(e.reshape(9, op.nel, op.Np)).ravel()
        LT[:, c] = op.rhs_adjoint(e.reshape(9, op.nel, op.Np)).ravel()
    np.testing.assert_allclose(LT, L.T, atol=1e-12 * np.max(np.abs(L)))


@pytest.mark.parametrize("rotate", [None, 5])
def test_adjoint_dot_products(rotate):
    op, mesh, x = _bc_operator(2, 3, 22, rotate)
    rng = np.random.default_rng(3)
    v = rng.standard_normal((9, op.nel, op.Np))
    w = rng.standard_normal((9, op.nel, op.Np))
    a, b = np.sum(w * op.rhs(v)), np.sum(op.rhs_adjoint(w) * v)
    assert abs(a - b) <= 1e-12 * abs(a)
    # one LSRK step as a linear map of (u, res)
    dt = 1e-3
    du, dr = rng.standard_normal((2, 9, op.nel, op.Np))
    lu, lr = rng.standard_normal((2, 9, op.nel, op.Np))
    u1, r1 = op.step(du, dr, dt)
    au, ar = op.adjoint_step(lu, lr, dt)
    lhs = np.sum(lu * u1) + np.sum(lr * r1)
    rhs = np.sum(au * du) + np.sum(ar * dr)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_receivers_sample_exactly_and_transpose():
    op, mesh, x = _bc_operator(2, 3, 23)
    rng = np.random.default_rng(4)
    xis = rng.uniform(-1, 1, (5, 3))
    xis[0] = [op.r[1], op.r[2], op.r[0]]                 # a receiver on a node
    op.set_receivers([0, 3, 5, 7, 2], xis)
    # a velocity field that is a polynomial of degree <= N in the reference coords
    rr = wl.mesh.reference_grid(op.r)
    u = np.zeros((9, op.nel, op.Np))
    poly = lambda p: p[..., 0] ** 3 - 2 * p[..., 1] * p[..., 2] + 0.5
    u[0] = poly(rr)[None, :]
    s = op.sample_receivers(u)
    np.testing.assert_allclose(s[:, 0], poly(xis), atol=1e-13)
    assert s[0, 0] == u[0, 0, 1 + 4 * (2 + 4 * 0)]
    g = rng.standard_normal((5, 3))
    v = rng.standard_normal((9, op.nel, op.Np))
    assert abs(np.sum(g * op.sample_receivers(v)) - np.sum(op.receivers_adjoint(g) * v)) < 1e-12


def test_adjoint_gradient_matches_finite_differences():
    op, mesh, x = _bc_operator(2, 2, 24)
    op.set_receivers([1, 6], [[0.1, -0.2, 0.3], [-0.4, 0.5, 0.0]])
    op.set_point_force(3, [0.2, 0.1, -0.3], [0.3, -0.5, 1.0], 4.0, 0.05)
    u0 = np.zeros((9, op.nel, op.Np))
    dt, nsteps = 0.02, 6
    # data: traces of a run with a perturbed medium
    saved = [v.copy() for v in (op.rho, op.lam, op.mu)]
    op.rho *= 1.05
    op.mu *= 0.97
    op._abs_cache.clear()
    op._qinv_cache.clear()
    _, data = op.forward_traces(u0, dt, nsteps)
    op.rho[:], op.lam[:], op.mu[:] = saved
    op._abs_cache.clear()
    op._qinv_cache.clear()
    pairs = [(0, 0), (3, 0), (3, 1), (5, 2), (6, 0)]     # (3, rho): the point force's element
    grad = op.gradient(u0, data, dt, nsteps, pairs)
    vals = [op.rho, op.lam, op.mu]
    for (e, p), g in zip(pairs, grad):
        base = vals[p][e]
        h = 1e-5 * abs(base)
        J = []
        for sgn in (1.0, -1.0):
            vals[p][e] = base + sgn * h
            op._abs_cache.clear()
            op._qinv_cache.clear()
            _, tr = op.forward_traces(u0, dt, nsteps)
            J.append(op.misfit(tr, data, dt))
        vals[p][e] = base
        op._abs_cache.clear()
        op._qinv_cache.clear()
        fd = (J[0] - J[1]) / (2 * h)
        assert abs(g - fd) <= 1e-6 * abs(fd), (e, p, g, fd)
