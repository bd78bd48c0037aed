"""Hand-written adjoint: parity with the oracle's adjoint and finite differences.

* one adjoint step (lu, lr) against the oracle's stage-by-stage transpose;
* receiver sampling and its transpose against the oracle;
* the material gradient of a receiver misfit against the oracle's adjoint
  gradient, and -- through the autograd function, with several checkpoint
  segments -- against central differences of the misfit on 20 random
  (element, parameter) pairs (1e-6 relative).
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from harness import assert_parity, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def problem(E=2, N=3, seed=31):
    from paper_1711_01175_gb300 import Solver, reference_nodes
    mesh = wl.structured_hex_mesh(E, (True, False, False),
                                  {2: wl.BC_FREE_SURFACE, 3: wl.BC_ABSORBING, 4: wl.BC_ABSORBING, 5: wl.BC_FREE_SURFACE})
    rho, lam, mu = wl.smooth_random_material(mesh, seed)
    r, _ = reference_nodes(N)
    x = wl.warped_node_coords(mesh, r, 0.08)
    s = Solver(N)
    s.upload_mesh(x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc)
    s.upload_material(rho, lam, mu)
    src = dict(element=min(3, mesh.nel - 1), xi=[0.2, 0.1, -0.3], force=[0.3, -0.5, 1.0], f0=4.0, t0=0.05)
    s.set_point_force(**src)
    rec_el = np.array([1 % mesh.nel, (mesh.nel * 3) // 4])
    rec_xi = np.array([[0.1, -0.2, 0.3], [-0.4, 0.5, 0.0]])
    s.set_receivers(rec_el, rec_xi)
    ro, _ = oracle.gll(N)
    xo = wl.warped_node_coords(mesh, ro, 0.08)
    op = oracle.ElasticDG(N, xo, mesh.etoe, mesh.etof, mesh.orient, mesh.bc, rho.copy(), lam.copy(), mu.copy(), 1)
    op.set_point_force(src["element"], src["xi"], src["force"], src["f0"], src["t0"])
    op.set_receivers(rec_el, rec_xi)
    return s, op, mesh, (rho, lam, mu)


def test_adjoint_step_and_receivers_match_oracle():
    import torch
    s, op, mesh, _ = problem()
    rng = np.random.default_rng(1)
    shape = (9, mesh.nel, 64)
    lu0, lr0, u0 = rng.standard_normal((3,) + shape)
    dt = 0.02
    lu = torch.from_numpy(lu0).cuda()
    lr = torch.from_numpy(lr0).cuda()
    grad = torch.zeros((3, mesh.nel), dtype=torch.float64, device="cuda")
    s.adjoint_step(lu, lr, grad, torch.from_numpy(u0).cuda(), dt, 1, t0=0.01)
    lu_o, lr_o = op.adjoint_step(lu0, lr0, dt)
    assert_parity(lu.cpu().numpy(), lu_o, 1e-12)
    # after a full step the register adjoint is a_0 w = 0 exactly on both sides
    assert np.all(lr.cpu().numpy() == 0.0) and np.all(lr_o == 0.0)
    out = torch.empty((2, 3), dtype=torch.float64, device="cuda")
    s.sample_receivers(torch.from_numpy(u0).cuda(), out)
    np.testing.assert_allclose(out.cpu().numpy(), op.sample_receivers(u0), rtol=1e-13, atol=1e-14)
    g = rng.standard_normal((2, 3))
    acc = torch.from_numpy(lu0).cuda()
    s.receivers_adjoint(acc, torch.from_numpy(g).cuda())
    np.testing.assert_allclose(acc.cpu().numpy() - lu0, op.receivers_adjoint(g), atol=1e-13)


def _misfit_setup(s, op, mesh, mat, nsteps, dt):
    """Zero initial state and seeded synthetic receiver data (the misfit gradient
    identity holds for any data)."""
    import torch
    u0 = torch.zeros((9, mesh.nel, (s.N + 1) ** 3), dtype=torch.float64, device="cuda")
    data = 1e-3 * np.random.default_rng(11).standard_normal((nsteps, 2, 3))
    return u0, torch.from_numpy(data).cuda()


def test_gradient_matches_oracle_adjoint():
    import torch
    from paper_1711_01175_gb300.adjoint import receiver_traces
    s, op, mesh, mat = problem()
    dt, nsteps = 0.02, 4
    u0, data = _misfit_setup(s, op, mesh, mat, nsteps, dt)
    m = torch.tensor(np.stack(mat), requires_grad=True)
    tr = receiver_traces(m, s, u0, dt, nsteps, checkpoint_every=3)
    J = 0.5 * dt * torch.sum((tr - data) ** 2)
    J.backward()
    g = m.grad.numpy()
    pairs = [(0, 0), (3, 0), (3, 1), (5, 2), (6, 0), (7, 1)]
    go = op.gradient(np.zeros((9, mesh.nel, 64)), 1e-3 * np.random.default_rng(11).standard_normal((nsteps, 2, 3)),
                     dt, nsteps, pairs)
    for (e, p), ref in zip(pairs, go):
        assert abs(g[p, e] - ref) <= 1e-7 * np.max(np.abs(go)), (e, p, g[p, e], ref)


def test_gradient_matches_central_differences():
    import torch
    from paper_1711_01175_gb300.adjoint import receiver_traces
    s, op, mesh, mat = problem(E=3, N=3, seed=32)
    dt, nsteps = 0.015, 20
    u0, data = _misfit_setup(s, op, mesh, mat, nsteps, dt)
    base = np.stack(mat)
    m = torch.tensor(base, requires_grad=True)
    tr = receiver_traces(m, s, u0, dt, nsteps, checkpoint_every=6)
    J = 0.5 * dt * torch.sum((tr - data) ** 2)
    J.backward()
    g = m.grad.numpy()

    def misfit(mm):
        with torch.no_grad():
            t = receiver_traces(torch.tensor(mm), s, u0, dt, nsteps)
        return 0.5 * dt * float(torch.sum((t - data) ** 2))

    rng = np.random.default_rng(7)
    pairs = [(int(rng.integers(mesh.nel)), int(rng.integers(3))) for _ in range(20)]
    scale = np.max(np.abs(g))
    for e, p in pairs:
        h = 1e-6 * base[p, e]
        mp, mm_ = base.copy(), base.copy()
        mp[p, e] += h
        mm_[p, e] -= h
        fd = (misfit(mp) - misfit(mm_)) / (2 * h)
        assert abs(g[p, e] - fd) <= 1e-6 * max(abs(fd), 1e-3 * scale), (e, p, g[p, e], fd)


def test_adjoint_refuses_mixed_precision():
    import torch
    from paper_1711_01175_gb300 import Solver, capi
    s = Solver(2, precision="mixed")
    mesh = wl.structured_hex_mesh(1)
    from paper_1711_01175_gb300 import reference_nodes
    s.upload_mesh(wl.warped_node_coords(mesh, reference_nodes(2)[0], 0.05), mesh.etoe, mesh.etof, mesh.orient, mesh.bc)
    s.upload_material(*wl.homogeneous_material(1))
    z = torch.zeros((9, 1, 27), dtype=torch.float64, device="cuda")
    g = torch.zeros((3, 1), dtype=torch.float64, device="cuda")
    st = capi.dgw_adjoint_step(s._ctx, z.data_ptr(), z.clone().data_ptr(), g.data_ptr(), z.clone().data_ptr(),
                               0.0, 0.01, 1, None)
    assert st == -7


def test_gradient_of_a_perturbed_medium_misfit_at_stable_time_steps():
    """The bench's experiment at small size: CFL 0.5 steps, a Ricker force at the
    centre element active within the window, receivers in the source element
    and its face neighbours, data from the same experiment in a 5 %-perturbed
    medium.  Central differences agree with the adjoint gradient to 1e-6
    relative on its ten largest entries and five random ones."""
    import torch
    from paper_1711_01175_gb300.adjoint import receiver_traces
    s, op, mesh, mat = problem(E=3, N=3, seed=33)
    dt = s.dt_cfl()
    nsteps = 30
    centre = int(np.nonzero(np.all(mesh.cell == 1, axis=1))[0][0])
    f0 = 3.0 / (nsteps * dt)
    s.set_point_force(centre, [0.1, -0.2, 0.3], [0.0, 0.0, 1.0], f0, 1.2 / f0)
    rng = np.random.default_rng(21)
    near = [centre] + [int(e) for e in mesh.etoe[centre] if e >= 0]
    s.set_receivers(rng.choice(near, 4), rng.uniform(-0.9, 0.9, (4, 3)))
    base = np.stack(mat)
    u0 = torch.zeros((9, mesh.nel, 64), dtype=torch.float64, device="cuda")
    with torch.no_grad():
        data = receiver_traces(torch.tensor(base * (1 + 0.05 * rng.uniform(-1, 1, base.shape))), s, u0, dt,
                               nsteps).clone()
    m = torch.tensor(base, requires_grad=True)
    tr = receiver_traces(m, s, u0, dt, nsteps, checkpoint_every=7)
    J = 0.5 * dt * torch.sum((tr - data) ** 2)
    J.backward()
    g = m.grad.numpy()
    assert float(J.detach()) > 0 and np.all(np.isfinite(g))

    def misfit(mm):
        with torch.no_grad():
            t = receiver_traces(torch.tensor(mm), s, u0, dt, nsteps)
        return 0.5 * dt * float(torch.sum((t - data) ** 2))

    order = np.argsort(-np.abs(g).ravel())
    picks = list(order[:10]) + [int(i) for i in rng.choice(g.size, 5, replace=False)]
    scale = np.max(np.abs(g))
    for flat in picks:
        p, e = np.unravel_index(flat, g.shape)
        h = 1e-6 * base[p, e]
        mp, mm_ = base.copy(), base.copy()
        mp[p, e] += h
        mm_[p, e] -= h
        fd = (misfit(mp) - misfit(mm_)) / (2 * h)
        assert abs(g[p, e] - fd) <= 1e-6 * max(abs(fd), 1e-3 * scale), (e, p, g[p, e], fd)


def test_adjoint_traces_segment_matches_step_by_step():
    """dgw_adjoint_traces over a segment of 5 steps (one forward recompute, every
    stage input kept) equals five dgw_adjoint_step calls of one step each with
    dgw_receivers_adjoint between them (a recompute per step): the same
    arithmetic in the same order, so lam_u, lam_res and the gradient agree to
    rounding."""
    import torch
    s, op, mesh, _ = problem(E=3, N=3, seed=34)
    rng = np.random.default_rng(5)
    shape = (9, mesh.nel, 64)
    u0 = torch.from_numpy(1e-2 * rng.standard_normal(shape)).cuda()
    g = torch.from_numpy(rng.standard_normal((5, 2, 3))).cuda()
    lu0 = rng.standard_normal(shape)
    dt, t0 = 0.01, 0.03
    out = []
    for mode in ("segment", "steps"):
        lu = torch.from_numpy(lu0).cuda()
        lr = torch.zeros_like(lu)
        grad = torch.zeros((3, mesh.nel), dtype=torch.float64, device="cuda")
        if mode == "segment":
            s.adjoint_traces(lu, lr, grad, u0, g, dt, 5, t0=t0)
        else:
            starts, u, res = [], u0.clone(), torch.zeros_like(u0)
            for k in range(5):
                starts.append(u.clone())
                s.step(u, res, dt, 1, t0=t0 + k * dt)
            for k in reversed(range(5)):
                s.receivers_adjoint(lu, g[k])
                s.adjoint_step(lu, lr, grad, starts[k], dt, 1, t0=t0 + k * dt)
        out.append((lu.cpu().numpy(), lr.cpu().numpy(), grad.cpu().numpy()))
    for a, b in zip(out[0], out[1]):
        assert rel_l2(a, b) < 1e-13 or np.array_equal(a, b)


def test_gradient_central_differences_at_recipe_size():
    """The adjoint recipe at full size: 32^3 hex mesh (warp 0.1, smooth random
    medium, free surface on top, absorbing bottom), N=4, 500 LSRK steps at CFL 0.5,
    a Ricker point force at the centre element, 32 receivers recording velocity in
    the elements within two faces of it, data from the same experiment in a
    5 %-perturbed medium, L2 misfit, checkpoints every 50 steps.  The adjoint
    gradient against central differences of the misfit on 20 random (element,
    parameter) pairs of the elements within four faces of the source, to 1e-6
    relative (absolute floor 1e-3 of the largest gradient entry)."""
    import torch
    from harness import graph_distance
    from paper_1711_01175_gb300 import Solver, reference_nodes
    from paper_1711_01175_gb300.adjoint import receiver_traces
    E, N, nsteps, every = 32, 4, 500, 50
    mesh = wl.structured_hex_mesh(E, (True, True, False), {4: wl.BC_ABSORBING, 5: wl.BC_FREE_SURFACE}, "morton")
    x = wl.warped_node_coords(mesh, reference_nodes(N)[0], 0.1)
    rho, lam, mu = wl.smooth_random_material(mesh, 5)
    s = Solver(N)
    s.upload_mesh(x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc)
    s.upload_material(rho, lam, mu)
    dt = s.dt_cfl()
    centre = int(np.nonzero(np.all(mesh.cell == E // 2, axis=1))[0][0])
    f0 = 3.0 / (nsteps * dt)
    s.set_point_force(centre, [0.1, -0.2, 0.3], [0.0, 0.0, 1.0], f0, 1.2 / f0)
    rng = np.random.default_rng(19)
    dist = graph_distance(mesh.etoe, [centre], 4)
    s.set_receivers(rng.choice(np.nonzero(dist <= 2)[0], 32), rng.uniform(-0.9, 0.9, (32, 3)))
    base = np.stack([rho, lam, mu])
    u0 = torch.zeros((9, mesh.nel, (N + 1) ** 3), dtype=torch.float64, device="cuda")
    with torch.no_grad():
        data = receiver_traces(torch.tensor(base * (1 + 0.05 * rng.uniform(-1, 1, base.shape))), s, u0, dt,
                               nsteps, checkpoint_every=nsteps).clone()
    m = torch.tensor(base, requires_grad=True)
    tr = receiver_traces(m, s, u0, dt, nsteps, checkpoint_every=every)
    J = 0.5 * dt * torch.sum((tr - data) ** 2)
    J.backward()
    g = m.grad.numpy()
    assert float(J.detach()) > 0 and np.all(np.isfinite(g))

    def misfit(mm):
        with torch.no_grad():
            t = receiver_traces(torch.tensor(mm), s, u0, dt, nsteps, checkpoint_every=nsteps)
        return 0.5 * dt * float(torch.sum((t - data) ** 2))

    near = np.nonzero(dist <= 4)[0]
    pairs = [(int(rng.choice(near)), int(rng.integers(3))) for _ in range(20)]
    scale = np.max(np.abs(g))
    worst = 0.0
    for e, p in pairs:
        h = 1e-6 * base[p, e]
        mp, mm_ = base.copy(), base.copy()
        mp[p, e] += h
        mm_[p, e] -= h
        fd = (misfit(mp) - misfit(mm_)) / (2 * h)
        err = abs(g[p, e] - fd) / max(abs(fd), 1e-3 * scale)
        worst = max(worst, err)
        assert err <= 1e-6, (e, p, g[p, e], fd)
    print(f"adjoint recipe 32^3 N=4 500 steps: misfit {float(J.detach()):.3e}, worst FD relative error {worst:.2e}")
    s.close()


def test_low_memory_adjoint_gives_the_same_gradient():
    """The adjoint keeps every stage's operator output for the gradient terms
    (default) or, with DGW_ADJOINT_LOW_MEMORY=1, recomputes it (the path taken
    when the larger scratch does not fit): the same lam_u and register, and the
    same gradient to rounding (the operator output is scaled by dt at another
    point of the arithmetic)."""
    import os
    import torch
    s, op, mesh, _ = problem(E=3, N=3, seed=35)
    rng = np.random.default_rng(6)
    shape = (9, mesh.nel, 64)
    u0 = torch.from_numpy(1e-2 * rng.standard_normal(shape)).cuda()
    g = torch.from_numpy(rng.standard_normal((4, 2, 3))).cuda()
    lu0 = rng.standard_normal(shape)
    out = []
    for low in ("0", "1"):
        os.environ["DGW_ADJOINT_LOW_MEMORY"] = low
        try:
            lu = torch.from_numpy(lu0).cuda()
            lr = torch.zeros_like(lu)
            grad = torch.zeros((3, mesh.nel), dtype=torch.float64, device="cuda")
            s.adjoint_traces(lu, lr, grad, u0, g, 0.01, 4, t0=0.02)
            out.append((lu.cpu().numpy(), lr.cpu().numpy(), grad.cpu().numpy()))
        finally:
            del os.environ["DGW_ADJOINT_LOW_MEMORY"]
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert rel_l2(out[0][2], out[1][2]) < 1e-13
