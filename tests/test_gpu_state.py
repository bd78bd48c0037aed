"""Checkpoint and resume through the C ABI (dgw_get_state / dgw_set_state):
a solve resumed from a checkpoint in a fresh context ends bit for bit where
the uninterrupted solve ends (between steps, and inside a step driven stage
by stage with the register in the checkpoint); damaged checkpoints and
checkpoints of another mesh are refused."""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _solver(mesh, x, mat, precision="fp64"):
    from paper_1711_01175_gb300 import Solver
    s = Solver(4, precision=precision)
    s.upload_mesh(x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc)
    s.upload_material(*mat)
    s.set_point_force(mesh.nel // 2, [0.1, 0.2, -0.3], [0.0, 0.0, 1.0], 6.0, 0.02)
    return s


@pytest.fixture(scope="module")
def case():
    from paper_1711_01175_gb300 import reference_nodes
    mesh = wl.structured_hex_mesh(4, (True, True, False), {4: wl.BC_ABSORBING, 5: wl.BC_FREE_SURFACE}, "morton")
    x = wl.warped_node_coords(mesh, reference_nodes(4)[0], 0.1)
    mat = wl.smooth_random_material(mesh, 3)
    return mesh, x, mat, 1e-2 * wl.random_state(mesh.nel, 125, 4)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_resume_between_steps_is_bit_exact(case, precision):
    import torch
    mesh, x, mat, u0 = case
    a = _solver(mesh, x, mat, precision)
    dt = a.dt_cfl()
    ua = torch.from_numpy(u0).cuda()
    a.step(ua, None, dt, 4)
    b = _solver(mesh, x, mat, precision)
    ub = torch.from_numpy(u0).cuda()
    b.step(ub, None, dt, 2)
    buf = b.get_state(ub, t=2 * dt, step=2)
    c = _solver(mesh, x, mat, precision)
    uc = torch.empty_like(ub)
    t, step = c.set_state(buf, uc)
    assert step == 2 and t == 2 * dt
    c.step(uc, None, dt, 2, t0=t)
    assert torch.equal(ua, uc)
    for s in (a, b, c):
        s.close()


def test_resume_inside_a_step_with_the_register(case):
    """Stages 0-2 of a step, a checkpoint with the register, stages 3-4 in a
    fresh context: the same state and register as the five stages in one go."""
    import torch
    mesh, x, mat, u0 = case
    a = _solver(mesh, x, mat)
    dt = a.dt_cfl()

    def stages(s, u, res, first, last):
        nxt = torch.empty_like(u)
        for st in range(first, last):
            s.stage(u, nxt, res, st, dt)
            u, nxt = nxt, u
        return u

    ua, ra = torch.from_numpy(u0).cuda(), torch.zeros((9, mesh.nel, 125), dtype=torch.float64, device="cuda")
    ua = stages(a, ua, ra, 0, 5)
    b = _solver(mesh, x, mat)
    ub, rb = torch.from_numpy(u0).cuda(), torch.zeros_like(ra)
    ub = stages(b, ub, rb, 0, 3)
    host = b.get_state(ub, rb, t=0.0, step=0)
    c = _solver(mesh, x, mat)
    uc, rc = torch.empty_like(ub), torch.empty_like(rb)
    c.set_state(host, uc, rc)
    uc = stages(c, uc, rc, 3, 5)
    assert torch.equal(ua, uc) and torch.equal(ra, rc)
    for s in (a, b, c):
        s.close()


def test_damaged_or_foreign_checkpoints_are_refused(case):
    import torch
    from paper_1711_01175_gb300 import DGWError
    mesh, x, mat, u0 = case
    a = _solver(mesh, x, mat)
    u = torch.from_numpy(u0).cuda()
    buf = a.get_state(u, t=0.5, step=7)
    bad = buf.copy()
    bad[100 + 8 * 1234] ^= 0x10               # one bit of the payload
    with pytest.raises(DGWError, match="checksum"):
        a.set_state(bad, torch.empty_like(u))
    with pytest.raises(DGWError, match="not a checkpoint"):
        a.set_state(np.zeros_like(buf), torch.empty_like(u))
    with pytest.raises(DGWError, match="register"):
        a.set_state(buf, torch.empty_like(u), torch.empty_like(u))
    with pytest.raises(DGWError, match="bytes"):
        from paper_1711_01175_gb300 import capi
        small = np.empty(64, dtype=np.uint8)
        a._check(capi.dgw_get_state(a._ctx, u.data_ptr(), None, 0.0, 0, small.ctypes.data, 64, None))
    other = wl.smooth_random_material(mesh, 4)       # same mesh, another medium
    b = _solver(mesh, x, other)
    with pytest.raises(DGWError, match="another mesh"):
        b.set_state(buf, torch.empty_like(u))
    target = torch.full_like(u, 3.0)
    with pytest.raises(DGWError):
        b.set_state(buf, target)
    assert bool(torch.all(target == 3.0))        # nothing copied on refusal
    a.close()
    b.close()
