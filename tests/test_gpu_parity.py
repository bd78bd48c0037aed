"""CUDA path vs the CPU oracle, element by element, through the C ABI.

FP64 path bar: relative L2 <= 1e-12 per right-hand side and per stage.
Mixed path bar: stated FP32-level bound (see MIXED_RHS_TOL).
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from harness import (BF16_RHS_TOL, FP64_TOL, MIXED_RHS_TOL, STEP10_TOL, TC_TOL, Case, assert_parity,
                     elem_max_rel, rel_l2)

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def torch_cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ------------------------------------------------------------------ rhs parity
def test_rhs_parity_workload_plane_wave():
    cfg = wl.parity_config()
    c = Case(cfg.E, cfg.N, cfg.amplitude, cfg.periodic, initial="plane_p_wave")
    assert_parity(c.gpu_rhs(c.u0), c.op.rhs(c.u0), FP64_TOL)


@pytest.mark.parametrize("N", range(1, 8))
def test_rhs_parity_every_degree_rotated_ragged(N):
    """27 elements (ragged last CTA for EPB > 1), all eight face permutation codes,
    free surface + absorbing boundaries, heterogeneous medium."""
    c = Case(3, N, 0.08, periodic=(True, False, False),
             boundary={2: wl.BC_FREE_SURFACE, 3: wl.BC_ABSORBING, 4: wl.BC_ABSORBING, 5: wl.BC_FREE_SURFACE},
             material=N, rotate=100 + N, seed=N)
    assert_parity(c.gpu_rhs(c.u0), c.op.rhs(c.u0), FP64_TOL)


def test_rhs_parity_single_self_periodic_element():
    c = Case(1, 4, 0.08, seed=3)
    assert_parity(c.gpu_rhs(c.u0), c.op.rhs(c.u0), FP64_TOL)


@pytest.mark.parametrize("tau", [0, 1])
def test_rhs_parity_flux_choice(tau):
    c = Case(3, 3, 0.1, material=7, tau=tau, seed=4)
    assert_parity(c.gpu_rhs(c.u0), c.op.rhs(c.u0), FP64_TOL)


def test_rhs_parity_large_cut():
    """16^3 cut of the large workload recipe: N=4, Morton order, warp 0.1, smooth
    random medium, z=0 absorbing, z=1 free surface."""
    cfg = wl.large_config(E=16)
    c = Case(cfg.E, cfg.N, cfg.amplitude, cfg.periodic, cfg.boundary, cfg.order, material=1,
             initial="gaussian_pulse")
    assert_parity(c.gpu_rhs(c.u0), c.op.rhs(c.u0), FP64_TOL)
    u = wl.random_state(c.mesh.nel, 125, 9)
    assert_parity(c.gpu_rhs(u), c.op.rhs(u), FP64_TOL)


# ---------------------------------------------------------------- stage parity
def _stages(c, dt):
    """Run one LSRK step stage by stage on both sides; compare after each stage."""
    import torch
    u = torch_cuda(c.u0)
    u_next = torch.empty_like(u)
    res = torch.zeros_like(u)
    uo, ro = c.u0.copy(), np.zeros_like(c.u0)
    worst = 0.0
    for s in range(5):
        c.solver.stage(u, u_next, res, s, dt)
        uo, ro = c.op.lsrk_stage(uo, ro, s, dt)
        un, rn = u_next.cpu().numpy(), res.cpu().numpy()
        worst = max(worst, rel_l2(un, uo), rel_l2(rn, ro), elem_max_rel(un, uo), elem_max_rel(rn, ro))
        u, u_next = u_next, u
    return worst


def test_stage_parity_workload():
    cfg = wl.parity_config()
    c = Case(cfg.E, cfg.N, cfg.amplitude, cfg.periodic, initial="plane_p_wave")
    dt = c.solver.dt_cfl()
    assert _stages(c, dt) < FP64_TOL


def test_stage_parity_large_cut():
    cfg = wl.large_config(E=12)
    c = Case(cfg.E, cfg.N, cfg.amplitude, cfg.periodic, cfg.boundary, cfg.order, material=1,
             initial="gaussian_pulse")
    assert _stages(c, c.solver.dt_cfl()) < FP64_TOL


def test_parity_workload_100_steps():
    """The full parity workload: 4^3, N=3, CFL 0.5, 100 LSRK steps."""
    import torch
    cfg = wl.parity_config()
    c = Case(cfg.E, cfg.N, cfg.amplitude, cfg.periodic, initial="plane_p_wave")
    dt = c.solver.dt_cfl()
    dt_or = oracle.cfl_dt(cfg.cfl, oracle.h_min_corner_edges(c.x_or, cfg.N), c.op.c_max(), cfg.N)
    assert abs(dt - dt_or) <= 1e-15 * dt_or
    u = torch_cuda(c.u0)
    res = torch.zeros_like(u)
    c.solver.step(u, res, dt, cfg.steps)
    uo, ro = c.u0.copy(), np.zeros_like(c.u0)
    for _ in range(cfg.steps):
        uo, ro = c.op.step(uo, ro, dt)
    assert_parity(u.cpu().numpy(), uo, FP64_TOL)
    assert_parity(res.cpu().numpy(), ro, 1e-11)


def test_point_source_parity_rhs_and_step():
    """Ricker point force: right-hand side at a given time and a full LSRK step
    from a nonzero start time (stage times t + c_s dt)."""
    import torch
    c = Case(3, 4, 0.1, periodic=(True, True, False), boundary={4: wl.BC_ABSORBING, 5: wl.BC_FREE_SURFACE},
             material=3, seed=2)
    u0 = 1e-3 * c.u0
    src = dict(element=13, xi=[0.3, -0.55, 0.1], force=[0.2, -1.0, 0.5], f0=6.0, t0=0.1)
    c.solver.set_point_force(**src)
    c.op.set_point_force(src["element"], src["xi"], src["force"], src["f0"], src["t0"])
    ud = torch_cuda(u0)
    out = torch.empty_like(ud)
    c.solver.rhs(ud, out, t=0.13)
    assert_parity(out.cpu().numpy(), c.op.rhs(u0, t=0.13), FP64_TOL)
    dt = c.solver.dt_cfl()
    res = torch.zeros_like(ud)
    c.solver.step(ud, res, dt, 2, t0=0.08)
    uo, ro = u0.copy(), np.zeros_like(u0)
    for k in range(2):
        uo, ro = c.op.step(uo, ro, dt, t=0.08 + k * dt)
    assert_parity(ud.cpu().numpy(), uo, FP64_TOL)
    # removing the source restores the source-free operator
    c.solver.set_point_force(-1, [0, 0, 0], [0, 0, 0], 1.0, 0.0)
    c.op.source = None
    c.solver.rhs(torch_cuda(u0), out, t=0.13)
    assert_parity(out.cpu().numpy(), c.op.rhs(u0, t=0.13), FP64_TOL)


# ---------------------------------------------------------------------- energy
def test_energy_parity_and_decay():
    import torch
    cfg = wl.large_config(E=8)
    c = Case(cfg.E, cfg.N, cfg.amplitude, cfg.periodic, cfg.boundary, cfg.order, material=1,
             initial="gaussian_pulse")
    u = torch_cuda(c.u0)
    e_gpu = c.solver.energy(u)
    e_or = c.op.energy(c.u0)
    assert abs(e_gpu - e_or) <= 1e-13 * e_or
    assert c.solver.energy(u) == e_gpu            # fixed reduction order: bit-reproducible
    res = torch.zeros_like(u)
    dt = c.solver.dt_cfl()
    prev = e_gpu
    for _ in range(10):
        c.solver.step(u, res, dt, 2)
        e = c.solver.energy(u)
        assert e <= prev * (1 + 1e-13)
        prev = e


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fused_stage_energy_matches_separate_calls(precision):
    """dgw_stage_energy writes the same stage output as dgw_stage and returns the
    energy of u_out as dgw_energy computes it (different summation order)."""
    import torch
    cfg = wl.large_config(E=6)
    c = Case(cfg.E, cfg.N, cfg.amplitude, cfg.periodic, cfg.boundary, cfg.order, material=1,
             initial="gaussian_pulse", precision=precision)
    dt = c.solver.dt_cfl()
    for s in (0, 3):
        u = torch_cuda(c.u0)
        res0 = torch_cuda(wl.random_state(c.mesh.nel, 125, 5 + s)) * 1e-3
        out_a, out_b = torch.empty_like(u), torch.empty_like(u)
        res_a, res_b = res0.clone(), res0.clone()
        c.solver.stage(u, out_a, res_a, s, dt)
        e = c.solver.stage_energy(u, out_b, res_b, s, dt)
        assert torch.equal(out_a, out_b) and torch.equal(res_a, res_b)
        e_ref = c.solver.energy(out_b)
        assert abs(e - e_ref) <= 1e-13 * e_ref
        if precision == "fp64":
            assert abs(e - c.op.energy(out_b.cpu().numpy())) <= 1e-13 * e_ref


def test_host_pointer_paths_match_device_paths():
    import torch
    c = Case(3, 4, 0.1, material=2, seed=8)
    dt = c.solver.dt_cfl()
    u_h = c.u0.copy()
    r_h = np.zeros_like(u_h)
    c.solver.step(u_h, r_h, dt, 2)
    u_d = torch_cuda(c.u0)
    r_d = torch.zeros_like(u_d)
    c.solver.step(u_d, r_d, dt, 2)
    assert np.array_equal(u_h, u_d.cpu().numpy())
    assert np.array_equal(r_h, r_d.cpu().numpy())
    out_h = np.empty_like(u_h)
    c.solver.rhs(c.u0, out_h)
    assert np.array_equal(out_h, c.gpu_rhs(c.u0))
    assert c.solver.energy(u_h) == c.solver.energy(u_d)


# -------------------------------------------------------------- mixed precision
@pytest.mark.parametrize("precision", ["mixed", "mixed_tc", "mixed_tc_bf16"])
def test_mixed_precision_rhs_bound(precision):
    cfg = wl.large_config(E=8)
    for initial in ("gaussian_pulse", "random"):
        c = Case(cfg.E, cfg.N, cfg.amplitude, cfg.periodic, cfg.boundary, cfg.order, material=1,
                 initial=initial, precision=precision)
        assert_parity(c.gpu_rhs(c.u0), c.op.rhs(c.u0), TC_TOL[precision], label=f"{precision} 8^3 {initial}")


@pytest.mark.parametrize("precision", ["mixed_tc", "mixed_tc_bf16"])
@pytest.mark.parametrize("N", range(1, 8))
def test_tensor_core_rhs_every_degree_rotated_ragged(N, precision):
    """The tensor-core volume form at every degree: 27 rotated elements (all
    eight face permutations, ragged last CTA for N <= 3), free-surface and
    absorbing faces, heterogeneous medium, random state."""
    c = Case(3, N, 0.08, periodic=(True, False, False),
             boundary={2: wl.BC_FREE_SURFACE, 3: wl.BC_ABSORBING, 4: wl.BC_ABSORBING, 5: wl.BC_FREE_SURFACE},
             material=N, rotate=100 + N, seed=N, precision=precision)
    assert_parity(c.gpu_rhs(c.u0), c.op.rhs(c.u0), TC_TOL[precision], label=f"{precision} N={N}")


@pytest.mark.parametrize("precision", ["mixed_tc", "mixed_tc_bf16"])
def test_tensor_core_rhs_scale_invariance(precision):
    """Stresses 1e6 times the velocities (a medium in SI-like units): the FP16
    form's per-row power-of-two scaling keeps the same relative accuracy, and
    the state's own scale does not enter either form."""
    c = Case(3, 4, 0.1, material=2, seed=11, precision=precision)
    u = c.u0.copy()
    u[3:] *= 1e6
    want = c.op.rhs(u)
    assert_parity(c.gpu_rhs(u), want, TC_TOL[precision], label=f"{precision} stress x 1e6")
    assert_parity(c.gpu_rhs(1e-30 * u), 1e-30 * want, TC_TOL[precision], label=f"{precision} state x 1e-30")


@pytest.mark.parametrize("precision", ["mixed", "mixed_tc", "mixed_tc_bf16"])
def test_mixed_precision_step_bound(precision):
    """Ten LSRK steps of the parity workload (4^3, N=3, plane wave, CFL 0.5)
    against the FP64 oracle: the FP32 right-hand side error (~1e-7 per stage)
    accumulates over 50 stages with dt ~ 7e-3."""
    import torch
    cfg = wl.parity_config()
    c = Case(cfg.E, cfg.N, cfg.amplitude, cfg.periodic, initial="plane_p_wave", precision=precision)
    dt = c.solver.dt_cfl()
    u = torch_cuda(c.u0)
    res = torch.zeros_like(u)
    c.solver.step(u, res, dt, 10)
    uo, ro = c.u0.copy(), np.zeros_like(c.u0)
    for _ in range(10):
        uo, ro = c.op.step(uo, ro, dt)
    assert_parity(u.cpu().numpy(), uo, STEP10_TOL[precision], label=f"{precision} 10 steps")


@pytest.mark.parametrize("N", range(1, 8))
def test_mixed_step_every_degree_rotated_ragged(N):
    """Three LSRK steps of the mixed path at every degree on the rotated ragged
    27-element mesh against the FP64 oracle: the FP32 stage takes per-degree
    choices in its LSRK mode (L1 prefetch of the register and the neighbour
    traces, L2 prefetch distance, shared-memory carveout) that the right-hand
    side tests do not reach.  The steps are stable ones: CFL 0.125 at N = 1 and
    0.4 at N = 2, where the convention dt = CFL h / (c N^2) at the default 0.5
    lies beyond the LSRK(5,4) stability limit for a rough state (the oracle
    alone: limits 0.125-0.15 and 0.45-0.5), 0.5 from N = 3 on.  Bound: the
    mixed step bound, 1e-6 (measured 7-10e-8 at every degree, element max up to
    2.3e-7 at N = 1; at CFL 0.5, where N = 1 and 2 are unstable, 1.1e-6)."""
    import torch
    c = Case(3, N, 0.08, periodic=(True, False, False),
             boundary={2: wl.BC_FREE_SURFACE, 3: wl.BC_ABSORBING, 4: wl.BC_ABSORBING, 5: wl.BC_FREE_SURFACE},
             material=N, rotate=100 + N, seed=N, precision="mixed")
    dt = c.solver.dt_cfl() * {1: 0.125, 2: 0.4}.get(N, 0.5) / 0.5
    u = torch_cuda(c.u0)
    res = torch.zeros_like(u)
    c.solver.step(u, res, dt, 3)
    uo, ro = c.u0.copy(), np.zeros_like(c.u0)
    for _ in range(3):
        uo, ro = c.op.step(uo, ro, dt)
    assert_parity(u.cpu().numpy(), uo, STEP10_TOL["mixed"], label=f"mixed N={N} 3 steps")


@pytest.mark.parametrize("precision", ["mixed_tc", "mixed_tc_bf16"])
def test_tensor_core_stage_and_fused_energy(precision):
    """The tensor-core form through the fused LSRK stage (register update in FP64)
    and the fused-energy stage, on a 6^3 cut of the large workload: stage output
    against the oracle's stage, and the fused energy against dgw_energy."""
    import torch
    cfg = wl.large_config(E=6)
    c = Case(cfg.E, cfg.N, cfg.amplitude, cfg.periodic, cfg.boundary, cfg.order, material=1,
             initial="gaussian_pulse", precision=precision)
    dt = c.solver.dt_cfl()
    u = torch_cuda(c.u0)
    res0 = torch_cuda(wl.random_state(c.mesh.nel, 125, 5)) * 1e-3
    out_a, out_b = torch.empty_like(u), torch.empty_like(u)
    res_a, res_b = res0.clone(), res0.clone()
    c.solver.stage(u, out_a, res_a, 2, dt)
    e = c.solver.stage_energy(u, out_b, res_b, 2, dt)
    assert torch.equal(out_a, out_b) and torch.equal(res_a, res_b)
    assert abs(e - c.solver.energy(out_b)) <= 1e-13 * e
    uo, ro = c.op.lsrk_stage(c.u0, res0.cpu().numpy(), 2, dt)
    # the stage changes u by b_s res ~ dt L(u): compare the increments
    assert_parity(out_a.cpu().numpy() - c.u0, uo - c.u0, TC_TOL[precision], label=f"{precision} stage increment")
    assert_parity(res_a.cpu().numpy(), ro, TC_TOL[precision], label=f"{precision} stage register")


# ------------------------------------------------------------------ full size
def test_full_size_large_workload_sampled():
    """64^3, N=4 (the benchmark workload, same launch path): the right-hand side of a
    random state and the first stage from the initial pulse, on sampled elements
    (interior, free-surface and absorbing layers) computed one by one by the oracle."""
    import torch
    cfg = wl.large_config()
    c = Case(cfg.E, cfg.N, cfg.amplitude, cfg.periodic, cfg.boundary, cfg.order, material=1,
             initial="gaussian_pulse")
    nel = c.mesh.nel
    rng = np.random.default_rng(0)
    bottom = np.nonzero(c.mesh.bc[:, 4] == wl.BC_ABSORBING)[0]
    top = np.nonzero(c.mesh.bc[:, 5] == wl.BC_FREE_SURFACE)[0]
    centre = np.nonzero(np.all(c.mesh.cell == 32, axis=1))[0]
    sample = np.unique(np.concatenate([rng.choice(nel, 24, replace=False), rng.choice(bottom, 4),
                                       rng.choice(top, 4), centre, [0, nel - 1]]))
    u = wl.random_state(nel, 125, 21)
    got = c.gpu_rhs(u)[:, sample]
    want = c.op.rhs(u, sample)
    assert_parity(got, want, FP64_TOL)
    # first LSRK stage from the Gaussian pulse
    ud = torch_cuda(c.u0)
    uo_d = torch.empty_like(ud)
    res = torch.zeros_like(ud)
    dt = c.solver.dt_cfl()
    c.solver.stage(ud, uo_d, res, 0, dt)
    u1, r1 = c.op.lsrk_stage(c.u0, np.zeros_like(c.u0), 0, dt, sample)
    assert_parity(uo_d.cpu().numpy()[:, sample], u1, FP64_TOL)
    assert_parity(res.cpu().numpy()[:, sample], r1, FP64_TOL)


def test_full_size_precision_workload_sampled():
    """48^3, N=7 (the precision recipe at full size, 110,592 elements, the launch
    path the bench times): the right-hand side of a random state on sampled
    elements (interior, free-surface and absorbing layers) computed one by one by
    the oracle -- FP64 to 1e-12, and the mixed path on the same sample to its
    FP32 bound."""
    import torch
    from paper_1711_01175_gb300 import Solver
    cfg = wl.precision_config()
    c = Case(cfg.E, cfg.N, cfg.amplitude, cfg.periodic, cfg.boundary, cfg.order, material=cfg.material_seed)
    nel, Np = c.mesh.nel, (cfg.N + 1) ** 3
    rng = np.random.default_rng(4)
    bottom = np.nonzero(c.mesh.bc[:, 4] == wl.BC_ABSORBING)[0]
    top = np.nonzero(c.mesh.bc[:, 5] == wl.BC_FREE_SURFACE)[0]
    sample = np.unique(np.concatenate([rng.choice(nel, 24, replace=False), rng.choice(bottom, 6),
                                       rng.choice(top, 6), [0, nel - 1]]))
    u = wl.random_state(nel, Np, 22)
    want = c.op.rhs(u, sample)
    assert_parity(c.gpu_rhs(u)[:, sample], want, FP64_TOL, label="48^3 N=7 sampled FP64")
    ud = torch.from_numpy(u).cuda()
    out = torch.empty_like(ud)
    for prec in ("mixed", "mixed_tc", "mixed_tc_bf16"):
        m = Solver(cfg.N, precision=prec)
        m.upload_mesh(c.x_lib, c.mesh.etoe, c.mesh.etof, c.mesh.orient, c.mesh.bc)
        m.upload_material(c.rho, c.lam, c.mu)
        m.rhs(ud, out)
        assert_parity(out.cpu().numpy()[:, sample], want, TC_TOL[prec], label=f"48^3 N=7 sampled {prec}")
        m.close()


# -------------------------------------------------------------- argument errors
def test_call_order_and_argument_errors():
    import torch
    from paper_1711_01175_gb300 import DGWError, Solver
    s = Solver(3)
    u = torch.zeros(9, 8, 64, dtype=torch.float64, device="cuda")
    with pytest.raises(DGWError, match="DGW_ERR_STATE"):
        s.rhs(u, torch.empty_like(u))
    mesh = wl.structured_hex_mesh(2)
    from paper_1711_01175_gb300 import reference_nodes
    r, _ = reference_nodes(3)
    x = wl.warped_node_coords(mesh, r, 0.05)
    bad = mesh.etoe.copy()
    bad[0, 1] = 5
    with pytest.raises(DGWError, match="symmetric|neighbour"):
        s.upload_mesh(x, bad, mesh.etof, mesh.orient, mesh.bc)
    badbc = mesh.bc.copy()
    badbc[0, 0] = 1
    with pytest.raises(DGWError, match="bc tag"):
        s.upload_mesh(x, mesh.etoe, mesh.etof, mesh.orient, badbc)
    # mirrored element: J < 0
    xf = x.copy()
    xf[3, :, 0] = 2 * xf[3, :, 0].mean() - xf[3, :, 0]
    with pytest.raises(DGWError, match="Jacobian"):
        s.upload_mesh(xf, mesh.etoe, mesh.etof, mesh.orient, mesh.bc)
    s.upload_mesh(x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc)
    with pytest.raises(DGWError, match="DGW_ERR_STATE"):
        s.rhs(u, torch.empty_like(u))
    rho, lam, mu = wl.homogeneous_material(8)
    with pytest.raises(DGWError, match="rho > 0"):
        s.upload_material(-rho, lam, mu)
    with pytest.raises(DGWError, match="rho > 0"):
        s.upload_material(rho, -mu, mu)
    s.upload_material(rho, lam, mu)
    with pytest.raises(DGWError, match="distinct"):
        s.rhs(u, u)
    with pytest.raises(DGWError, match="distinct"):
        s.stage(u, u, torch.zeros_like(u), 0, 1e-3)
    with pytest.raises(DGWError, match="stage"):
        s.stage(u, torch.empty_like(u), torch.zeros_like(u), 5, 1e-3)
    from paper_1711_01175_gb300 import capi
    assert capi.dgw_adjoint_step(s._ctx, None, None, None, None, 0.0, 0.1, 1, None) == -1
    s.close()


def test_size_limits_and_empty_calls():
    """nel <= 0 and nel Np >= 2^31 (32-bit node indices) are refused before any
    array is read; nsteps = 0 leaves the state and register as they are; a
    non-finite dt is refused."""
    import ctypes
    import torch
    from paper_1711_01175_gb300 import Solver, capi, reference_nodes
    s = Solver(3)
    one = np.zeros(64, dtype=np.float64)
    i64 = np.zeros(6, dtype=np.int64)
    i8 = np.zeros(6, dtype=np.int8)
    ptrs = [one.ctypes.data, i64.ctypes.data, i8.ctypes.data, i8.ctypes.data, i8.ctypes.data]
    assert capi.dgw_mesh_upload(s._ctx, 0, *ptrs) == -1
    assert capi.dgw_mesh_upload(s._ctx, -4, *ptrs) == -1
    assert capi.dgw_mesh_upload(s._ctx, (1 << 31) // 64 + 1, *ptrs) == -1
    assert "2^31" in capi.dgw_last_error(s._ctx)
    mesh = wl.structured_hex_mesh(2)
    x = wl.warped_node_coords(mesh, reference_nodes(3)[0], 0.05)
    s.upload_mesh(x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc)
    s.upload_material(*wl.homogeneous_material(mesh.nel))
    u0 = wl.random_fields(9, mesh.nel, 64, 3)
    u = torch.from_numpy(u0).cuda()
    r = torch.full_like(u, 7.0)
    s.step(u, r, 1e-3, 0)
    assert np.array_equal(u.cpu().numpy(), u0) and bool(torch.all(r == 7.0))
    assert capi.dgw_step(s._ctx, u.data_ptr(), r.data_ptr(), 0.0, float("nan"), 1, None) == -1
    s.close()
