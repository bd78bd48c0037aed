"""dgw_step / dgw_step_energy contract on the GPU, through the C ABI.

* the first stage never reads the register (a_0 = 0): a register full of NaN
  gives the same step as a zero one, for device and host buffers;
* res = NULL (the context's own register) gives the same state;
* dgw_step_energy gives the state of dgw_step and the energy of dgw_energy
  on it (fused into the last stage: agreement to rounding), FP64 and mixed,
  elastic and a generic system; host buffers give the device results.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _elastic(precision, E=4, N=3):
    from paper_1711_01175_gb300 import Solver, reference_nodes
    cfg = wl.large_config(E=E, N=N)
    w = cfg.build(reference_nodes(N)[0])
    m = w["mesh"]
    s = Solver(N, precision=precision)
    s.upload_mesh(w["x"], m.etoe, m.etof, m.orient, m.bc)
    s.upload_material(w["rho"], w["lam"], w["mu"])
    u0 = w["u0"] + 0.1 * wl.random_fields(9, m.nel, (N + 1) ** 3, 4)
    return s, u0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_register_is_not_read_and_may_be_omitted(precision):
    import torch
    s, u0 = _elastic(precision)
    dt = s.dt_cfl()
    ref = torch.from_numpy(u0).cuda()
    r0 = torch.zeros_like(ref)
    s.step(ref, r0, dt, 3)
    u = torch.from_numpy(u0).cuda()
    rn = torch.full_like(u, float("nan"))
    s.step(u, rn, dt, 3)
    assert torch.equal(u, ref) and torch.equal(rn, r0)
    u = torch.from_numpy(u0).cuda()
    s.step(u, None, dt, 3)
    assert torch.equal(u, ref)
    uh = u0.copy()
    rh = np.full_like(u0, np.nan)
    s.step(uh, rh, dt, 3)
    assert np.array_equal(uh, ref.cpu().numpy()) and np.array_equal(rh, r0.cpu().numpy())
    uh = u0.copy()
    s.step(uh, None, dt, 3)
    assert np.array_equal(uh, ref.cpu().numpy())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_energy_is_step_then_energy(precision):
    import torch
    s, u0 = _elastic(precision)
    dt = s.dt_cfl()
    ref = torch.from_numpy(u0).cuda()
    s.step(ref, None, dt, 2)
    e_ref = s.energy(ref)
    u = torch.from_numpy(u0).cuda()
    e = s.step_energy(u, None, dt, 2)
    assert torch.equal(u, ref)
    assert abs(e - e_ref) <= 1e-13 * e_ref
    uh = u0.copy()
    eh = s.step_energy(uh, None, dt, 2)
    assert np.array_equal(uh, ref.cpu().numpy()) and eh == e
    from paper_1711_01175_gb300 import capi
    assert capi.dgw_step_energy(s._ctx, u.data_ptr(), None, 0.0, dt, 0, None)[0] == -1


def test_step_energy_of_a_generic_system():
    import torch
    from paper_1711_01175_gb300 import Solver, reference_nodes
    mesh = wl.structured_hex_mesh((4, 4, 1), (False, False, True),
                                  {0: wl.BC_WALL, 1: wl.BC_WALL, 2: wl.BC_WALL, 3: wl.BC_WALL})
    x = wl.warped_node_coords(mesh, reference_nodes(3)[0], 0.0)
    s = Solver(3, system="shallow_water")
    s.upload_mesh(x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc)
    u0 = wl.shallow_water_standing_wave(x)
    dt = s.dt_cfl()
    ref = torch.from_numpy(u0).cuda()
    s.step(ref, None, dt, 4)
    u = torch.from_numpy(u0).cuda()
    e = s.step_energy(u, None, dt, 4)
    assert torch.equal(u, ref)
    e_ref = s.energy(ref)
    assert abs(e - e_ref) <= 1e-13 * e_ref
