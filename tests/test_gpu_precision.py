"""Precision form: the mixed paths against the FP64 path at T = 1.

Workload: the precision recipe (N=7, warp 0.1, smooth random medium seed 2,
Gaussian stress pulse, z=0 absorbing, z=1 free surface) on 8^3- and
16^3-element cuts.  The CPU oracle cannot reach T = 1 (thousands of steps), so
the reference is the GPU FP64 path, which the parity tests check against the
oracle stage by stage at 1e-12.  Reported: relative L2 error of the mixed
state at T = 1 and the energy drift |E_mixed(T) - E_fp64(T)| / E(0), for the
CUDA-core FP32 volume form ("mixed") and the tensor-core FP16 hi/lo form
("mixed_tc").
"""
import math

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

# Bounds stated after measurement (see the design notes): FP32 volume/flux
# arithmetic accumulated over 5,729 (8^3) and 11,522 (16^3) LSRK steps.
# Measured rel L2 at T = 1: mixed 2.7e-7 (8^3) and 1.7e-6 (16^3); mixed_tc
# 1.1e-6 and 2.5e-7.  Energy drift: mixed 2.2e-8 and 3.5e-8; mixed_tc 4.0e-8
# and 1.3e-9.
MIXED_T1_REL_L2 = 5e-6
MIXED_T1_ENERGY_DRIFT = 1e-7


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("E", [8, 16])
def test_mixed_vs_fp64_to_T1_precision_recipe(E):
    import torch
    from paper_1711_01175_gb300 import Solver, reference_nodes
    cfg = wl.precision_config(E=E)
    r, _ = reference_nodes(cfg.N)
    data = cfg.build(r)
    m = data["mesh"]
    solvers = {}
    for prec in ("fp64", "mixed", "mixed_tc"):
        s = Solver(cfg.N, tau=1, precision=prec, cfl=cfg.cfl)
        s.upload_mesh(data["x"], m.etoe, m.etof, m.orient, m.bc)
        s.upload_material(data["rho"], data["lam"], data["mu"])
        solvers[prec] = s
    dt0 = solvers["fp64"].dt_cfl()
    nsteps = math.ceil(1.0 / dt0)
    dt = 1.0 / nsteps
    states, energies = {}, {}
    for prec, s in solvers.items():
        u = torch.from_numpy(data["u0"]).cuda()
        res = torch.zeros_like(u)
        e0 = s.energy(u)
        s.step(u, res, dt, nsteps)
        energies[prec] = (e0, s.energy(u))
        states[prec] = u.cpu().numpy()
        s.close()
    ref = states["fp64"]
    e0 = energies["fp64"][0]
    assert energies["fp64"][1] < e0                      # upwind + absorbing: dissipative
    for prec in ("mixed", "mixed_tc"):
        err = float(np.linalg.norm(states[prec] - ref) / np.linalg.norm(ref))
        drift = abs(energies[prec][1] - energies["fp64"][1]) / e0
        print(f"precision recipe {E}^3 N=7: {nsteps} steps to T=1, {prec} rel L2 {err:.3e}, "
              f"energy drift {drift:.3e}, E(T)/E(0) fp64 {energies['fp64'][1] / e0:.6f}")
        assert err < MIXED_T1_REL_L2
        assert drift < MIXED_T1_ENERGY_DRIFT
