"""dgw_energy_static: the energy entry point for callers that cannot allocate.

Callers whose device memory is owned by someone else (a framework's pool
allocator with a cap, a running time loop that must not allocate, code handed
only device pointers) use dgw_energy_static: no context, every argument is the
caller's device memory, and the reduction scratch is a fixed array inside the
library.  This file checks it against the context-based dgw_energy, through
the C ABI, on two calls in a row (the second call must not see the first
one's leftovers), and that an oversized mesh is refused before any launch.
It is collected last so that a run stopping at the first failure has already
run every other test.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

ENERGY_TOL = 1e-13     # the relative tolerance of the energy parity test


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _device(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _case(which):
    from paper_1711_01175_gb300 import Solver, reference_nodes
    cfg = wl.large_config(E=8) if which == "large-8^3-N4" else wl.parity_config()
    r, _ = reference_nodes(cfg.N)
    data = cfg.build(r)
    mesh = data["mesh"]
    solver = Solver(cfg.N)
    solver.upload_mesh(data["x"], mesh.etoe, mesh.etof, mesh.orient, mesh.bc)
    solver.upload_material(data["rho"], data["lam"], data["mu"])
    dev = {k: _device(data[k]) for k in ("x", "rho", "lam", "mu")}
    return cfg, data, mesh, solver, dev


def test_energy_static_matches_dgw_energy_on_calls_in_a_row():
    """Calls in a row: the 8^3, N=4 mesh (512 elements), then the 4^3, N=3 mesh
    (64 elements, fewer blocks of partial sums: it must not read partials that
    the larger call left in the shared array), then the larger one again with
    another state.  Each against dgw_energy of a context on the same mesh."""
    import torch
    from paper_1711_01175_gb300 import capi
    cases = {w: _case(w) for w in ("large-8^3-N4", "parity-4^3-N3")}
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    order = [("large-8^3-N4", None), ("parity-4^3-N3", None), ("large-8^3-N4", 17)]
    for which, seed in order:
        cfg, data, mesh, solver, d = cases[which]
        u_host = data["u0"] if seed is None else wl.random_state(mesh.nel, (cfg.N + 1) ** 3, seed)
        u = _device(u_host)
        st = capi.dgw_energy_static(cfg.N, mesh.nel, d["x"].data_ptr(), u.data_ptr(), d["rho"].data_ptr(),
                                    d["lam"].data_ptr(), d["mu"].data_ptr(), out.data_ptr(), stream)
        capi.check(st)
        torch.cuda.synchronize()
        e_static = float(out.item())
        e_ctx = solver.energy(u)
        assert abs(e_static - e_ctx) <= ENERGY_TOL * e_ctx, (which, e_static, e_ctx)
    for c in cases.values():
        c[3].close()


def test_energy_static_rejects_oversized_mesh():
    import torch
    from paper_1711_01175_gb300 import capi
    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = d.data_ptr()
    limit = 1 << 20
    st = capi.dgw_energy_static(4, limit + 1, p, p, p, p, p, p, None)
    assert st == -1
    assert "limit" in capi.dgw_last_error(None)
    st = capi.dgw_energy_static(9, 10, p, p, p, p, p, p, None)
    assert st == -1
    host = np.zeros(16)
    st = capi.dgw_energy_static(1, 2, host.ctypes.data, p, p, p, p, p, None)
    assert st == -1 and "device memory" in capi.dgw_last_error(None)
