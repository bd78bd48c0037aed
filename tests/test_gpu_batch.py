"""Batched solves (the serving path) against the same solves run alone.

Each solve in a batch must end where the single-solve path (dgw_step) ends,
and the batch may change composition between step pairs.  The arithmetic per
element is the same; the source amplitude comes from a device-side time in the
batch, so results agree to rounding, not bit for bit: 1e-13 relative L2 for
FP64, 1e-6 for the mixed path (where the amplitude differs in its last bit,
the FP32 rounding of the point force can flip).
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as wl
from harness import assert_parity, rel_l2

pytestmark = pytest.mark.gpu

BATCH_TOL = {"fp64": 1e-13, "mixed": 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def make_solve(E, N, seed, precision="fp64", source=True):
    from paper_1711_01175_gb300 import Solver, reference_nodes
    r, _ = reference_nodes(N)
    mesh = wl.structured_hex_mesh(E, (True, True, False), {4: wl.BC_ABSORBING, 5: wl.BC_FREE_SURFACE}, "morton")
    x = wl.warped_node_coords(mesh, r, 0.1)
    rho, lam, mu = wl.smooth_random_material(mesh, seed)
    s = Solver(N, precision=precision)
    s.upload_mesh(x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc)
    s.upload_material(rho, lam, mu)
    src = None
    if source:
        src = dict(element=mesh.nel // 2, xi=[0.2, -0.3, 0.4], force=[0.0, 0.0, 1.0], f0=8.0, t0=0.05)
        s.set_point_force(**src)
    u0 = 1e-2 * wl.random_state(mesh.nel, (N + 1) ** 3, seed)
    return dict(solver=s, mesh=mesh, x=x, mat=(rho, lam, mu), src=src, u0=u0, dt=s.dt_cfl(), N=N)


class Batch:
    def __init__(self, N, precision="fp64"):
        from paper_1711_01175_gb300 import capi
        self.capi = capi
        st, self.h = capi.dgw_batch_create(0, N, 0 if precision == "fp64" else 1, 1, 64)
        assert st == 0, capi.dgw_last_error(None)

    def set(self, items, t0s, stream):
        n = len(items)
        P = ctypes.c_void_p * max(n, 1)
        D = ctypes.c_double * max(n, 1)
        ctxs = P(*[it["solver"]._ctx.value for it in items])
        u = P(*[it["u"].data_ptr() for it in items])
        res = P(*[it["res"].data_ptr() for it in items])
        st = self.capi.dgw_batch_set(self.h, n, ctxs, u, res, D(*[it["dt"] for it in items]), D(*t0s), stream)
        assert st == 0, self.capi.dgw_batch_last_error(self.h)

    def run(self, npairs, stream):
        assert self.capi.dgw_batch_run(self.h, npairs, stream) == 0, self.capi.dgw_batch_last_error(self.h)

    def close(self):
        self.capi.dgw_batch_destroy(self.h)


def alone(item, nsteps, t0=0.0):
    import torch
    u = torch.from_numpy(item["u0"]).cuda()
    res = torch.zeros_like(u)
    item["solver"].step(u, res, item["dt"], nsteps, t0=t0)
    return u.cpu().numpy()


@pytest.mark.parametrize("precision,N", [("fp64", 4), ("mixed", 4), ("mixed", 5)])
def test_batch_matches_single_solves_with_composition_change(precision, N):
    """N = 5 reaches the FP32 stage's L1-prefetch form (N = 3, 5, 6, 7), N = 4 the
    form without it."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    items = [make_solve(2, N, 1, precision), make_solve(3, N, 2, precision), make_solve(2, N, 3, precision, False)]
    late = make_solve(3, N, 4, precision)
    for it in items + [late]:
        it["u"] = torch.from_numpy(it["u0"]).cuda()
        it["res"] = torch.zeros_like(it["u"])
    b = Batch(N, precision)
    # pairs 0-1: first three solves; then solve 1 leaves and `late` joins for 2 more pairs
    b.set(items, [0.0, 0.0, 0.0], stream)
    b.run(2, stream)
    torch.cuda.synchronize()
    left = items[1]
    got_left = left["u"].cpu().numpy()
    cont = [items[0], items[2], late]
    b.set(cont, [4 * items[0]["dt"], 4 * items[2]["dt"], 0.0], stream)       # no new graph: uploads only
    b.run(2, stream)
    torch.cuda.synchronize()
    tol = BATCH_TOL[precision]
    assert_parity(got_left, alone(left, 4), tol)
    assert_parity(items[0]["u"].cpu().numpy(), alone(items[0], 8), tol)
    assert_parity(items[2]["u"].cpu().numpy(), alone(items[2], 8), tol)
    assert_parity(late["u"].cpu().numpy(), alone(late, 4), tol)
    b.close()


def test_batched_solve_matches_oracle():
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    it = make_solve(2, 3, 5)
    it["u"] = torch.from_numpy(it["u0"]).cuda()
    it["res"] = torch.zeros_like(it["u"])
    b = Batch(3)
    b.set([it], [0.0], stream)
    b.run(1, stream)
    torch.cuda.synchronize()
    m = it["mesh"]
    r, _ = oracle.gll(3)
    xo = wl.warped_node_coords(m, r, 0.1)
    op = oracle.ElasticDG(3, xo, m.etoe, m.etof, m.orient, m.bc, *it["mat"], 1)
    src = it["src"]
    op.set_point_force(src["element"], src["xi"], src["force"], src["f0"], src["t0"])
    uo, ro = it["u0"].copy(), np.zeros_like(it["u0"])
    for k in range(2):
        uo, ro = op.step(uo, ro, it["dt"], t=k * it["dt"])
    assert_parity(it["u"].cpu().numpy(), uo, 1e-12)
    b.close()


def test_batch_rejects_mismatched_solves():
    import torch
    from paper_1711_01175_gb300 import capi
    stream = torch.cuda.current_stream().cuda_stream
    a = make_solve(2, 4, 1)
    c = make_solve(2, 3, 1)
    for it in (a, c):
        it["u"] = torch.from_numpy(it["u0"]).cuda()
        it["res"] = torch.zeros_like(it["u"])
    b = Batch(4)
    P = ctypes.c_void_p * 2
    D = ctypes.c_double * 2
    st = capi.dgw_batch_set(b.h, 2, P(a["solver"]._ctx.value, c["solver"]._ctx.value),
                            P(a["u"].data_ptr(), c["u"].data_ptr()), P(a["res"].data_ptr(), c["res"].data_ptr()),
                            D(a["dt"], c["dt"]), D(0.0, 0.0), stream)
    assert st == -1 and "differs" in capi.dgw_batch_last_error(b.h)
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_full_size_solve_sampled_oracle(precision):
    """The largest solve of the serving recipe (48^3 elements, N=5, warp 0.1,
    smooth random medium, Ricker point force at the centre element, free surface
    on top, absorbing bottom) advanced by the batched kernel for one step pair
    from a random state, against the oracle on sampled elements (the source
    element, a free-surface and an absorbing element, an interior one), which
    it evaluates exactly through the shrinking dependence regions of the ten
    stages."""
    import torch
    from harness import oracle_sampled_steps
    stream = torch.cuda.current_stream().cuda_stream
    it = make_solve(48, 5, 11, precision)
    it["u"] = torch.from_numpy(it["u0"]).cuda()
    it["res"] = torch.zeros_like(it["u"])
    b = Batch(5, precision)
    b.set([it], [0.0], stream)
    b.run(1, stream)
    torch.cuda.synchronize()
    m = it["mesh"]
    rng = np.random.default_rng(3)
    top = np.nonzero(m.bc[:, 5] == wl.BC_FREE_SURFACE)[0]
    bottom = np.nonzero(m.bc[:, 4] == wl.BC_ABSORBING)[0]
    sample = np.unique([it["src"]["element"], int(rng.choice(top)), int(rng.choice(bottom)), int(rng.integers(m.nel))])
    r, _ = oracle.gll(5)
    xo = wl.warped_node_coords(m, r, 0.1)
    op = oracle.ElasticDG(5, xo, m.etoe, m.etof, m.orient, m.bc, *it["mat"], 1)
    src = it["src"]
    op.set_point_force(src["element"], src["xi"], src["force"], src["f0"], src["t0"])
    uo, _ = oracle_sampled_steps(op, it["u0"], np.zeros_like(it["u0"]), it["dt"], 2, sample)
    got = it["u"].cpu().numpy()[:, sample]
    # the step pair changes u by O(dt |L u|): compare the increments
    du_o = uo - it["u0"][:, sample]
    assert_parity(got - it["u0"][:, sample], du_o, 1e-12 if precision == "fp64" else 1e-6,
                  label=f"48^3 N=5 batched {precision} sampled")
    b.close()
