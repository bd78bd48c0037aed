"""The parity check itself, on the CPU: an error planted in one element of an
oracle right-hand side (made here, on the host) is caught by the per-element
bound of ``assert_parity`` at the tolerances the GPU parity tests use, where a
global relative L2 norm alone lets it through."""
import numpy as np
import pytest

import oracle
import workloads as wl
from harness import FP64_TOL, MIXED_RHS_TOL, assert_parity, elem_max_rel, rel_l2


@pytest.fixture(scope="module")
def rhs():
    N = 3
    mesh = wl.structured_hex_mesh(4, order="morton")
    r, _ = oracle.gll(N)
    x = wl.warped_node_coords(mesh, r, 0.05)
    rho, lam, mu = wl.smooth_random_material(mesh, 1)
    op = oracle.ElasticDG(N, x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc, rho, lam, mu, 1)
    return op.rhs(wl.random_state(mesh.nel, (N + 1) ** 3, 3))


def test_rounding_level_noise_passes(rhs):
    rng = np.random.default_rng(0)
    got = rhs * (1.0 + 1e-15 * rng.standard_normal(rhs.shape))
    assert_parity(got, rhs, FP64_TOL)


def test_one_node_off_by_1e9_fails_the_fp64_bound(rhs):
    got = rhs.copy()
    got[4, 17, 9] += 1e-9 * np.abs(rhs).max()
    assert elem_max_rel(got, rhs) > FP64_TOL
    with pytest.raises(AssertionError):
        assert_parity(got, rhs, FP64_TOL)


def test_one_node_off_by_2e6_fails_the_mixed_bound(rhs):
    got = rhs.copy()
    got[7, 40, 21] += 2e-6 * np.abs(rhs).max()
    assert rel_l2(got, rhs) < MIXED_RHS_TOL             # diluted over 36,864 values
    with pytest.raises(AssertionError):
        assert_parity(got, rhs, MIXED_RHS_TOL)
