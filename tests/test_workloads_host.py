"""The seeded synthetic inputs follow their stated recipes (CPU only).

* serving stream (the full recipe: 2000 requests, E log-uniform in [8, 48],
  N in {3, 4, 5}, 200-2000 steps, Poisson arrivals): ranges, the log-uniform
  median, even step counts, arrival gaps of mean 1/rate, unit forces, seeded
  reproducibility;
* smooth random medium: cp in [2, 6], rho in [1, 3], cs = cp/sqrt(3)(1 +- 0.1),
  lambda > 0 (per-element constants);
* warp x_i + a prod_j sin(2 pi x_j): vanishes on the cube faces, J > 0;
* Gaussian stress pulse: s11 = s22 = s33, the other fields zero;
* the serving loop's device-memory estimate grows with the mesh.
"""
import numpy as np
import pytest

import oracle
import workloads as wl


def test_serving_request_stream_recipe():
    reqs = wl.make_requests(2000, seed=7, rate=80.0)
    E = np.array([r.E for r in reqs])
    N = np.array([r.N for r in reqs])
    steps = np.array([r.steps for r in reqs])
    t = np.array([r.arrival for r in reqs])
    assert E.min() >= 8 and E.max() <= 48
    assert abs(np.median(np.log(E)) - 0.5 * (np.log(8) + np.log(48))) < 0.1     # log-uniform
    assert set(N) == {3, 4, 5} and all(abs(np.mean(N == n) - 1 / 3) < 0.05 for n in (3, 4, 5))
    assert steps.min() >= 200 and steps.max() <= 2000 and np.all(steps % 2 == 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and abs(gaps.mean() * 80.0 - 1.0) < 0.06            # Poisson, rate 80/s
    assert abs(np.std(gaps) / np.mean(gaps) - 1.0) < 0.1                         # exponential gaps
    assert all(abs(np.linalg.norm(r.force) - 1.0) < 1e-12 for r in reqs)
    assert all(max(abs(v) for v in r.xi) <= 0.5 for r in reqs)
    again = wl.make_requests(2000, seed=7, rate=80.0)
    assert [(r.E, r.N, r.steps, r.arrival) for r in again] == [(r.E, r.N, r.steps, r.arrival) for r in reqs]


def test_medium_recipe():
    mesh = wl.structured_hex_mesh(12, (True, True, False))
    rho, lam, mu = wl.smooth_random_material(mesh, 1)
    cs = np.sqrt(mu / rho)
    cp = np.sqrt((lam + 2 * mu) / rho)
    assert rho.shape == (mesh.nel,)
    assert rho.min() >= 1 - 1e-12 and rho.max() <= 3 + 1e-12
    assert cp.min() >= 2 - 1e-9 and cp.max() <= 6 + 1e-9
    ratio = cs * np.sqrt(3) / cp
    assert ratio.min() >= 0.9 - 1e-12 and ratio.max() <= 1.1 + 1e-12
    assert lam.min() > 0
    assert np.ptp(cp) > 2.0                       # the field spans most of the range


def test_warp_recipe():
    N = 4
    mesh = wl.structured_hex_mesh(4, (False, False, False))
    r, _ = oracle.gll(N)
    x0 = wl.warped_node_coords(mesh, r, 0.0)
    x = wl.warped_node_coords(mesh, r, 0.1)
    on_face = np.any((np.abs(x0) < 1e-14) | (np.abs(x0 - 1) < 1e-14), axis=-1)
    assert np.abs(x[on_face] - x0[on_face]).max() < 1e-14
    s = np.prod(np.sin(2 * np.pi * x0), axis=-1)
    assert np.abs(x - (x0 + 0.1 * s[..., None])).max() < 1e-14
    op = oracle.ElasticDG(N, x, mesh.etoe, mesh.etof, mesh.orient, mesh.bc, *wl.homogeneous_material(mesh.nel))
    _, J = op.geometry(np.arange(mesh.nel))
    assert J.min() > 0


def test_gaussian_pulse_recipe():
    mesh = wl.structured_hex_mesh(2)
    x = wl.warped_node_coords(mesh, oracle.gll(3)[0], 0.0)
    u = wl.gaussian_stress_pulse(x)
    assert np.array_equal(u[3], u[4]) and np.array_equal(u[3], u[5])
    assert not np.any(u[[0, 1, 2, 6, 7, 8]])
    d2 = np.sum((x - 0.5) ** 2, axis=-1)
    assert np.allclose(u[3], np.exp(-d2 / 0.05 ** 2), rtol=1e-14, atol=0)


def test_serving_memory_estimate():
    serving = pytest.importorskip("paper_1711_01175_gb300.serving")
    for prec in ("mixed", "fp64"):
        b = [serving.bytes_per_request(E, 4, prec) for E in (8, 16, 32)]
        assert b[0] < b[1] < b[2]
        nel, Np = 16 ** 3, 125
        assert serving.bytes_per_request(16, 4, prec) >= nel * Np * 9 * 8 * 3      # three FP64 states
    assert serving.bytes_per_request(16, 4, "mixed") < serving.bytes_per_request(16, 4, "fp64")
