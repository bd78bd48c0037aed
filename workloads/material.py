"""Seeded per-element isotropic elastic material (rho, lambda, mu).

The heterogeneous medium is a smooth random field sampled at the undeformed
element centres: each of P-wave speed and density is a sum of eight Fourier
modes with integer wave vectors 0 < |k| <= 3, affinely rescaled to the
requested range.  The shear speed is cp / sqrt(3) with a uniform +-10 %
per-element perturbation.  Lame parameters follow from
mu = rho cs^2 and lambda = rho (cp^2 - 2 cs^2), which stay positive because
cs^2 <= 1.21 cp^2 / 3 < cp^2 / 2.
"""
from __future__ import annotations

import numpy as np

from .mesh import Mesh, cell_centroids


def _integer_wavevectors(rng, n_modes, kmax):
    out = []
    while len(out) < n_modes:
        k = rng.integers(-kmax, kmax + 1, size=3)
        n2 = int(k @ k)
        if 0 < n2 <= kmax * kmax:
            out.append(k)
    return np.array(out, dtype=np.float64)


def _unit_field(rng, centres, n_modes, kmax):
    k = _integer_wavevectors(rng, n_modes, kmax)
    amp = rng.uniform(0.5, 1.0, size=n_modes)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    f = np.cos(2.0 * np.pi * centres @ k.T + phase) @ amp
    lo, hi = f.min(), f.max()
    if hi - lo <= 1e-300:
        return np.full_like(f, 0.5)
    return (f - lo) / (hi - lo)


def smooth_random_material(mesh: Mesh, seed: int, cp_range=(2.0, 6.0), rho_range=(1.0, 3.0),
                           cs_noise=0.1, n_modes=8, kmax=3):
    """Return (rho, lam, mu), each float64 [nel]."""
    rng = np.random.default_rng(seed)
    c = cell_centroids(mesh)
    cp = cp_range[0] + (cp_range[1] - cp_range[0]) * _unit_field(rng, c, n_modes, kmax)
    rho = rho_range[0] + (rho_range[1] - rho_range[0]) * _unit_field(rng, c, n_modes, kmax)
    noise = rng.uniform(-1.0, 1.0, size=mesh.nel)
    cs = cp / np.sqrt(3.0) * (1.0 + cs_noise * noise)
    mu = rho * cs * cs
    lam = rho * (cp * cp - 2.0 * cs * cs)
    return rho, lam, mu


def homogeneous_material(nel: int, rho=1.0, lam=2.0, mu=1.0):
    return (np.full(nel, float(rho)), np.full(nel, float(lam)), np.full(nel, float(mu)))
