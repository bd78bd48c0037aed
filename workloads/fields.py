"""Initial data for the velocity-stress system, in the layout u[9][nel][Np].

Field order: (v1, v2, v3, s11, s22, s33, s23, s13, s12) -- velocity, then the
Voigt stress vector.
"""
from __future__ import annotations

import numpy as np


def plane_p_wave(x, rho, lam, mu, t=0.0, direction=(1, 1, 0)):
    """Exact plane P-wave of the homogeneous isotropic medium.

    With integer direction d, n = d/|d|, xi = n.x - cp t and
    g(xi) = sin(2 pi |d| xi) (periodic on the unit cube):
    v = n g(xi) and sigma = -(lam I + 2 mu n n^T) g(xi) / cp,
    cp = sqrt((lam + 2 mu) / rho).  Material must be homogeneous (scalars).
    """
    x = np.asarray(x, dtype=np.float64)
    d = np.asarray(direction, dtype=np.float64)
    dn = float(np.sqrt(d @ d))
    n = d / dn
    cp = float(np.sqrt((lam + 2.0 * mu) / rho))
    xi = x @ n - cp * t                          # [nel, Np]
    g = np.sin(2.0 * np.pi * dn * xi)
    sig = -(lam * np.eye(3) + 2.0 * mu * np.outer(n, n)) / cp
    u = np.empty((9,) + xi.shape)
    for i in range(3):
        u[i] = n[i] * g
    voigt = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    for q, (i, j) in enumerate(voigt):
        u[3 + q] = sig[i, j] * g
    return u


def gaussian_stress_pulse(x, centre=(0.5, 0.5, 0.5), width=0.05):
    """s11 = s22 = s33 = exp(-|x - x0|^2 / w^2), all other fields zero."""
    x = np.asarray(x, dtype=np.float64)
    r2 = np.sum((x - np.asarray(centre)) ** 2, axis=-1)
    u = np.zeros((9,) + r2.shape)
    p = np.exp(-r2 / (width * width))
    u[3] = p
    u[4] = p
    u[5] = p
    return u


def random_state(nel: int, Np: int, seed: int):
    """Standard-normal state, for operator identities and parity on rough data."""
    return np.random.default_rng(seed).standard_normal((9, nel, Np))
