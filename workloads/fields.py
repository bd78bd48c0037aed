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


# ---- Generic Friedrichs-system instances (u[m][nel][Np]) ----------------------

def transport_periodic(x, beta, t=0.0):
    """Exact solution u = g(x - beta t) of u_t + beta . grad u = 0 with the
    periodic profile g(y) = sin(2 pi y1) sin(2 pi y2) sin(2 pi y3) (period 1 on
    the unit cube): the periodic stand-in for the paper's translating Gaussian
    of the time-dependent 3-D transport test (Section 6.1).  Shape [1, nel, Np]."""
    x = np.asarray(x, dtype=np.float64)
    y = x - np.asarray(beta, dtype=np.float64) * t
    return np.prod(np.sin(2.0 * np.pi * y), axis=-1)[None]


def transport_gaussian(x, t=0.0, shift=0.35):
    """The paper's translating Gaussian exp(-5 |x - shift t (1,1,1)|^2) (Section 6.1
    prints the shift 0.35 t with beta = (0.2, 0.2, 0.2)).  Shape [1, nel, Np]."""
    x = np.asarray(x, dtype=np.float64)
    return np.exp(-5.0 * np.sum((x - shift * t) ** 2, axis=-1))[None]


def shallow_water_standing_wave(x, t=0.0):
    """The linear standing wave of the paper's shallow-water test (Section 6.2,
    Phi = 1, f = gamma = 0, no wind stress) on [0,1]^2 with walls:
    phi = cos(pi x) cos(pi y) cos(sqrt2 pi t),
    u = sin(pi x) cos(pi y) sin(sqrt2 pi t) / sqrt2,
    v = cos(pi x) sin(pi y) sin(sqrt2 pi t) / sqrt2.
    Returns (phi, Phi u, Phi v), shape [3, nel, Np]; independent of z."""
    x = np.asarray(x, dtype=np.float64)
    X, Y = np.pi * x[..., 0], np.pi * x[..., 1]
    w = np.sqrt(2.0) * np.pi * t
    out = np.empty((3,) + X.shape)
    out[0] = np.cos(X) * np.cos(Y) * np.cos(w)
    out[1] = np.sin(X) * np.cos(Y) * np.sin(w) / np.sqrt(2.0)
    out[2] = np.cos(X) * np.sin(Y) * np.sin(w) / np.sqrt(2.0)
    return out


def random_fields(m: int, nel: int, Np: int, seed: int):
    """Standard-normal m-component state."""
    return np.random.default_rng(seed).standard_normal((m, nel, Np))
