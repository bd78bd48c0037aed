"""Plain FP64 CPU oracle for the iHDG-II iteration (the paper's Section 3 and
Algorithm "The iHDG-II approach") on the upwind DG/HDG transport operator.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU-baseline / reference leg) may import or run this module.

The problem is  sigma u - L(u) = b  with L the semi-discrete operator of
``FriedrichsDG`` (upwind flux, trace eliminated) and b given; for transport:
* sigma = 0, b = f: the steady transport equation (Section 4.1,
  eq. transport) with forcing f;
* sigma = 1/dt, b = u^m / dt + f: one implicit Euler step of the
  time-dependent transport equation (Section 4.2; eq. implicitHDG, Section 4.3), of which
  iHDG-II is the locally implicit solver (Section 4.3);
and for the shallow-water system sigma = 2/dt, b = sigma u^m + L(u^m): one
Crank-Nicolson step, the time scheme of the paper's shallow-water test
(Section 6.2).

iHDG-II, iteration k -> k+1 (eqs. iHDGlocal and iHDGtrace): every element K
solves its local problem with its own unknowns at k+1 and its neighbours'
at k inside the weighted trace.  The operator is linear, so
L(u)_K = L_K^self u_K + L_K^nbr(u) with L_K^self the map u_K -> L(u)_K when
every other element is zero, and the local solve reads
    (sigma I - L_K^self) u_K^{k+1} = b_K + L_K^nbr(u^k).
Stopping: eq. tolerancecriteria when the exact solution is given, else
eq. tolerancecriteriarelerror, with the L2 norm of the mass matrix.
"""
from __future__ import annotations

import numpy as np


def element_coloring(etoe):
    """Greedy colouring of the element graph: elements sharing a face differ in colour."""
    nel = etoe.shape[0]
    color = -np.ones(nel, dtype=np.int64)
    for e in range(nel):
        used = {int(color[n]) for n in etoe[e] if n >= 0 and color[n] >= 0}
        c = 0
        while c in used:
            c += 1
        color[e] = c
    return color


class IHDG:
    """iHDG-II for a FriedrichsDG operator with m fields; sigma >= 0.

    L_K^self is the operator with the interior neighbour states zero (boundary
    states keep their dependence on the element's own values), assembled
    column by column: the unit vector of (field q, node j) in every element at
    once."""

    def __init__(self, op, sigma):
        self.op = op
        self.sigma = float(sigma)
        self.m, self.nel, self.Np = op.m, op.nel, op.Np
        _, J = op.geometry(np.arange(op.nel))
        self.wJ = op.w_vol[None, :] * J                      # [nel, Np] mass weights
        n = self.m * self.Np
        self.Lself = np.zeros((self.nel, n, n))             # rows/columns (field, node), field-major
        op.self_only = True
        try:
            for q in range(self.m):
                for j in range(self.Np):
                    u = np.zeros((self.m, self.nel, self.Np))
                    u[q, :, j] = 1.0
                    self.Lself[:, :, q * self.Np + j] = np.moveaxis(op.rhs(u, source=False), 0, 1).reshape(self.nel, n)
        finally:
            op.self_only = False
        self.local = self.sigma * np.eye(n)[None] - self.Lself      # sigma I - L_K^self

    def _flat(self, u):
        return np.moveaxis(u, 0, 1).reshape(self.nel, -1)            # [nel, m Np]

    def _unflat(self, v):
        return np.moveaxis(v.reshape(self.nel, self.m, self.Np), 1, 0)

    def neighbour_term(self, u):
        """L_K^nbr(u) = L(u)_K - L_K^self u_K for every element: [m, nel, Np]."""
        return self.op.rhs(u, source=False) - self._unflat(np.einsum("eij,ej->ei", self.Lself, self._flat(u)))

    def iterate(self, b, u):
        """One iHDG-II iteration from u^k: the local solves of every element."""
        rhs = self._flat(b + self.neighbour_term(u))
        return self._unflat(np.linalg.solve(self.local, rhs[..., None])[..., 0])

    def norm(self, d):
        return float(np.sqrt(np.sum(self.wJ[None] * d * d)))

    def solve(self, b, u0, tol=1e-10, max_iter=1000, exact=None):
        """Iterate to the paper's stopping criterion; returns (u, iterations, history of
        ||u^k - u^{k-1}||)."""
        u = np.array(u0, dtype=np.float64)
        hist = []
        prev_err = None if exact is None else self.norm(u - exact)
        for k in range(1, max_iter + 1):
            un = self.iterate(b, u)
            hist.append(self.norm(un - u))
            u = un
            if exact is not None:
                err = self.norm(u - exact)
                if abs(err - prev_err) < tol:
                    return u, k, hist
                prev_err = err
            elif hist[-1] < tol:
                return u, k, hist
        return u, max_iter, hist

    def direct(self, b):
        """The fixed point by a direct solve of sigma u - L(u) = b (assembled by columns)."""
        n = self.m * self.nel * self.Np
        A = np.zeros((n, n))
        for j in range(n):
            e = np.zeros(n)
            e[j] = 1.0
            A[:, j] = self.sigma * e - self.op.rhs(e.reshape(self.m, self.nel, self.Np), source=False).ravel()
        return np.linalg.solve(A, b.ravel()).reshape(b.shape)


class IHDGTransport(IHDG):
    """iHDG-II for the scalar transport operator."""

    def __init__(self, op, sigma):
        if op.m != 1:
            raise ValueError("IHDGTransport: scalar transport only")
        super().__init__(op, sigma)
