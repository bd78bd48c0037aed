"""Plain FP64 CPU oracle for the upwind DG operator of generic Friedrichs systems.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU-baseline / reference leg) may import or run this module.
It shares no code with the CUDA library and imports nothing from it.

The model problem is the paper's Section 2 system (eq. LPDE) with a time
derivative, du/dt + sum_k d_k(A_k u) = 0, m components, constant symmetric
A_k, Q = I and C = 0.  Two instances from the paper's numerical sections:

* transport: m = 1, A_k = beta_k (the time-dependent 3-D transport of
  Section 6.1);
* linearized shallow water: m = 3, u = (phi, Phi u, Phi v), A_1 and A_2 of
  eq. linearizedShallow with Phi = 1, no Coriolis force, friction or wind
  stress (the setting of the standing-wave test, Section 6.2); the 2-D
  problem is posed on a mesh one element thick in z with periodic z faces,
  and A_3 = 0.

The discretisation is the one of the elastic oracle (``dg_elastic``): GLL
collocation, split-form volume term with curl-form metrics, the HDG flux of
eq. RiemannFluxBoth with the trace eliminated through eq. iHDGtrace, diagonal
lift, LSRK(5,4).  The stabilisation |A(n)| is taken literally from an
eigen-decomposition of the symmetric A(n) (eq. RiemannFluxBoth).  Boundary
states: tag 1 is the shallow-water wall (normal momentum reflected), tag 2 a
zero exterior state.

Layouts: ``u[m][nel][Np]`` with node index ``i + n*(j + n*k)``, r fastest.
"""
from __future__ import annotations

import numpy as np

from .dg_elastic import ElasticDG, LSRK_A, LSRK_B, LSRK_C, hdg_flux, weighted_trace


class FriedrichsSystem:
    """m, the constant symmetric A_k (3 x m x m) and the boundary states."""

    def __init__(self, name, A_stack, wave_speed):
        self.name = name
        self.A_stack = np.asarray(A_stack, dtype=np.float64)
        self.m = self.A_stack.shape[1]
        self.wave_speed = float(wave_speed)
        for k in range(3):
            if not np.allclose(self.A_stack[k], self.A_stack[k].T):
                raise ValueError("A_k must be symmetric")

    def A_of(self, n):
        """A(n) = sum_k n_k A_k, vectorised over the leading axes of n."""
        return np.einsum("...k,kij->...ij", np.asarray(n, dtype=np.float64), self.A_stack)

    def abs_A(self, n):
        """|A(n)| = R |S| R^T from the eigen-decomposition of the symmetric A(n)."""
        S, R = np.linalg.eigh(self.A_of(n))
        return np.einsum("...ij,...j,...kj->...ik", R, np.abs(S), R)

    def ghost(self, um, nrm, tag):
        """Exterior state on a boundary face: um [..., m], unit normal nrm [..., 3]."""
        if tag == 2:
            return np.zeros_like(um)
        if tag == 1 and self.name == "shallow_water":
            # wall: phi unchanged, the momentum's component along the horizontal
            # normal reflected
            up = um.copy()
            nxy = nrm[..., :2]
            nn = np.sum(nxy * nxy, axis=-1)
            qn = np.sum(um[..., 1:3] * nxy, axis=-1) / np.where(nn > 0, nn, 1.0)
            up[..., 1:3] = um[..., 1:3] - 2.0 * qn[..., None] * nxy
            return up
        raise ValueError(f"boundary tag {tag} is not defined for {self.name}")


def transport(beta):
    beta = np.asarray(beta, dtype=np.float64)
    return FriedrichsSystem("transport", beta.reshape(3, 1, 1), np.linalg.norm(beta))


def shallow_water():
    A1 = np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    A2 = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    return FriedrichsSystem("shallow_water", np.stack([A1, A2, np.zeros((3, 3))]), 1.0)


class FriedrichsDG(ElasticDG):
    """du/dt = L(u) for a FriedrichsSystem on one mesh (Q = I).

    Mesh handling, reference derivatives and curl-form metrics are those of
    ElasticDG; the physics (A_k, stabilisation, boundary states, energy) is
    the system's."""

    def __init__(self, N, x, etoe, etof, orient, bc, system, tau=1):
        nel = np.asarray(x).shape[0]
        one = np.ones(nel)
        super().__init__(N, x, etoe, etof, orient, bc, one, one, one, tau)
        self.system = system
        self.m = system.m
        self.self_only = False      # True: interior neighbour states taken as zero (L_K^self)

    def set_point_force(self, *args, **kwargs):
        raise NotImplementedError("point forces are defined for the elastic system only")

    def exterior_state(self, u, elems, f, nrm=None):
        """(u^-, u^+) at the face nodes of face f: [m, ne, nf] each."""
        fn = self.face_nodes[f]
        um = u[:, elems][:, :, fn]
        nbr = self._neighbour_map(f, elems)
        tag = self.bc[elems, f]
        interior = (self.etoe[elems, f] >= 0) & (tag == 0)
        if np.any(~interior & (tag == 0)):
            raise ValueError(f"face {f}: element without neighbour and without boundary tag")
        flat = u.reshape(self.m, -1)
        up = np.zeros_like(um)
        if not self.self_only:
            up[:, interior] = flat[:, nbr[interior]]
        for t in (1, 2):
            sel = tag == t
            if np.any(sel):
                g = self.system.ghost(np.moveaxis(um[:, sel], 0, -1), nrm[sel], t)
                up[:, sel] = np.moveaxis(g, -1, 0)
        return um, up

    def volume_term(self, u_e, Ja, J, sign=1.0):
        """-1/2 [ 1/J sum_i d_i(sum_k Ja^i_k A_k u) + 1/J sum_i sum_k Ja^i_k A_k d_i u ]."""
        Ak = [sign * self.system.A_stack[k] for k in range(3)]
        Au = [np.einsum("pq,qen->pen", Ak[k], u_e) for k in range(3)]
        cons = np.zeros_like(u_e)
        noncons = np.zeros_like(u_e)
        for i in range(3):
            Ftilde = sum(Ja[i][k][None] * Au[k] for k in range(3))
            cons += self.dref(Ftilde, i)
            du = self.dref(u_e, i)
            noncons += sum(Ja[i][k][None] * np.einsum("pq,qen->pen", Ak[k], du) for k in range(3))
        return -0.5 * (cons + noncons) / J[None]

    def _face(self, u, elems, Ja, f):
        m = self.outward_scaled_normal(Ja, f)                   # [ne, nf, 3]
        sJ = np.linalg.norm(m, axis=-1)
        nrm = m / sJ[..., None]
        um, up = self.exterior_state(u, elems, f, nrm)
        return sJ, nrm, np.moveaxis(um, 0, -1), np.moveaxis(up, 0, -1)

    def surface_term(self, u, elems, Ja, J, sign=1.0):
        """Sum over faces of (w_f sJ)/(w_vol J) (F(u^-).n - F_hat.n) at the face nodes."""
        out = np.zeros((self.m, len(elems), self.Np))
        for f in range(6):
            fn = self.face_nodes[f]
            sJ, nrm, um, up = self._face(u, elems, Ja, f)
            An = sign * self.system.A_of(nrm)
            stab = self.tau * self.system.abs_A(nrm)
            s_uhat = weighted_trace(An, stab, um, up)
            Fhat = hdg_flux(An, stab, um, s_uhat)
            q = np.einsum("...ij,...j->...i", An, um) - Fhat
            scale = self.w_face[None, :] * sJ / (self.w_vol[fn][None, :] * J[:, fn])
            out[:, :, fn] += np.moveaxis(q * scale[..., None], -1, 0)
        return out

    def rhs(self, u, elems=None, t=0.0, sign=1.0, source=True):
        u = np.asarray(u, dtype=np.float64)
        elems = np.arange(self.nel) if elems is None else np.asarray(elems, dtype=np.int64)
        Ja, J = self.geometry(elems)
        if np.any(J <= 0.0):
            raise ValueError("non-positive Jacobian")
        return self.volume_term(u[:, elems], Ja, J, sign) + self.surface_term(u, elems, Ja, J, sign)

    def energy(self, u):
        """E = 1/2 sum_K sum_nodes w J |u|^2."""
        _, J = self.geometry(np.arange(self.nel))
        return 0.5 * float(np.sum(self.w_vol[None, None, :] * J[None] * u * u))

    def energy_rate(self, u):
        """dE/dt = sum w J u . L(u)."""
        _, J = self.geometry(np.arange(self.nel))
        return float(np.sum(self.w_vol[None, None, :] * J[None] * u * self.rhs(u)))

    def energy_rate_from_faces(self, u):
        """The rate from face quantities only (the volume term is skew):
        sum over element-face sides of w_f sJ (-1/2 u^-.A(n)u^+ - 1/2 u^-.Stab(u^- - u^+))."""
        elems = np.arange(self.nel)
        Ja, _ = self.geometry(elems)
        total = 0.0
        for f in range(6):
            sJ, nrm, um, up = self._face(u, elems, Ja, f)
            An = self.system.A_of(nrm)
            stab = self.tau * self.system.abs_A(nrm)
            t = (-0.5 * np.einsum("...i,...ij,...j->...", um, An, up)
                 - 0.5 * np.einsum("...i,...ij,...j->...", um, stab, um - up))
            total += np.sum(self.w_face[None, :] * sJ * t)
        return total

    def c_max(self):
        return self.system.wave_speed


__all__ = ["FriedrichsSystem", "FriedrichsDG", "transport", "shallow_water", "LSRK_A", "LSRK_B", "LSRK_C"]
