"""Plain FP64 CPU oracle for the upwind DG (eliminated HDG) velocity-stress operator.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU-baseline / reference leg) may import or run this module.
It shares no code with the CUDA library and imports nothing from it.  It is
deliberately slow and follows the method step by step:

* The model problem is the linear Friedrichs system of the paper's Section 2
  (eq. LPDE), sum_k d_k(A_k u) + C u = f, here written with a time derivative
  Q du/dt and m = 9 components (velocity, Voigt stress): A_k constant and
  symmetric, the medium only in Q, C = 0, f = 0.
* Upwind HDG stabilisation |A| = R|S|R^{-1} (Section 2, eq. RiemannFluxBoth)
  is taken literally from an eigen-decomposition of the flux matrix of the
  system written as du/dt + sum_k d_k(Q^{-1} A_k u) = 0, i.e. Q^{-1} A(n),
  and multiplied back by Q for the Q-weighted equation; where the medium
  jumps across a face (outside Section 2's continuity assumption) the two
  sides' (rho, lambda, mu) are averaged.
* The weighted trace |A| u_hat is computed from the face conservation
  condition (Section 2, eq. HDGeqn) in the form of Section 3, eq. iHDGtrace,
  with both sides at the same time level, and the HDG flux
  F_hat.n = A(n)u + |A|(u - u_hat) follows (eq. RiemannFluxBoth).
* The element-by-element explicit scheme of Section 4.3 ("iHDG as a locally
  implicit method": explicit HDG with forward Euler) is advanced here with a
  five-stage low-storage Runge-Kutta method instead of forward Euler.

Readings where the paper is silent (each one is also listed in the design
notes): GLL collocation with N+1 points per axis; strong form with the
split (skew-symmetric) volume term; curl-form metric terms; face-averaged
medium in the stabilisation; free-surface mirror state and zero absorbing
state; Carpenter-Kennedy (1994) LSRK(5,4) coefficients; CFL convention
dt = CFL h / (c_max N^2), which reproduces the CFL column of the paper's
weak-scaling table for time-dependent transport (Section 6.1).

Layouts: ``u[9][nel][Np]`` with node index ``i + n*(j + n*k)``, n = N+1,
r (i) fastest.  Field order (v1, v2, v3, s11, s22, s33, s23, s13, s12).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

NFIELD = 9
VOIGT = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


# --------------------------------------------------------------------------
# Reference element: Gauss-Lobatto-Legendre nodes, weights, derivative matrix
# (no paper source; the quadrature reading of the design notes)
# --------------------------------------------------------------------------
def legendre(N: int, x):
    """P_N(x) and P_N'(x) by the three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0, p1 = np.ones_like(x), x.copy()
    if N == 0:
        return p0, np.zeros_like(x)
    d0, d1 = np.zeros_like(x), np.ones_like(x)
    for k in range(1, N):
        p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
        d2 = d0 + (2 * k + 1) * p1
        p0, p1, d0, d1 = p1, p2, d1, d2
    return p1, d1


def gll(N: int):
    """GLL nodes (ascending) and weights: the end points and the roots of P_N'."""
    if N < 1:
        raise ValueError("N >= 1")
    x = -np.cos(np.pi * np.arange(N + 1) / N)            # Chebyshev-Lobatto start
    for _ in range(100):
        # Newton on q(x) = (1 - x^2) P_N'(x); q'(x) = -N(N+1) P_N(x)
        P, dP = legendre(N, x)
        q = (1.0 - x * x) * dP
        dq = -N * (N + 1) * P
        step = np.zeros_like(x)
        inner = slice(1, N)
        step[inner] = q[inner] / dq[inner]
        x = x - step
        if np.max(np.abs(step)) < 1e-16:
            break
    x[0], x[-1] = -1.0, 1.0
    P, _ = legendre(N, x)
    w = 2.0 / (N * (N + 1) * P * P)
    return x, w


def lagrange_derivative_matrix(r):
    """D[i, j] = l_j'(r_i) for the Lagrange basis on nodes r (barycentric form)."""
    r = np.asarray(r, dtype=np.float64)
    n = r.size
    lam = np.array([1.0 / np.prod([r[j] - r[k] for k in range(n) if k != j]) for j in range(n)])
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (lam[j] / lam[i]) / (r[i] - r[j])
        D[i, i] = sum(1.0 / (r[i] - r[k]) for k in range(n) if k != i)
    return D


# --------------------------------------------------------------------------
# The Friedrichs system for velocity-stress elasticity (Section 2, eq. LPDE
# with m = 9; the elastic instance is the design reading Q1)
# --------------------------------------------------------------------------
def B_of(n):
    """6x3 map v -> Voigt(sym(n (x) v)) with engineering shear."""
    n1, n2, n3 = n
    return np.array([[n1, 0, 0],
                     [0, n2, 0],
                     [0, 0, n3],
                     [0, n3, n2],
                     [n3, 0, n1],
                     [n2, n1, 0]], dtype=np.float64)


def A_of(n):
    """A(n) = sum_k A_k n_k = -[[0, B(n)^T], [B(n), 0]] (9x9, symmetric)."""
    B = B_of(n)
    A = np.zeros((9, 9))
    A[:3, 3:] = -B.T
    A[3:, :3] = -B
    return A


A_K = [A_of(np.eye(3)[k]) for k in range(3)]
A_STACK = np.stack(A_K)


def stiffness_voigt(lam, mu):
    """Isotropic Voigt stiffness C_V (6x6)."""
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    for i in range(3):
        C[i, i] = lam + 2.0 * mu
        C[3 + i, 3 + i] = mu
    return C


def Q_of(rho, lam, mu):
    """Q = diag(rho I_3, C_V^{-1}): the time-derivative weight (energy matrix)."""
    Q = np.zeros((9, 9))
    Q[:3, :3] = rho * np.eye(3)
    Q[3:, 3:] = np.linalg.inv(stiffness_voigt(lam, mu))
    return Q


def abs_A(n):
    """|A(n)| = R |S| R^{-1} from the eigen-decomposition of the symmetric A(n)
    (Section 2, eq. RiemannFluxBoth).  Vectorised over leading axes of n."""
    n = np.asarray(n, dtype=np.float64)
    lead = n.shape[:-1]
    A = np.stack([A_of(v) for v in n.reshape(-1, 3)]).reshape(lead + (9, 9))
    S, R = np.linalg.eigh(A)
    return np.einsum("...ij,...j,...kj->...ik", R, np.abs(S), R)


def abs_A_Q(n, rho, lam, mu):
    """Stabilisation for the Q-weighted system: Q |Q^{-1} A(n)| = Q R |S| R^{-1}.

    eq. RiemannFluxBoth applied to the system in the form
    du/dt + sum_k d_k(Q^{-1} A_k u) = 0, whose flux matrix is Q^{-1} A(n) with
    real eigenvalues (+-cp, +-cs twice, 0 three times); the Q-weighted equation
    then carries Q R|S|R^{-1}.  Computed stably: Q^{-1}A = Q^{-1/2} At Q^{1/2}
    with At = Q^{-1/2} A Q^{-1/2} symmetric, so R = Q^{-1/2} V for At = V S V^T
    and Q R|S|R^{-1} = Q^{1/2} V |S| V^T Q^{1/2}.  Vectorised over the leading
    axes of n; rho, lam, mu broadcast against them."""
    n = np.asarray(n, dtype=np.float64)
    lead = n.shape[:-1]
    rho, lam, mu = (np.broadcast_to(np.asarray(v, dtype=np.float64), lead).reshape(-1) for v in (rho, lam, mu))
    A = np.einsum("kc,cij->kij", n.reshape(-1, 3), A_STACK)
    Q = np.stack([Q_of(r_, l_, m_) for r_, l_, m_ in zip(rho, lam, mu)])
    w, U = np.linalg.eigh(Q)
    Qh = np.einsum("kij,kj,klj->kil", U, np.sqrt(w), U)
    Qih = np.einsum("kij,kj,klj->kil", U, 1.0 / np.sqrt(w), U)
    At = Qih @ A @ Qih
    S, V = np.linalg.eigh(At)
    out = Qh @ np.einsum("kij,kj,klj->kil", V, np.abs(S), V) @ Qh
    return out.reshape(lead + (9, 9))


def weighted_trace(An, stab, um, up):
    """Stab * u_hat from the conservation condition, eq. iHDGtrace, with both the
    own (-) and neighbour (+) states at the same level and n^+ = -n^-:
    2 Stab u_hat = Stab (u^- + u^+) + A(n^-) u^- + A(n^+) u^+."""
    Apos = -An
    return 0.5 * (np.einsum("...ij,...j->...i", stab, um + up)
                  + np.einsum("...ij,...j->...i", An, um)
                  + np.einsum("...ij,...j->...i", Apos, up))


def hdg_flux(An, stab, um, stab_uhat):
    """F_hat . n = F(u^-).n + Stab (u^- - u_hat)  (eq. RiemannFluxBoth)."""
    return (np.einsum("...ij,...j->...i", An, um)
            + np.einsum("...ij,...j->...i", stab, um) - stab_uhat)


# --------------------------------------------------------------------------
# LSRK(5,4): Carpenter & Kennedy (1994), 2N-storage, five stages, fourth order
# --------------------------------------------------------------------------
LSRK_A = [Fraction(0), Fraction(-567301805773, 1357537059087),
          Fraction(-2404267990393, 2016746695238), Fraction(-3550918686646, 2091501179385),
          Fraction(-1275806237668, 842570457699)]
LSRK_B = [Fraction(1432997174477, 9575080441755), Fraction(5161836677717, 13612068292357),
          Fraction(1720146321549, 2090206949498), Fraction(3134564353537, 4481467310338),
          Fraction(2277821191437, 14882151754819)]
LSRK_C = [Fraction(0), Fraction(1432997174477, 9575080441755),
          Fraction(2526269341429, 6820363962896), Fraction(2006345519317, 3224310063776),
          Fraction(2802321613138, 2924317926251)]


def ricker(t, f0, t0):
    """Ricker wavelet (1 - 2 (pi f0 (t - t0))^2) exp(-(pi f0 (t - t0))^2)."""
    a = (np.pi * f0 * (np.asarray(t, dtype=np.float64) - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def lagrange_values(r, xi):
    """l_j(xi) for the Lagrange basis on nodes r (product formula)."""
    r = np.asarray(r, dtype=np.float64)
    out = np.ones(r.size)
    for j in range(r.size):
        for k in range(r.size):
            if k != j:
                out[j] *= (xi - r[k]) / (r[j] - r[k])
    return out


def cfl_dt(cfl, h, c_max, N):
    """dt = CFL h / (c_max N^2): the CFL number CFL = dt |beta| p^2 / h that the
    paper's time-dependent transport table lists (Section 6.1)."""
    return cfl * h / (c_max * N * N)


def cfl_number(dt, h, c_max, N):
    return dt * c_max * N * N / h


# --------------------------------------------------------------------------
# Mesh geometry, connectivity and the semi-discrete operator
# --------------------------------------------------------------------------
TANGENTS = {0: (1, 2), 1: (0, 2), 2: (0, 1)}


def face_node_indices(f: int, N: int):
    """Volume node indices of local face f, ordered by face-local (a, b), a fastest."""
    n = N + 1
    d, side = f // 2, (-1 if f % 2 == 0 else 1)
    t0, t1 = TANGENTS[d]
    out = []
    for b in range(n):
        for a in range(n):
            ijk = [0, 0, 0]
            ijk[d] = 0 if side < 0 else N
            ijk[t0] = a
            ijk[t1] = b
            out.append(ijk[0] + n * (ijk[1] + n * ijk[2]))
    return np.array(out, dtype=np.int64)


def neighbour_face_position(o: int, a: int, b: int, N: int):
    """Face-node permutation: own (a, b) -> neighbour (a', b')."""
    a1, b1 = (b, a) if (o & 1) else (a, b)
    return (N - a1 if (o & 2) else a1), (N - b1 if (o & 4) else b1)


class ElasticDG:
    """The semi-discrete operator du/dt = L(u) on one mesh and medium."""

    def __init__(self, N, x, etoe, etof, orient, bc, rho, lam, mu, tau=1):
        self.N = int(N)
        n = self.N + 1
        self.n, self.Np = n, n ** 3
        self.r, self.w = gll(self.N)
        self.D = lagrange_derivative_matrix(self.r)
        self.x = np.asarray(x, dtype=np.float64)
        self.nel = self.x.shape[0]
        self.etoe = np.asarray(etoe, dtype=np.int64)
        self.etof = np.asarray(etof, dtype=np.int64)
        self.orient = np.asarray(orient, dtype=np.int64)
        self.bc = np.asarray(bc, dtype=np.int64)
        self.rho = np.asarray(rho, dtype=np.float64)
        self.lam = np.asarray(lam, dtype=np.float64)
        self.mu = np.asarray(mu, dtype=np.float64)
        self.tau = float(tau)
        self.m = NFIELD
        self.self_only = False      # True: interior neighbour states taken as zero (L_K^self)
        self.face_nodes = [face_node_indices(f, self.N) for f in range(6)]
        wv = np.einsum("k,j,i->kji", self.w, self.w, self.w).ravel()
        self.w_vol = wv                                        # [Np]
        self.w_face = np.einsum("b,a->ba", self.w, self.w).ravel()   # [n^2], a fastest
        self.source = None
        self.receivers = []
        self._geo_cache = {}
        self._nbr_cache = {}
        self._abs_cache = {}
        self._qinv_cache = {}

    # ---- reference derivatives: u[..., Np] -> d/dxi_axis -----------------
    def dref(self, u, axis):
        n = self.n
        v = u.reshape(u.shape[:-1] + (n, n, n))              # [..., k, j, i]
        if axis == 0:
            out = np.einsum("ai,...kji->...kja", self.D, v)
        elif axis == 1:
            out = np.einsum("aj,...kji->...kai", self.D, v)
        else:
            out = np.einsum("ak,...kji->...aji", self.D, v)
        return out.reshape(u.shape)

    # ---- geometry (curl-form metric terms, Kopriva 2006) -----------------
    def geometry(self, elems):
        """Ja[i][k] = J d xi_i / d x_k in conservative curl form, and J, for elems."""
        key = elems.tobytes()
        if key in self._geo_cache:
            return self._geo_cache[key]
        # Element-centred coordinates: the discrete metrics are unchanged in exact
        # arithmetic (D annihilates constants and the discrete curl of c grad X_m
        # vanishes because D_j and D_k commute), but rounding no longer scales
        # with |x| / h.
        xe = self.x[elems]
        X = np.moveaxis(xe - xe.mean(axis=1, keepdims=True), 2, 0)   # [3, ne, Np]
        dX = np.stack([self.dref(X, ax) for ax in range(3)])  # dX[axis][coord]
        Ja = np.zeros((3, 3) + X.shape[1:])
        for ncomp in range(3):
            m, l = (ncomp + 1) % 3, (ncomp + 2) % 3
            W = [X[l] * dX[k][m] for k in range(3)]          # W_k = X_l d_k X_m
            Ja[0][ncomp] = -(self.dref(W[2], 1) - self.dref(W[1], 2))
            Ja[1][ncomp] = -(self.dref(W[0], 2) - self.dref(W[2], 0))
            Ja[2][ncomp] = -(self.dref(W[1], 0) - self.dref(W[0], 1))
        # J = det(dX/dxi): rows = coordinate, columns = reference axis
        G = np.stack([np.stack([dX[ax][c] for ax in range(3)], axis=-1) for c in range(3)], axis=-2)
        J = np.linalg.det(G)
        self._geo_cache[key] = (Ja, J)
        return Ja, J

    def outward_scaled_normal(self, Ja, f):
        """n sJ on local face f at its face nodes: +-Ja[d] (Ja[d] points to +xi_d)."""
        d, side = f // 2, (-1 if f % 2 == 0 else 1)
        return side * np.moveaxis(Ja[d][:, :, self.face_nodes[f]], 0, -1)   # [ne, nf, 3]

    def face_material(self, elems, f):
        """(rho, lam, mu) on face f of each element: the average of the two sides
        on interior faces (the medium may jump there), the element's own on
        boundary faces."""
        e2 = self.etoe[elems, f]
        interior = (e2 >= 0) & (self.bc[elems, f] == 0)
        other = np.where(interior, e2, elems)
        return tuple(0.5 * (v[elems] + v[other]) for v in (self.rho, self.lam, self.mu))

    def _abs_A_cached(self, elems, f, nrm):
        key = (elems.tobytes(), f)
        if key not in self._abs_cache:
            rho, lam, mu = self.face_material(elems, f)
            shape = nrm.shape[:-1]
            self._abs_cache[key] = abs_A_Q(nrm, *(np.broadcast_to(v[:, None], shape) for v in (rho, lam, mu)))
        return self._abs_cache[key]

    def Qinv(self, elems):
        key = elems.tobytes()
        if key not in self._qinv_cache:
            self._qinv_cache[key] = np.stack([np.linalg.inv(Q_of(self.rho[e], self.lam[e], self.mu[e]))
                                              for e in elems])
        return self._qinv_cache[key]

    def _neighbour_map(self, f, elems=None):
        """For face f of each element in elems (default all): flat index e2*Np + node2
        of the matching neighbour node per face node (-1 on tagged boundary faces)."""
        elems = np.arange(self.nel) if elems is None else np.asarray(elems, dtype=np.int64)
        key = (elems.tobytes(), f)
        if key in self._nbr_cache:
            return self._nbr_cache[key]
        N, n = self.N, self.N + 1
        out = -np.ones((len(elems), n * n), dtype=np.int64)
        for idx, e in enumerate(elems):
            e2 = self.etoe[e, f]
            if e2 < 0 or self.bc[e, f] != 0:
                continue
            fn2 = self.face_nodes[self.etof[e, f]]
            o = self.orient[e, f]
            for b in range(n):
                for a in range(n):
                    a2, b2 = neighbour_face_position(o, a, b, N)
                    out[idx, a + n * b] = e2 * self.Np + fn2[a2 + n * b2]
        self._nbr_cache[key] = out
        return out

    def exterior_state(self, u, elems, f):
        """(u^-, u^+) at the face nodes of face f of each element in elems: [9, ne, nf]."""
        fn = self.face_nodes[f]
        um = u[:, elems][:, :, fn]
        nbr = self._neighbour_map(f, elems)                   # [ne, nf]
        tag = self.bc[elems, f]
        interior = (self.etoe[elems, f] >= 0) & (tag == 0)
        if np.any(~interior & (tag == 0)):
            raise ValueError(f"face {f}: element without neighbour and without boundary tag")
        flat = u.reshape(NFIELD, -1)
        up = np.zeros_like(um)
        if not self.self_only:
            up[:, interior] = flat[:, nbr[interior]]
        free = tag == 1           # traction-free: keep the velocity, mirror the stress
        up[:3, free] = um[:3, free]
        up[3:, free] = -um[3:, free]
        # tag == 2, absorbing: zero exterior state (already zero)
        return um, up

    # ---- the operator ----------------------------------------------------
    def volume_term(self, u_e, Ja, J, sign=1.0):
        """Split (skew-symmetric) strong form of -sum_k d_k(A_k u):
        -1/2 [ 1/J sum_i d_i(sum_k Ja^i_k A_k u) + 1/J sum_i sum_k Ja^i_k A_k d_i u ].
        sign = -1 evaluates the same form with A_k replaced by -A_k."""
        Ak = [sign * A_K[k] for k in range(3)]
        Au = [np.einsum("pq,qen->pen", Ak[k], u_e) for k in range(3)]
        cons = np.zeros_like(u_e)
        noncons = np.zeros_like(u_e)
        for i in range(3):
            Ftilde = sum(Ja[i][k][None] * Au[k] for k in range(3))
            cons += self.dref(Ftilde, i)
            du = self.dref(u_e, i)
            noncons += sum(Ja[i][k][None] * np.einsum("pq,qen->pen", Ak[k], du) for k in range(3))
        return -0.5 * (cons + noncons) / J[None]

    def surface_term(self, u, elems, Ja, J, sign=1.0):
        """Sum over faces of (w_f sJ)/(w_vol J) (F(u^-).n - F_hat.n) at the face nodes.
        sign = -1: flux matrices A(n) replaced by -A(n), stabilisation unchanged."""
        out = np.zeros((NFIELD, len(elems), self.Np))
        for f in range(6):
            fn = self.face_nodes[f]
            m = self.outward_scaled_normal(Ja, f)             # [ne, nf, 3]
            sJ = np.linalg.norm(m, axis=-1)
            nrm = m / sJ[..., None]
            um, up = self.exterior_state(u, elems, f)
            um = np.moveaxis(um, 0, -1)                        # [ne, nf, 9]
            up = np.moveaxis(up, 0, -1)
            An = sign * np.einsum("...k,kij->...ij", nrm, A_STACK)
            stab = self.tau * self._abs_A_cached(elems, f, nrm)
            s_uhat = weighted_trace(An, stab, um, up)
            Fhat = hdg_flux(An, stab, um, s_uhat)
            q = np.einsum("...ij,...j->...i", An, um) - Fhat   # F(u^-).n - F_hat.n
            scale = self.w_face[None, :] * sJ / (self.w_vol[fn][None, :] * J[:, fn])
            out[:, :, fn] += np.moveaxis(q * scale[..., None], -1, 0)
        return out

    def set_point_force(self, element, xi, force, f0, t0):
        """Point force F R(t) delta(x - x_s) in the velocity equations (the forcing f
        of eq. LPDE), x_s the image of reference point xi in `element`, R a Ricker
        wavelet of peak frequency f0 centred at t0."""
        self.source = (int(element), np.asarray(xi, dtype=np.float64), np.asarray(force, dtype=np.float64),
                       float(f0), float(t0))

    def source_nodal(self, t):
        """Collocation projection of the point force: M^{-1} int f phi_j, i.e.
        F R(t) l_j(xi_s) / (w_j J_j) at the nodes of the source element (before Q^{-1})."""
        e, xi, F, f0, t0 = self.source
        li = [lagrange_values(self.r, xi[a]) for a in range(3)]
        l3 = np.einsum("k,j,i->kji", li[2], li[1], li[0]).ravel()
        _, J = self.geometry(np.array([e]))
        s = np.zeros((NFIELD, self.Np))
        s[:3] = F[:, None] * float(ricker(t, f0, t0)) * l3[None, :] / (self.w_vol * J[0])[None, :]
        return e, s

    def rhs(self, u, elems=None, t=0.0, sign=1.0, source=True):
        """L(u) = Q^{-1}[volume + surface + source] for the elements in elems (default all).
        sign = -1 gives the reversed operator L_rev (A_k -> -A_k, same stabilisation)."""
        u = np.asarray(u, dtype=np.float64)
        elems = np.arange(self.nel) if elems is None else np.asarray(elems, dtype=np.int64)
        Ja, J = self.geometry(elems)
        if np.any(J <= 0.0):
            raise ValueError("non-positive Jacobian")
        u_e = u[:, elems]
        r = self.volume_term(u_e, Ja, J, sign) + self.surface_term(u, elems, Ja, J, sign)
        if source and self.source is not None:
            es, sn = self.source_nodal(t)
            hit = np.nonzero(elems == es)[0]
            if hit.size:
                r[:, hit[0]] += sn
        return np.einsum("epq,qen->pen", self.Qinv(elems), r)

    # ---- adjoint ---------------------------------------------------------
    def mass_Q(self, u, inverse=False):
        """Apply M Q (or its inverse) node by node: w J Q_e u (Q_e per element)."""
        elems = np.arange(self.nel)
        _, J = self.geometry(elems)
        out = np.empty_like(u)
        for e in elems:
            Q = Q_of(self.rho[e], self.lam[e], self.mu[e])
            wJ = self.w_vol * J[e]
            if inverse:
                out[:, e] = np.linalg.solve(Q, u[:, e]) / wJ[None, :]
            else:
                out[:, e] = (Q @ u[:, e]) * wJ[None, :]
        return out

    def rhs_adjoint(self, w):
        """L^T w (Euclidean transpose of the linear part of L).  M Q L splits into a
        part that is skew and linear in A (volume + central flux) and a symmetric
        part independent of the sign of A (stabilisation), so
        L^T = (M Q) L_rev (M Q)^{-1}, L_rev = L with A_k -> -A_k."""
        return self.mass_Q(self.rhs(self.mass_Q(w, inverse=True), sign=-1.0, source=False))

    def adjoint_stage(self, lu, lr, s, dt):
        """Transpose of the stage map (u, res) -> (u + b_s res', res'),
        res' = a_s res + dt L u:  w = b_s lu + lr;  lu <- lu + dt L^T w;  lr <- a_s w."""
        a, b = float(LSRK_A[s]), float(LSRK_B[s])
        w = b * lu + lr
        return lu + dt * self.rhs_adjoint(w), a * w

    def adjoint_step(self, lu, lr, dt):
        for s in reversed(range(5)):
            lu, lr = self.adjoint_stage(lu, lr, s, dt)
        return lu, lr

    # ---- receivers --------------------------------------------------------
    def set_receivers(self, elems, xis):
        self.receivers = [(int(e), np.asarray(x, dtype=np.float64)) for e, x in zip(elems, xis)]

    def _receiver_basis(self, xi):
        li = [lagrange_values(self.r, xi[a]) for a in range(3)]
        return np.einsum("k,j,i->kji", li[2], li[1], li[0]).ravel()

    def sample_receivers(self, u):
        """Velocity at the receivers: sum_j l_j(xi_r) v_j over the receiver's element."""
        return np.array([u[:3, e] @ self._receiver_basis(xi) for e, xi in self.receivers])

    def receivers_adjoint(self, g):
        """Transpose of sample_receivers: g [nrec, 3] -> a state-shaped array."""
        out = np.zeros((NFIELD, self.nel, self.Np))
        for (e, xi), gr in zip(self.receivers, g):
            out[:3, e] += gr[:, None] * self._receiver_basis(xi)[None, :]
        return out

    # ---- misfit and material gradient (small problems) --------------------
    def forward_traces(self, u0, dt, nsteps, t0=0.0):
        """States at step starts and receiver traces after each step."""
        u, res = u0.copy(), np.zeros_like(u0)
        starts, traces = [], []
        for k in range(nsteps):
            starts.append(u.copy())
            u, res = self.step(u, res, dt, t=t0 + k * dt)
            traces.append(self.sample_receivers(u))
        return starts, np.array(traces)

    def misfit(self, traces, data, dt):
        """J = 1/2 dt sum_n sum_r |v_r(t_n) - d_r(t_n)|^2."""
        return 0.5 * dt * float(np.sum((traces - data) ** 2))

    def dL_dm(self, u, e, p, t=0.0, h_rel=1e-6):
        """d/dm of the stage right-hand side L(u) + Q^{-1} f(t) for parameter p in
        {0: rho, 1: lam, 2: mu} of element e, by a central difference in that
        parameter (the operator is smooth in the medium; the point force enters
        through Q^{-1}); only e and its neighbours change."""
        vals = [self.rho, self.lam, self.mu]
        base = vals[p][e]
        h = h_rel * abs(base)
        nb = sorted({int(e)} | {int(x) for x in self.etoe[e] if x >= 0})
        elems = np.array(nb)
        out = []
        for sgn in (1.0, -1.0):
            vals[p][e] = base + sgn * h
            self._abs_cache.clear()
            self._qinv_cache.clear()
            out.append(self.rhs(u, elems, t=t))
        vals[p][e] = base
        self._abs_cache.clear()
        self._qinv_cache.clear()
        return elems, (out[0] - out[1]) / (2 * h)

    def gradient(self, u0, data, dt, nsteps, elems_params, t0=0.0):
        """dJ/dm for the listed (element, parameter) pairs by the discrete adjoint:
        backward over steps and stages, with the stage inputs recomputed from the
        step starts, accumulating dt w_s^T (dL/dm) u_{s-1}."""
        starts, traces = self.forward_traces(u0, dt, nsteps, t0)
        lu = np.zeros_like(u0)
        lr = np.zeros_like(u0)
        grad = np.zeros(len(elems_params))
        for k in reversed(range(nsteps)):
            lu = lu + self.receivers_adjoint(dt * (traces[k] - data[k]))
            # stage inputs of step k
            u, res = starts[k].copy(), np.zeros_like(u0)
            ins = []
            for s in range(5):
                ins.append(u)
                u, res = self.lsrk_stage(u, res, s, dt, t=t0 + k * dt)
            for s in reversed(range(5)):
                a, b = float(LSRK_A[s]), float(LSRK_B[s])
                w = b * lu + lr
                ts = t0 + k * dt + float(LSRK_C[s]) * dt
                for i, (e, p) in enumerate(elems_params):
                    el, d = self.dL_dm(ins[s], e, p, ts)
                    grad[i] += dt * float(np.sum(w[:, el] * d))
                lu, lr = lu + dt * self.rhs_adjoint(w), a * w
        return grad

    # ---- time stepping ---------------------------------------------------
    def lsrk_stage(self, u, res, s, dt, elems=None, t=0.0):
        """One 2N-storage stage from step time t: res <- a_s res + dt L(u, t + c_s dt);
        u <- u + b_s res."""
        elems = np.arange(self.nel) if elems is None else np.asarray(elems, dtype=np.int64)
        a, b = float(LSRK_A[s]), float(LSRK_B[s])
        res_new = a * res[:, elems] + dt * self.rhs(u, elems, t + float(LSRK_C[s]) * dt)
        u_new = u[:, elems] + b * res_new
        return u_new, res_new

    def step(self, u, res, dt, t=0.0):
        u = u.copy()
        res = res.copy()
        for s in range(5):
            u, res = self.lsrk_stage(u, res, s, dt, t=t)
        return u, res

    # ---- energy -----------------------------------------------------------
    def energy(self, u):
        """E = 1/2 sum_K sum_nodes w J u^T Q u."""
        elems = np.arange(self.nel)
        _, J = self.geometry(elems)
        E = 0.0
        for e in elems:
            Q = Q_of(self.rho[e], self.lam[e], self.mu[e])
            ue = u[:, e, :]
            E += 0.5 * np.sum(self.w_vol * J[e] * np.einsum("pn,pq,qn->n", ue, Q, ue))
        return E

    def energy_rate(self, u):
        """dE/dt = sum w J u^T Q L(u) along the semi-discrete flow."""
        elems = np.arange(self.nel)
        _, J = self.geometry(elems)
        L = self.rhs(u)
        E = 0.0
        for e in elems:
            Q = Q_of(self.rho[e], self.lam[e], self.mu[e])
            E += np.sum(self.w_vol * J[e] * np.einsum("pn,pq,qn->n", u[:, e], Q, L[:, e]))
        return E

    def energy_rate_from_faces(self, u):
        """The same rate written with face quantities only:
        sum over element-face sides of w_f sJ (-1/2 u^-.A(n)u^+ - 1/2 u^-.Stab(u^- - u^+))."""
        elems = np.arange(self.nel)
        Ja, J = self.geometry(elems)
        total = 0.0
        for f in range(6):
            m = self.outward_scaled_normal(Ja, f)
            sJ = np.linalg.norm(m, axis=-1)
            nrm = m / sJ[..., None]
            um, up = self.exterior_state(u, elems, f)
            um = np.moveaxis(um, 0, -1)
            up = np.moveaxis(up, 0, -1)
            An = np.einsum("...k,kij->...ij", nrm, A_STACK)
            stab = self.tau * self._abs_A_cached(elems, f, nrm)
            t = (-0.5 * np.einsum("...i,...ij,...j->...", um, An, up)
                 - 0.5 * np.einsum("...i,...ij,...j->...", um, stab, um - up))
            total += np.sum(self.w_face[None, :] * sJ * t)
        return total

    def c_max(self):
        return float(np.max(np.sqrt((self.lam + 2.0 * self.mu) / self.rho)))


def h_min_corner_edges(x, N):
    """Shortest element edge: the smallest distance between element corner nodes
    joined by an element edge (12 per hexahedron)."""
    n = N + 1
    corners = [i + n * (j + n * k) for k in (0, N) for j in (0, N) for i in (0, N)]
    xc = np.asarray(x)[:, corners, :]                       # [nel, 8, 3], corner c = (i, j, k) bits
    edges = [(0, 1), (2, 3), (4, 5), (6, 7), (0, 2), (1, 3), (4, 6), (5, 7), (0, 4), (1, 5), (2, 6), (3, 7)]
    return float(min(np.min(np.linalg.norm(xc[:, a] - xc[:, b], axis=-1)) for a, b in edges))
