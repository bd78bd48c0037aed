"""Structured hexahedral meshes of the unit cube (topology and node coordinates).

The paper runs every experiment on structured quadrilateral/hexahedral meshes
of the unit square/cube (Section 6).  This module builds such meshes:

* element ordering: lexicographic, or Morton (z-order) as produced by
  forest-of-octree mesh libraries;
* connectivity arrays in the library's layout: for element ``e`` and local
  face ``f`` (0: r=-1, 1: r=+1, 2: s=-1, 3: s=+1, 4: t=-1, 5: t=+1)
  ``etoe[e, f]`` is the neighbour element (-1 on a physical boundary),
  ``etof[e, f]`` the neighbour's local face, ``orient[e, f]`` the face-node
  permutation code and ``bc[e, f]`` the boundary tag;
* optional random rigid re-orientation of each element's local frame, which
  exercises all eight face-node permutation codes;
* node coordinates at caller-supplied 1-D reference nodes, mapped through the
  smooth curvilinear warp ``x_i -> x_i + a * prod_j sin(2 pi x_j)``.

Face-node permutation code ``o`` (0..7).  A face's nodes are indexed by
face-local ``(a, b)``: ``a`` runs along the lower-numbered tangential axis,
``b`` along the higher one.  The matching node on the neighbour's face is
``(a', b')`` with ``(a1, b1) = (b, a) if o & 1 else (a, b)``,
``a' = N - a1 if o & 2 else a1`` and ``b' = N - b1 if o & 4 else b1``.

Nothing here computes any part of the discretisation (no quadrature, no
derivatives, no fluxes): the reference node positions are an argument.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field, replace

import numpy as np

BC_INTERIOR = 0       # interior or periodic face: neighbour via etoe/etof/orient
BC_FREE_SURFACE = 1   # traction-free surface
BC_WALL = 1           # the same tag for the shallow-water system: reflecting wall
BC_ABSORBING = 2      # zero exterior state

_TANGENTS = {0: (1, 2), 1: (0, 2), 2: (0, 1)}


@dataclass
class Mesh:
    E: tuple                      # elements per axis (Ex, Ey, Ez)
    cell: np.ndarray              # [nel, 3] int64 cell index of each element
    frame: np.ndarray             # [nel, 3, 3] int64 signed permutation: canonical = frame @ local
    etoe: np.ndarray              # [nel, 6] int64
    etof: np.ndarray              # [nel, 6] int8
    orient: np.ndarray            # [nel, 6] int8
    bc: np.ndarray                # [nel, 6] int8
    periodic: tuple = (True, True, True)
    boundary: dict = field(default_factory=dict)

    @property
    def nel(self) -> int:
        return int(self.cell.shape[0])


def _morton_key(cell: np.ndarray) -> np.ndarray:
    key = np.zeros(cell.shape[0], dtype=np.int64)
    for bit in range(21):
        for ax in range(3):
            key |= ((cell[:, ax] >> bit) & 1) << (3 * bit + ax)
    return key


def _apply_orient(o: int, a, b, N: int):
    a1, b1 = (b, a) if (o & 1) else (a, b)
    a2 = N - a1 if (o & 2) else a1
    b2 = N - b1 if (o & 4) else b1
    return a2, b2


def _connect(cell, frame, E, periodic, boundary):
    """Connectivity for arbitrary per-element frames (signed permutations)."""
    nel = cell.shape[0]
    E = np.asarray(E, dtype=np.int64)
    index = -np.ones(tuple(E), dtype=np.int64)
    index[cell[:, 0], cell[:, 1], cell[:, 2]] = np.arange(nel)
    etoe = -np.ones((nel, 6), dtype=np.int64)
    etof = -np.ones((nel, 6), dtype=np.int8)
    orient = np.zeros((nel, 6), dtype=np.int8)
    bc = np.zeros((nel, 6), dtype=np.int8)

    identity = bool(np.all(frame == np.eye(3, dtype=frame.dtype)))
    if identity:
        # Aligned frames: face f of e meets face f^1 of the neighbour, same node order.
        for f in range(6):
            d, side = f // 2, (-1 if f % 2 == 0 else 1)
            nb = cell.copy()
            nb[:, d] += side
            outside = (nb[:, d] < 0) | (nb[:, d] >= E[d])
            if periodic[d]:
                nb[:, d] %= E[d]
                outside[:] = False
            inside = ~outside
            etoe[inside, f] = index[nb[inside, 0], nb[inside, 1], nb[inside, 2]]
            etof[inside, f] = f ^ 1
            bc[outside, f] = boundary.get(f, BC_ABSORBING)
        return etoe, etof, orient, bc

    # General frames: per element and face (small test meshes only).
    corners = [(0, 0), (1, 0), (0, 1)]
    for e in range(nel):
        Fe = frame[e]
        for f in range(6):
            d, side = f // 2, (-1 if f % 2 == 0 else 1)
            vec = Fe[:, d] * side                      # canonical outward direction
            dc = int(np.nonzero(vec)[0][0])
            sc = int(vec[dc])
            nb = cell[e].copy()
            nb[dc] += sc
            if not (0 <= nb[dc] < E[dc]) and not periodic[dc]:
                bc[e, f] = boundary.get(2 * dc + (1 if sc > 0 else 0), BC_ABSORBING)
                continue
            nbw = nb.copy()
            nbw[dc] %= E[dc]
            en = int(index[tuple(nbw)])
            Fn = frame[en]
            fn = None
            for g in range(6):
                dg, sg = g // 2, (-1 if g % 2 == 0 else 1)
                if np.array_equal(Fn[:, dg] * sg, -vec):
                    fn = g
                    break
            t0, t1 = _TANGENTS[d]
            dn = fn // 2
            u0, u1 = _TANGENTS[dn]
            found = None
            for o in range(8):
                ok = True
                for (a, b) in corners:
                    rho = np.zeros(3, dtype=np.int64)
                    rho[d] = side
                    rho[t0] = 2 * a - 1
                    rho[t1] = 2 * b - 1
                    twice_p = 2 * cell[e] + Fe @ rho + 1          # 2 * canonical position
                    rho_n = Fn.T @ (twice_p - 2 * nb - 1)        # neighbour local coords
                    an, bn = (rho_n[u0] + 1) // 2, (rho_n[u1] + 1) // 2
                    if _apply_orient(o, a, b, 1) != (an, bn):
                        ok = False
                        break
                if ok:
                    found = o
                    break
            assert found is not None
            etoe[e, f] = en
            etof[e, f] = fn
            orient[e, f] = found
    return etoe, etof, orient, bc


def structured_hex_mesh(E, periodic=(True, True, True), boundary=None, order="lex") -> Mesh:
    """Ex x Ey x Ez hexahedra filling the unit cube.

    ``boundary`` maps a canonical face id (0: x=0, 1: x=1, 2: y=0, 3: y=1,
    4: z=0, 5: z=1) to a boundary tag for the non-periodic axes; untagged
    boundary faces are absorbing.  ``order`` is ``"lex"`` (x fastest) or
    ``"morton"`` (z-order of the cell index).
    """
    if np.isscalar(E):
        E = (int(E),) * 3
    E = tuple(int(v) for v in E)
    boundary = dict(boundary or {})
    ez, ey, ex = np.meshgrid(np.arange(E[2]), np.arange(E[1]), np.arange(E[0]), indexing="ij")
    cell = np.stack([ex.ravel(), ey.ravel(), ez.ravel()], axis=1).astype(np.int64)
    if order == "morton":
        cell = cell[np.argsort(_morton_key(cell), kind="stable")]
    elif order != "lex":
        raise ValueError(f"unknown element order {order!r}")
    frame = np.broadcast_to(np.eye(3, dtype=np.int64), (cell.shape[0], 3, 3)).copy()
    etoe, etof, orient, bc = _connect(cell, frame, E, tuple(periodic), boundary)
    return Mesh(E, cell, frame, etoe, etof, orient, bc, tuple(periodic), boundary)


def _proper_rotations():
    rots = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), dtype=np.int64)
            for i, p in enumerate(perm):
                R[p, i] = signs[i]
            if round(np.linalg.det(R)) == 1:
                rots.append(R)
    return rots


def rotate_elements(mesh: Mesh, seed: int) -> Mesh:
    """Give every element a random proper rotation of its local frame (24 choices)."""
    rots = _proper_rotations()
    rng = np.random.default_rng(seed)
    choice = rng.integers(0, len(rots), size=mesh.nel)
    frame = np.stack([rots[c] for c in choice]).astype(np.int64)
    etoe, etof, orient, bc = _connect(mesh.cell, frame, mesh.E, mesh.periodic, mesh.boundary)
    return replace(mesh, frame=frame, etoe=etoe, etof=etof, orient=orient, bc=bc)


def reference_grid(r1d) -> np.ndarray:
    """[Np, 3] local reference coordinates; node index i + (N+1)(j + (N+1)k), r fastest."""
    r1d = np.asarray(r1d, dtype=np.float64)
    t, s, r = np.meshgrid(r1d, r1d, r1d, indexing="ij")
    return np.stack([r.ravel(), s.ravel(), t.ravel()], axis=1)


def warped_node_coords(mesh: Mesh, r1d, amplitude: float) -> np.ndarray:
    """Physical coordinates [nel, Np, 3] of the nodes at reference positions ``r1d``.

    The undeformed map sends local reference coords through the element frame
    to the cell ``[c/E, (c+1)/E]``; the warp is ``x_i + a * prod_j sin(2 pi x_j)``
    for every axis i (it vanishes on the cube's faces, so periodicity and flat
    boundary faces are kept).
    """
    rho = reference_grid(r1d)                                   # [Np, 3]
    rho_c = np.einsum("eij,nj->eni", mesh.frame.astype(np.float64), rho)
    E = np.asarray(mesh.E, dtype=np.float64)
    X = (mesh.cell[:, None, :].astype(np.float64) + (rho_c + 1.0) * 0.5) / E
    if amplitude != 0.0:
        S = np.prod(np.sin(2.0 * np.pi * X), axis=2)
        X = X + amplitude * S[:, :, None]
    return np.ascontiguousarray(X)


def cell_centroids(mesh: Mesh) -> np.ndarray:
    """Undeformed element centres [nel, 3]."""
    return (mesh.cell.astype(np.float64) + 0.5) / np.asarray(mesh.E, dtype=np.float64)
