"""Structured meshes for the four element families (P1, P2, Q1, Q2) in 2D and 3D.

This module only builds inputs: node coordinates and element connectivity on a
box, in the reference node orders of the paper's Appendix (P1/P2 tetrahedra,
Q1/Q2 hexahedra) and their plane analogues (P1/P2 triangles, Q1 quadrilateral,
8-node serendipity Q2 quadrilateral).  It holds none of the method's
arithmetic (no basis functions, no quadrature, no Jacobians).

Node numbering follows a lattice with spacing h (order 1) or h/2 (order 2),
x fastest, then y, then z.  Serendipity Q2 meshes drop the lattice points that
no element uses (cell centres in 2D; face and cell centres in 3D) and renumber
the rest in the same lexicographic order.

Element splits:
  * 2D simplices: every square (i,j) is cut along its (i,j)-(i+1,j+1) diagonal
    into two counter-clockwise triangles.
  * 3D simplices: every cube is cut into the six Kuhn tetrahedra that share the
    (0,0,0)-(1,1,1) diagonal (the split is conforming across cube faces); each
    tetrahedron is ordered so that its Jacobian determinant is positive.

All connectivity is 0-based int32 with shape [n_e][n_p]; coordinates are
float64 with shape [n_n][dim].
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

ELEMENT_FAMILIES = ("P1", "P2", "Q1", "Q2")

# number of nodes per element, by (family, dim)
N_NODES = {
    ("P1", 2): 3, ("P2", 2): 6, ("Q1", 2): 4, ("Q2", 2): 8,
    ("P1", 3): 4, ("P2", 3): 10, ("Q1", 3): 8, ("Q2", 3): 20,
}


@dataclass
class Mesh:
    elem_type: str          # "P1" | "P2" | "Q1" | "Q2"
    dim: int                # 2 (plane strain) or 3
    coords: np.ndarray      # float64 [n_n][dim]
    elem: np.ndarray        # int32 [n_e][n_p], 0-based
    shape: tuple            # cells per axis
    size: tuple             # box edge lengths

    @property
    def n_nodes(self) -> int:
        return self.coords.shape[0]

    @property
    def n_elem(self) -> int:
        return self.elem.shape[0]

    @property
    def n_p(self) -> int:
        return self.elem.shape[1]


def _lattice(n_cells, order):
    """Lattice points per axis for the given element order."""
    return tuple(order * n + 1 for n in n_cells)


def _lin(idx, dims):
    """Lexicographic (x fastest) index of lattice coordinates."""
    out = np.zeros_like(idx[0])
    stride = 1
    for a, d in zip(idx, dims):
        out = out + a * stride
        stride *= d
    return out


def _cell_origins(n_cells):
    """Integer origins of all cells, x fastest; returns list of arrays per axis."""
    grids = np.meshgrid(*[np.arange(n) for n in n_cells], indexing="ij")
    # x fastest: flatten in Fortran order over (x, y[, z])
    return [g.ravel(order="F") for g in grids]


def _kuhn_tets():
    """Six Kuhn tetrahedra of the unit cube as vertex offsets, positively oriented."""
    tets = []
    for perm in itertools.permutations(range(3)):
        v = [np.zeros(3, dtype=np.int64)]
        cur = np.zeros(3, dtype=np.int64)
        for ax in perm:
            cur = cur.copy()
            cur[ax] += 1
            v.append(cur)
        m = np.array([v[1] - v[0], v[2] - v[0], v[3] - v[0]], dtype=np.float64)
        if np.linalg.det(m) < 0:
            v[2], v[3] = v[3], v[2]
        tets.append(v)
    return tets


# local edge lists for the quadratic elements (midpoint order of the Appendix)
_TRI_P2_EDGES = [(0, 1), (1, 2), (0, 2)]
_TET_P2_EDGES = [(0, 1), (1, 2), (0, 2), (1, 3), (2, 3), (0, 3)]
_QUAD_Q2_EDGES = [(0, 1), (1, 2), (2, 3), (3, 0)]
_HEX_Q2_EDGES = [(0, 1), (1, 2), (2, 3), (3, 0), (4, 5), (5, 6), (6, 7), (7, 4),
                 (0, 4), (1, 5), (2, 6), (3, 7)]
# reference hexahedron corner order (Appendix, Q1): (-1,-1,-1),(1,-1,-1),(1,1,-1),(-1,1,-1), then z=+1
_HEX_CORNERS = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
                (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
_QUAD_CORNERS = [(0, 0), (1, 0), (1, 1), (0, 1)]


def structured_mesh(elem_type: str, dim: int, n_cells, size=None) -> Mesh:
    """Structured mesh of the box [0,size_0] x ... with n_cells cells per axis."""
    if elem_type not in ELEMENT_FAMILIES:
        raise ValueError(f"unknown element type {elem_type}")
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    n_cells = tuple(int(n) for n in n_cells)
    if len(n_cells) != dim or min(n_cells) < 1:
        raise ValueError("n_cells must have one positive entry per axis")
    size = tuple(float(s) for s in (size if size is not None else (10.0,) * dim))
    order = 2 if elem_type in ("P2", "Q2") else 1
    lat = _lattice(n_cells, order)
    origins = _cell_origins(n_cells)
    o = [order * a for a in origins]          # cell origin in lattice units

    def node(offsets):
        """lattice index of cell-local lattice offsets (in lattice units)"""
        return _lin([o[a] + offsets[a] for a in range(dim)], lat)

    cols = []
    if dim == 2:
        if elem_type in ("P1", "P2"):
            a, b, c, d = [(0, 0), (1, 0), (1, 1), (0, 1)]
            tris = [(a, b, c), (a, c, d)]
            per_cell = []
            for tri in tris:
                verts = [tuple(order * t for t in v) for v in tri]
                nodes = list(verts)
                if elem_type == "P2":
                    for i, j in _TRI_P2_EDGES:
                        nodes.append(tuple((verts[i][k] + verts[j][k]) // 2 for k in range(2)))
                per_cell.append([node(v) for v in nodes])
            # interleave the two triangles of each cell: element 2*cell + t
            elem = np.stack([np.stack(t, axis=1) for t in per_cell], axis=1).reshape(-1, len(per_cell[0]))
        else:
            corners = [tuple(order * t for t in v) for v in _QUAD_CORNERS]
            nodes = list(corners)
            if elem_type == "Q2":
                for i, j in _QUAD_Q2_EDGES:
                    nodes.append(tuple((corners[i][k] + corners[j][k]) // 2 for k in range(2)))
            elem = np.stack([node(v) for v in nodes], axis=1)
    else:
        if elem_type in ("P1", "P2"):
            per_cell = []
            for tet in _kuhn_tets():
                verts = [tuple(int(order * t) for t in v) for v in tet]
                nodes = list(verts)
                if elem_type == "P2":
                    for i, j in _TET_P2_EDGES:
                        nodes.append(tuple((verts[i][k] + verts[j][k]) // 2 for k in range(3)))
                per_cell.append([node(v) for v in nodes])
            elem = np.stack([np.stack(t, axis=1) for t in per_cell], axis=1).reshape(-1, len(per_cell[0]))
        else:
            corners = [tuple(order * t for t in v) for v in _HEX_CORNERS]
            nodes = list(corners)
            if elem_type == "Q2":
                for i, j in _HEX_Q2_EDGES:
                    nodes.append(tuple((corners[i][k] + corners[j][k]) // 2 for k in range(3)))
            elem = np.stack([node(v) for v in nodes], axis=1)

    # lattice coordinates
    axes = [np.linspace(0.0, size[a], lat[a]) for a in range(dim)]
    grids = np.meshgrid(*axes, indexing="ij")
    coords = np.stack([g.ravel(order="F") for g in grids], axis=1)

    # drop unused lattice points (serendipity) and renumber
    used = np.zeros(coords.shape[0], dtype=bool)
    used[elem.ravel()] = True
    if not used.all():
        new_id = -np.ones(coords.shape[0], dtype=np.int64)
        new_id[used] = np.arange(int(used.sum()))
        elem = new_id[elem]
        coords = coords[used]
    return Mesh(elem_type, dim, np.ascontiguousarray(coords, dtype=np.float64),
                np.ascontiguousarray(elem, dtype=np.int32), n_cells, size)


# ----------------------------------------------------------------------------
# Boundary surfaces of the structured box, as lists of face nodes.
# ----------------------------------------------------------------------------

def boundary_nodes(mesh: Mesh, axis: int, side: str, tol: float = 1e-9) -> np.ndarray:
    """Indices of nodes on the box face x_axis = 0 (side='min') or = size (side='max')."""
    target = 0.0 if side == "min" else mesh.size[axis]
    return np.nonzero(np.abs(mesh.coords[:, axis] - target) <= tol * max(1.0, mesh.size[axis]))[0]


def top_faces(mesh: Mesh):
    """Faces of the box face x_dim = size (top), as (kind, node array [n_f][n_fn]).

    kind is the face element type: in 2D 'L1'/'L2' (2- or 3-node edges, the
    3-node order being (end, end, midpoint)); in 3D 'T1'/'T2' (3-/6-node
    triangles, 6-node order (v1,v2,v3,m12,m23,m13)) or 'S1'/'S2' (4-node and
    8-node serendipity squares, corners counter-clockwise then edge mids).
    """
    dim = mesh.dim
    order = 2 if mesh.elem_type in ("P2", "Q2") else 1
    n_cells = mesh.shape
    lat = _lattice(n_cells, order)
    # map from lattice index to node id (identity unless serendipity renumbered)
    full = int(np.prod(lat))
    axes = [np.linspace(0.0, mesh.size[a], lat[a]) for a in range(dim)]
    # build lattice->node map by coordinates (structured, exact)
    steps = [mesh.size[a] / (lat[a] - 1) for a in range(dim)]
    ijk = np.rint(mesh.coords / np.array(steps)).astype(np.int64)
    lat_ids = _lin([ijk[:, a] for a in range(dim)], lat)
    lat2node = -np.ones(full, dtype=np.int64)
    lat2node[lat_ids] = np.arange(mesh.n_nodes)
    del axes
    top = lat[dim - 1] - 1
    if dim == 2:
        i = np.arange(n_cells[0]) * order
        if order == 1:
            faces = np.stack([_lin([i, np.full_like(i, top)], lat),
                              _lin([i + 1, np.full_like(i, top)], lat)], axis=1)
            kind = "L1"
        else:
            faces = np.stack([_lin([i, np.full_like(i, top)], lat),
                              _lin([i + 2, np.full_like(i, top)], lat),
                              _lin([i + 1, np.full_like(i, top)], lat)], axis=1)
            kind = "L2"
        return kind, lat2node[faces]
    # 3D: top face is a structured 2D grid of squares
    gi, gj = np.meshgrid(np.arange(n_cells[0]) * order, np.arange(n_cells[1]) * order, indexing="ij")
    gi, gj = gi.ravel(order="F"), gj.ravel(order="F")
    k = np.full_like(gi, top)

    def L(di, dj):
        return _lin([gi + di, gj + dj, k], lat)

    s = order
    if mesh.elem_type in ("Q1", "Q2"):
        corners = [L(0, 0), L(s, 0), L(s, s), L(0, s)]
        if order == 1:
            return "S1", lat2node[np.stack(corners, axis=1)]
        mids = [L(1, 0), L(2, 1), L(1, 2), L(0, 1)]
        return "S2", lat2node[np.stack(corners + mids, axis=1)]
    # Kuhn split: the top face of each cube is cut along its (0,0)-(1,1) diagonal
    t1 = [L(0, 0), L(s, 0), L(s, s)]
    t2 = [L(0, 0), L(s, s), L(0, s)]
    if order == 1:
        f = np.concatenate([np.stack(t1, axis=1), np.stack(t2, axis=1)], axis=0)
        return "T1", lat2node[f]
    m1 = [L(1, 0), L(2, 1), L(1, 1)]
    m2 = [L(1, 1), L(1, 2), L(0, 1)]
    f = np.concatenate([np.stack(t1 + m1, axis=1), np.stack(t2 + m2, axis=1)], axis=0)
    return "T2", lat2node[f]
