"""Finite element assembly in the paper's sparse-matrix form (plain numpy/scipy, FP64).

Test infrastructure: part of the CPU oracle; never used by the product path.

Follows Sections 6 and 7:
  * Jacobians, determinants, inverses and physical basis gradients at all
    integration points (Section 6.1, eqs. (Jacobian), (Jacobian2),
    (basis_derivative)); integration points are ordered element-major with
    the quadrature index fastest.
  * The sparse strain-displacement matrix B of eq. (local_strain-displ)
    (Section 6.2): 6 rows per point in 3D, 3 rows (e11, e22, 2e12) in 2D;
    DOF index = dim*node + component (the ordering of U(:) in Section 5).
  * WEIGHT = |det J| * w_q (Section 6.3), the block-diagonal D matrices, and
    K_elast = B^T D_elast B (Section 6.3, eq. (K_elast-split)).
  * K_tangent = K_elast + B^T (D_tangent - D_elast) B (eq. (K-split)) and the
    internal forces F = B^T (WEIGHT * S) (Section 7); the one-product form
    K = B^T D_tangent B (Section 9, eq. (K-split_Petr)); and a per-element
    dense sum of G_q^T D_q G_q as an independent route for tiny meshes.
  * Consistent surface loads: integral of the traction times the basis over
    the loaded faces (Section 4, the vector f_k), by face quadrature.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import elements


class Geometry:
    """Quadrature-point geometry of a mesh (Section 6.1)."""

    def __init__(self, coords: np.ndarray, elem: np.ndarray, elem_type: str, dim: int):
        self.dim = dim
        self.elem_type = elem_type
        self.coords = np.asarray(coords, dtype=np.float64)
        self.elem = np.asarray(elem, dtype=np.int64)
        self.n_n = self.coords.shape[0]
        self.n_e, self.n_p = self.elem.shape
        Xi, WF = elements.quadrature(elem_type, dim)
        HatP, DHatP = elements.basis(elem_type, dim, Xi)
        self.Xi, self.WF, self.HatP, self.DHatP = Xi, WF, HatP, DHatP
        self.n_q = WF.size
        self.n_int = self.n_e * self.n_q
        d, n_p, n_q, n_e = dim, self.n_p, self.n_q, self.n_e
        # DHatPhi_i: [n_p][n_int] replicated per element (repmat over elements)
        DHatPhi = np.tile(DHatP, (1, 1, n_e))                   # [d][n_p][n_int]
        # COORDint_j: [n_p][n_int] (coordinates of the element's nodes, repeated per point)
        COORDe = self.coords[self.elem.T]                       # [n_p][n_e][d]
        COORDint = np.repeat(COORDe, n_q, axis=1)               # [n_p][n_int][d]
        # J_ij = sum_p dPhi_p/dxi_i * x_{p,j}
        J = np.einsum("ipq,pqj->ijq", DHatPhi, COORDint)        # [d][d][n_int]
        self.J = J
        self.DET = np.linalg.det(np.moveaxis(J, 2, 0))
        Jinv = np.moveaxis(np.linalg.inv(np.moveaxis(J, 2, 0)), 0, 2)   # [d][d][n_int]
        # physical gradients: DPhi_i = sum_j Jinv_ij DHatPhi_j (eq. (basis_derivative))
        self.DPhi = np.einsum("ijq,jpq->ipq", Jinv, DHatPhi)    # [d][n_p][n_int]
        self.WEIGHT = np.abs(self.DET) * np.tile(WF, n_e)
        self.bad_elements = np.unique(np.nonzero(self.DET <= 0)[0] // n_q)

    @property
    def n_strain(self) -> int:
        return 3 if self.dim == 2 else 6

    def B(self) -> sp.csr_matrix:
        """Sparse strain-displacement matrix (Section 6.2), [n_strain*n_int][dim*n_n]."""
        d, ns, n_int, n_p = self.dim, self.n_strain, self.n_int, self.n_p
        node = np.repeat(self.elem, self.n_q, axis=0)           # [n_int][n_p]
        rows, cols, vals = [], [], []
        base = ns * np.arange(n_int)
        if d == 3:
            # (row, component, derivative direction) of eq. (local_strain-displ)
            pattern = [(0, 0, 0), (1, 1, 1), (2, 2, 2), (3, 0, 1), (3, 1, 0),
                       (4, 1, 2), (4, 2, 1), (5, 0, 2), (5, 2, 0)]
        else:
            pattern = [(0, 0, 0), (1, 1, 1), (2, 0, 1), (2, 1, 0)]
        for p in range(n_p):
            for r, comp, der in pattern:
                rows.append(base + r)
                cols.append(d * node[:, p] + comp)
                vals.append(self.DPhi[der, p, :])
        rows = np.concatenate(rows)
        cols = np.concatenate(cols)
        vals = np.concatenate(vals)
        return sp.csr_matrix((vals, (rows, cols)), shape=(ns * n_int, d * self.n_n))

    def strain(self, B: sp.csr_matrix, u: np.ndarray) -> np.ndarray:
        """E = reshape(B u, n_strain, n_int) (Section 6.2)."""
        return (B @ u).reshape(self.n_int, self.n_strain).T.copy()

    def block_diag(self, DS: np.ndarray, weighted: bool = True) -> sp.csr_matrix:
        """Block-diagonal sparse matrix from per-point blocks DS [ns][ns][n_int] (Section 6.3)."""
        ns, n_int = self.n_strain, self.n_int
        vals = DS * (self.WEIGHT if weighted else 1.0)
        aux = ns * np.arange(n_int)
        i = (aux[None, None, :] + np.arange(ns)[:, None, None]) * np.ones((1, ns, 1), dtype=np.int64)
        j = (aux[None, None, :] + np.arange(ns)[None, :, None]) * np.ones((ns, 1, 1), dtype=np.int64)
        return sp.csr_matrix((vals.ravel(), (i.ravel(), j.ravel())), shape=(ns * n_int, ns * n_int))


class Assembler:
    """Holds B, D_elast and K_elast of a mesh, as the paper's elastic_stiffness_matrix does."""

    def __init__(self, geom: Geometry, DS_elast_in: np.ndarray):
        self.geom = geom
        self.B = geom.B()
        self.BT = self.B.T.tocsr()
        n_int = geom.n_int
        DS = np.repeat(DS_elast_in[:, :, None], n_int, axis=2)
        self.D_elast = geom.block_diag(DS)
        self.K_elast = (self.BT @ self.D_elast @ self.B).tocsr()

    def tangent_split(self, DS_in: np.ndarray) -> sp.csr_matrix:
        """K_tangent = K_elast + B^T (D_tangent - D_elast) B (eq. (K-split))."""
        D_t = self.geom.block_diag(DS_in)
        return (self.K_elast + self.BT @ (D_t - self.D_elast) @ self.B).tocsr()

    def tangent_full(self, DS_in: np.ndarray) -> sp.csr_matrix:
        """K_tangent = B^T D_tangent B (eq. (K-split_Petr))."""
        return (self.BT @ self.geom.block_diag(DS_in) @ self.B).tocsr()

    def internal_force(self, S_in: np.ndarray) -> np.ndarray:
        """F = B^T reshape(S .* WEIGHT) (Section 7)."""
        return self.BT @ (S_in * self.geom.WEIGHT).T.ravel()


def element_matrices_bruteforce(geom: Geometry, DS_in: np.ndarray) -> np.ndarray:
    """Dense local matrices K_e = sum_q w_q G_q^T D_q G_q, [n_e][d n_p][d n_p] (loops).

    G_q is the local matrix of eq. (local_strain-displ) built entry by entry.
    """
    d, n_p, n_q = geom.dim, geom.n_p, geom.n_q
    ns = geom.n_strain
    Ke = np.zeros((geom.n_e, d * n_p, d * n_p))
    for e in range(geom.n_e):
        for q in range(n_q):
            ip = e * n_q + q
            Gm = np.zeros((ns, d * n_p))
            for p in range(n_p):
                g = geom.DPhi[:, p, ip]
                if d == 3:
                    Gm[0, 3 * p] = g[0]
                    Gm[1, 3 * p + 1] = g[1]
                    Gm[2, 3 * p + 2] = g[2]
                    Gm[3, 3 * p], Gm[3, 3 * p + 1] = g[1], g[0]
                    Gm[4, 3 * p + 1], Gm[4, 3 * p + 2] = g[2], g[1]
                    Gm[5, 3 * p], Gm[5, 3 * p + 2] = g[2], g[0]
                else:
                    Gm[0, 2 * p] = g[0]
                    Gm[1, 2 * p + 1] = g[1]
                    Gm[2, 2 * p], Gm[2, 2 * p + 1] = g[1], g[0]
            Ke[e] += geom.WEIGHT[ip] * Gm.T @ DS_in[:, :, ip] @ Gm
    return Ke


def scatter_elements(geom: Geometry, Ke: np.ndarray) -> sp.csr_matrix:
    """Global matrix from local matrices by explicit index scatter."""
    d = geom.dim
    dofs = (d * geom.elem[:, :, None] + np.arange(d)[None, None, :]).reshape(geom.n_e, -1)
    i = np.repeat(dofs[:, :, None], dofs.shape[1], axis=2)
    j = np.repeat(dofs[:, None, :], dofs.shape[1], axis=1)
    return sp.csr_matrix((Ke.ravel(), (i.ravel(), j.ravel())), shape=(d * geom.n_n, d * geom.n_n))


# ----------------------------------------------------------------------------
# Surface loads (vector f_k of Section 4), by quadrature on boundary faces
# ----------------------------------------------------------------------------

# local faces per element: (face kind, local node indices)
LOCAL_FACES = {
    ("P1", 2): ("L1", [(0, 1), (1, 2), (2, 0)]),
    ("P2", 2): ("L2", [(0, 1, 3), (1, 2, 4), (2, 0, 5)]),
    ("Q1", 2): ("L1", [(0, 1), (1, 2), (2, 3), (3, 0)]),
    ("Q2", 2): ("L2", [(0, 1, 4), (1, 2, 5), (2, 3, 6), (3, 0, 7)]),
    ("P1", 3): ("T1", [(0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3)]),
    ("P2", 3): ("T2", [(0, 1, 2, 4, 5, 6), (0, 1, 3, 4, 7, 9), (1, 2, 3, 5, 8, 7), (0, 2, 3, 6, 8, 9)]),
    ("Q1", 3): ("S1", [(0, 1, 2, 3), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7)]),
    ("Q2", 3): ("S2", [(0, 1, 2, 3, 8, 9, 10, 11), (4, 5, 6, 7, 12, 13, 14, 15),
                       (0, 1, 5, 4, 8, 17, 12, 16), (1, 2, 6, 5, 9, 18, 13, 17),
                       (2, 3, 7, 6, 10, 19, 14, 18), (3, 0, 4, 7, 11, 16, 15, 19)]),
}


def surface_load(coords, elem, elem_type, dim, on_face, traction) -> np.ndarray:
    """f_j = int_{Gamma} t . Phi_j ds over element faces whose nodes all satisfy on_face(x)."""
    coords = np.asarray(coords, dtype=np.float64)
    kind, faces = LOCAL_FACES[(elem_type, dim)]
    fb, pts, w = elements.face_rule(kind)
    P, dP = fb(pts)                                    # [n_fn][n_qs], [dim-1][n_fn][n_qs]
    f = np.zeros((coords.shape[0], dim))
    t = np.asarray(traction, dtype=np.float64)
    for loc in faces:
        fn = np.asarray(elem)[:, list(loc)]            # [n_e][n_fn]
        X = coords[fn]                                 # [n_e][n_fn][dim]
        sel = np.all(on_face(X.reshape(-1, dim)).reshape(fn.shape), axis=1)
        if not sel.any():
            continue
        X = X[sel]
        T = np.einsum("kfq,efd->ekdq", dP, X)          # tangents [n_sel][dim-1][dim][n_qs]
        if dim == 2:
            jac = np.sqrt(np.sum(T[:, 0] ** 2, axis=1))
        else:
            cr = np.cross(T[:, 0], T[:, 1], axis=1)
            jac = np.sqrt(np.sum(cr ** 2, axis=1))
        contrib = np.einsum("fq,eq,q->ef", P, jac, w)  # integral of Phi_f over each face
        for a in range(dim):
            np.add.at(f[:, a], fn[sel].ravel(), (contrib * t[a]).ravel())
    return f.ravel()
