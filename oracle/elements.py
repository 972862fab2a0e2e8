"""Reference elements, basis functions and quadrature rules (plain numpy, FP64).

Test infrastructure: part of the CPU oracle; never used by the product path.

3D elements follow the paper's Appendix ("P1 and P2 tetrahedral elements",
"Q1 and Q2 hexahedral elements"): reference nodes, basis functions and the
quadrature rules named there.  The paper states the 2D elements only as the
plane reduction of these (Section 1); the 2D tables below are the standard
plane analogues (P1/P2 triangles with midpoints ordered 12, 23, 13; 4-node
Q1 and 8-node serendipity Q2 quadrilaterals on [-1,1]^2).

The 11-point tetrahedral rule is printed in the Appendix with truncated
digits; the exact values used here are w1 = -74/5625, w2..5 = 343/45000,
w6..11 = 56/2250 and abscissae 1/14, 11/14, (1 +- sqrt(5/14))/4.  The P2
triangle uses the 7-point degree-5 rule.

Every function returns arrays indexed [p][q] (basis p at point q) in the
layout of the paper's `local_basis_volume` (Section 6).
"""
from __future__ import annotations

import math

import numpy as np


def quadrature(elem: str, dim: int):
    """Quadrature points Xi [dim][n_q] and weights WF [n_q] (Appendix; eq. (quadrature))."""
    if dim == 3:
        if elem == "P1":
            return np.full((3, 1), 0.25), np.array([1.0 / 6.0])
        if elem == "P2":
            a, b = 1.0 / 14.0, 11.0 / 14.0
            s = math.sqrt(5.0 / 14.0)
            c, d = (1.0 + s) / 4.0, (1.0 - s) / 4.0
            pts = [(0.25, 0.25, 0.25), (a, a, a), (b, a, a), (a, b, a), (a, a, b),
                   (c, d, d), (d, c, d), (d, d, c), (c, c, d), (c, d, c), (d, c, c)]
            w = [-74.0 / 5625.0] + [343.0 / 45000.0] * 4 + [56.0 / 2250.0] * 6
            return np.array(pts).T.copy(), np.array(w)
        if elem in ("Q1", "Q2"):
            g, gw = _gauss_1d(2 if elem == "Q1" else 3)
            pts, w = [], []
            # xi_1 fastest
            for k in range(len(g)):
                for j in range(len(g)):
                    for i in range(len(g)):
                        pts.append((g[i], g[j], g[k]))
                        w.append(gw[i] * gw[j] * gw[k])
            return np.array(pts).T.copy(), np.array(w)
    if dim == 2:
        if elem == "P1":
            return np.full((2, 1), 1.0 / 3.0), np.array([0.5])
        if elem == "P2":
            r = math.sqrt(15.0)
            a1, b1 = (6.0 - r) / 21.0, (9.0 + 2.0 * r) / 21.0
            a2, b2 = (6.0 + r) / 21.0, (9.0 - 2.0 * r) / 21.0
            w1, w2 = (155.0 - r) / 2400.0, (155.0 + r) / 2400.0
            pts = [(1.0 / 3.0, 1.0 / 3.0),
                   (a1, a1), (b1, a1), (a1, b1),
                   (a2, a2), (b2, a2), (a2, b2)]
            w = [9.0 / 80.0] + [w1] * 3 + [w2] * 3
            return np.array(pts).T.copy(), np.array(w)
        if elem in ("Q1", "Q2"):
            g, gw = _gauss_1d(2 if elem == "Q1" else 3)
            pts, w = [], []
            for j in range(len(g)):
                for i in range(len(g)):
                    pts.append((g[i], g[j]))
                    w.append(gw[i] * gw[j])
            return np.array(pts).T.copy(), np.array(w)
    raise ValueError(f"unsupported element {elem} in {dim}D")


def _gauss_1d(n: int):
    """Gauss-Legendre points on [-1,1]: +-1/sqrt(3) (weights 1) or 0, +-sqrt(3/5) (8/9, 5/9)."""
    if n == 2:
        g = 1.0 / math.sqrt(3.0)
        return [-g, g], [1.0, 1.0]
    if n == 3:
        g = math.sqrt(3.0 / 5.0)
        return [-g, 0.0, g], [5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0]
    raise ValueError(n)


def nodes(elem: str, dim: int) -> np.ndarray:
    """Reference nodes N_p as [n_p][dim] (Appendix)."""
    if dim == 3:
        tet = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
        if elem == "P1":
            return np.array(tet, dtype=float)
        if elem == "P2":
            mids = [(.5, 0, 0), (.5, .5, 0), (0, .5, 0), (.5, 0, .5), (0, .5, .5), (0, 0, .5)]
            return np.array(tet + mids, dtype=float)
        hexc = [(-1, -1, -1), (1, -1, -1), (1, 1, -1), (-1, 1, -1),
                (-1, -1, 1), (1, -1, 1), (1, 1, 1), (-1, 1, 1)]
        if elem == "Q1":
            return np.array(hexc, dtype=float)
        if elem == "Q2":
            mids = [(0, -1, -1), (1, 0, -1), (0, 1, -1), (-1, 0, -1),
                    (0, -1, 1), (1, 0, 1), (0, 1, 1), (-1, 0, 1),
                    (-1, -1, 0), (1, -1, 0), (1, 1, 0), (-1, 1, 0)]
            return np.array(hexc + mids, dtype=float)
    if dim == 2:
        tri = [(0, 0), (1, 0), (0, 1)]
        if elem == "P1":
            return np.array(tri, dtype=float)
        if elem == "P2":
            return np.array(tri + [(.5, 0), (.5, .5), (0, .5)], dtype=float)
        quad = [(-1, -1), (1, -1), (1, 1), (-1, 1)]
        if elem == "Q1":
            return np.array(quad, dtype=float)
        if elem == "Q2":
            return np.array(quad + [(0, -1), (1, 0), (0, 1), (-1, 0)], dtype=float)
    raise ValueError(f"unsupported element {elem} in {dim}D")


def basis(elem: str, dim: int, Xi: np.ndarray):
    """Basis values HatP [n_p][n_q] and gradients DHatP [dim][n_p][n_q] at points Xi [dim][n_q].

    Counterpart of `local_basis_volume` (Section 6): DHatP[i] holds
    d(hat Phi_p)/d(xi_{i+1}) at the points.
    """
    Xi = np.asarray(Xi, dtype=float)
    if dim == 3:
        x1, x2, x3 = Xi
        if elem == "P1":
            x0 = 1.0 - x1 - x2 - x3
            P = np.array([x0, x1, x2, x3])
            o, z = np.ones_like(x1), np.zeros_like(x1)
            D1 = np.array([-o, o, z, z])
            D2 = np.array([-o, z, o, z])
            D3 = np.array([-o, z, z, o])
            return P, np.array([D1, D2, D3])
        if elem == "P2":
            x0 = 1.0 - x1 - x2 - x3
            P = np.array([x0 * (2 * x0 - 1), x1 * (2 * x1 - 1), x2 * (2 * x2 - 1), x3 * (2 * x3 - 1),
                          4 * x0 * x1, 4 * x1 * x2, 4 * x0 * x2, 4 * x1 * x3, 4 * x2 * x3, 4 * x0 * x3])
            # derivatives via barycentric chain rule: d x0 / d xi_i = -1
            z = np.zeros_like(x1)
            d0 = -(4 * x0 - 1)
            D = []
            for i, xi in enumerate((x1, x2, x3)):
                e = [z, z, z]
                e[i] = 4 * xi - 1
                dvert = [d0, e[0], e[1], e[2]]
                # d/dxi_i of 4*a*b with a,b in (x0,x1,x2,x3); dx0 = -1, dxk = delta_ik
                bary = (x0, x1, x2, x3)
                dbar = [-np.ones_like(x1)] + [np.ones_like(x1) if k == i else z for k in range(3)]
                pairs = [(0, 1), (1, 2), (0, 2), (1, 3), (2, 3), (0, 3)]
                dmid = [4 * (dbar[a] * bary[b] + bary[a] * dbar[b]) for a, b in pairs]
                D.append(np.array(dvert + dmid))
            return P, np.array(D)
        if elem == "Q1":
            N = nodes("Q1", 3)
            P, D = [], [[], [], []]
            for a, b, c in N:
                f1, f2, f3 = 1 + a * x1, 1 + b * x2, 1 + c * x3
                P.append(f1 * f2 * f3 / 8)
                D[0].append(a * f2 * f3 / 8)
                D[1].append(b * f1 * f3 / 8)
                D[2].append(c * f1 * f2 / 8)
            return np.array(P), np.array(D)
        if elem == "Q2":
            N = nodes("Q2", 3)
            P, D = [], [[], [], []]
            for a, b, c in N[:8]:
                f1, f2, f3 = 1 + a * x1, 1 + b * x2, 1 + c * x3
                g = -2 + a * x1 + b * x2 + c * x3
                P.append(f1 * f2 * f3 * g / 8)
                D[0].append(a * f2 * f3 * (g + f1) / 8)
                D[1].append(b * f1 * f3 * (g + f2) / 8)
                D[2].append(c * f1 * f2 * (g + f3) / 8)
            for a, b, c in N[8:]:
                # one coordinate is 0 (bubble direction), the others +-1
                if a == 0:
                    q, dq = 1 - x1 * x1, -2 * x1
                    f2, f3 = 1 + b * x2, 1 + c * x3
                    P.append(q * f2 * f3 / 4)
                    D[0].append(dq * f2 * f3 / 4)
                    D[1].append(q * b * f3 / 4)
                    D[2].append(q * f2 * c / 4)
                elif b == 0:
                    q, dq = 1 - x2 * x2, -2 * x2
                    f1, f3 = 1 + a * x1, 1 + c * x3
                    P.append(f1 * q * f3 / 4)
                    D[0].append(a * q * f3 / 4)
                    D[1].append(f1 * dq * f3 / 4)
                    D[2].append(f1 * q * c / 4)
                else:
                    q, dq = 1 - x3 * x3, -2 * x3
                    f1, f2 = 1 + a * x1, 1 + b * x2
                    P.append(f1 * f2 * q / 4)
                    D[0].append(a * f2 * q / 4)
                    D[1].append(f1 * b * q / 4)
                    D[2].append(f1 * f2 * dq / 4)
            return np.array(P), np.array(D)
    if dim == 2:
        x1, x2 = Xi
        if elem == "P1":
            o, z = np.ones_like(x1), np.zeros_like(x1)
            return (np.array([1 - x1 - x2, x1, x2]),
                    np.array([[-o, o, z], [-o, z, o]]))
        if elem == "P2":
            x0 = 1 - x1 - x2
            P = np.array([x0 * (2 * x0 - 1), x1 * (2 * x1 - 1), x2 * (2 * x2 - 1),
                          4 * x0 * x1, 4 * x1 * x2, 4 * x0 * x2])
            z = np.zeros_like(x1)
            D1 = np.array([-(4 * x0 - 1), 4 * x1 - 1, z, 4 * (x0 - x1), 4 * x2, -4 * x2])
            D2 = np.array([-(4 * x0 - 1), z, 4 * x2 - 1, -4 * x1, 4 * x1, 4 * (x0 - x2)])
            return P, np.array([D1, D2])
        if elem == "Q1":
            N = nodes("Q1", 2)
            P, D = [], [[], []]
            for a, b in N:
                f1, f2 = 1 + a * x1, 1 + b * x2
                P.append(f1 * f2 / 4)
                D[0].append(a * f2 / 4)
                D[1].append(b * f1 / 4)
            return np.array(P), np.array(D)
        if elem == "Q2":
            N = nodes("Q2", 2)
            P, D = [], [[], []]
            for a, b in N[:4]:
                f1, f2 = 1 + a * x1, 1 + b * x2
                g = -1 + a * x1 + b * x2
                P.append(f1 * f2 * g / 4)
                D[0].append(a * f2 * (g + f1) / 4)
                D[1].append(b * f1 * (g + f2) / 4)
            for a, b in N[4:]:
                if a == 0:
                    q, dq = 1 - x1 * x1, -2 * x1
                    f2 = 1 + b * x2
                    P.append(q * f2 / 2)
                    D[0].append(dq * f2 / 2)
                    D[1].append(q * b / 2)
                else:
                    q, dq = 1 - x2 * x2, -2 * x2
                    f1 = 1 + a * x1
                    P.append(f1 * q / 2)
                    D[0].append(a * q / 2)
                    D[1].append(f1 * dq / 2)
            return np.array(P), np.array(D)
    raise ValueError(f"unsupported element {elem} in {dim}D")


# ----------------------------------------------------------------------------
# Face (boundary) elements, for surface loads (Section 4, the vector f_k)
# ----------------------------------------------------------------------------

def face_rule(kind: str):
    """Reference face element for surface integrals: (basis(s) -> (P, dP), points, weights).

    kinds: 'L1','L2' edges on [-1,1] with nodes (-1, 1[, 0]); 'T1','T2' triangles
    (P1/P2 triangle tables above); 'S1','S2' squares (Q1/Q2 quadrilateral tables).
    """
    if kind in ("L1", "L2"):
        g = math.sqrt(3.0 / 5.0)
        pts = np.array([[-g, 0.0, g]])
        w = np.array([5 / 9, 8 / 9, 5 / 9])

        def fb(s):
            s = s[0]
            if kind == "L1":
                return np.array([(1 - s) / 2, (1 + s) / 2]), np.array([[-0.5 + 0 * s, 0.5 + 0 * s]])
            return (np.array([s * (s - 1) / 2, s * (s + 1) / 2, 1 - s * s]),
                    np.array([[s - 0.5, s + 0.5, -2 * s]]))
        return fb, pts, w
    fam = {"T1": "P1", "T2": "P2", "S1": "Q1", "S2": "Q2"}[kind]
    pts, w = quadrature("P2" if fam in ("P1", "P2") else "Q2", 2)
    return (lambda s: basis(fam, 2, s)), pts, w
