"""Shared helpers for the GPU parity tests: building inputs and oracle references."""
from __future__ import annotations

import math

import numpy as np

from oracle import constitutive as OC
from oracle.fem import Assembler, Geometry
from synthetic import DP, ELASTIC, VM_ISO, VM_KIN, Material, generic_box
from synthetic.random_states import random_displacement, random_state

ALL_ELEMS = [(e, d) for d in (2, 3) for e in ("P1", "P2", "Q1", "Q2")]
E_MOD, NU = 206900.0, 0.29
Y_VM = 450.0 * math.sqrt(2.0 / 3.0)


def material(model: int, dim: int = 2) -> Material:
    if model == ELASTIC:
        return Material(ELASTIC, E=E_MOD, nu=NU)
    if model == VM_KIN:
        return Material(VM_KIN, E=E_MOD, nu=NU, Y=Y_VM, H=1e4)
    if model == VM_ISO:
        return Material(VM_ISO, E=E_MOD, nu=NU, Y=Y_VM, H=1e4)
    return Material(DP, E=E_MOD, nu=NU, c0=450.0, phi=math.radians(30.0), psi=math.radians(10.0), Hc=1e3)


def small_problem(elem: str, dim: int, n: int, model: int, perturb: float = 0.1, seed: int = 0):
    p = generic_box(elem, dim, n, material(model, dim), t_max=300.0, n_steps=4)
    if elem == "P2" and dim == 3:
        perturb = min(perturb, 0.03)    # Kuhn tetrahedra are thin: larger moves invert curved P2 tets
    if perturb:
        m = p.mesh
        g = np.random.default_rng(seed)
        h = 10.0 / n
        inner = np.all((m.coords > 1e-9) & (m.coords < 10 - 1e-9), axis=1)
        m.coords[inner] += g.uniform(-perturb * h, perturb * h, (int(inner.sum()), dim))
        assert Geometry(m.coords, m.elem, elem, dim).DET.min() > 0, "perturbed test mesh is inverted"
    return p


def fed_iterate(problem, seed: int, strain_scale: float = 2.5e-3, dilate: float = 0.0):
    """(u, ep, hard) giving a mix of elastic and plastic points."""
    m = problem.mesh
    dim = m.dim
    nc = OC.n_comp(dim)
    g = Geometry(m.coords, m.elem, m.elem_type, dim)
    u = random_displacement(m.coords, problem.dirichlet, strain_scale * 10.0 / max(m.shape), seed,
                            affine=max(m.shape) * 0.1)
    u = u + dilate * m.coords.ravel() * (1 - problem.dirichlet)
    ep_, alpha = random_state(g.n_int, nc, 3e-4, seed + 1, hard_scale=1e-3)
    if dim == 2:
        ep_[3] = 0.0 * ep_[3] + np.random.default_rng(seed + 2).standard_normal(g.n_int) * 1e-4
    if problem.material.model == VM_KIN:
        beta6 = OC.DEV @ OC.embed_state(np.random.default_rng(seed + 3).standard_normal((nc, g.n_int)) * 40.0, dim)
        hard = OC.extract_state(beta6, dim)
    else:
        hard = alpha
    return u, ep_, hard


def oracle_eval(problem, u, ep_, hard, split=True):
    m = problem.mesh
    dim = m.dim
    g = Geometry(m.coords, m.elem, m.elem_type, dim)
    K, G = OC.moduli(problem.material.E, problem.material.nu)
    De = OC.elastic_tangent(K, G)
    if dim == 2:
        De = De[np.ix_(OC.PLANE_INPLANE_IDX, OC.PLANE_INPLANE_IDX)]
    asm = Assembler(g, De)
    E = g.strain(asm.B, u)
    res = OC.constitutive(problem.material, dim, E, ep_, hard)
    F = asm.internal_force(res["S_in"])
    Kt = asm.tangent_split(res["DS_in"]) if split else asm.tangent_full(res["DS_in"])
    return dict(geom=g, asm=asm, res=res, F=F, K=Kt, E=E)


def rel_fro(A, B):
    d = A - B
    num = math.sqrt(float(d.multiply(d).sum())) if hasattr(d, "multiply") else float(np.linalg.norm(d))
    den = math.sqrt(float(B.multiply(B).sum())) if hasattr(B, "multiply") else float(np.linalg.norm(B))
    return num / den if den > 0 else num


def rel_max(a, b):
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / den) if den > 0 else float(np.abs(a - b).max())
