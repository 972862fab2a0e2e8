"""Semismooth Newton method and load path (plain numpy/scipy, FP64).

Test infrastructure: part of the CPU oracle; never used by the product path.

Algorithm ALG-NEWTON (Section 4): start from an initial iterate carrying the
Dirichlet values of step k, solve K(u) du = f_k - F(u) on the free DOFs
(eq. (lin_syst), the restriction K(Q,Q) of Section 5) by a sparse direct
solver, update u, and stop.  Readings where the paper leaves a choice:
  * stopping test: ||(f_k - F(u))_free||_2 <= tol * max(||f_free||_2, ||F(u)||_2)
    (the energy-norm increment of ALG-NEWTON is computed and logged too);
  * initial iterate: 'previous' = the last converged u with the new Dirichlet
    values (ALG-NEWTON's u_{D,k} extended by the last solution), or
    'extrapolate' = u_{k-1} + (dzeta_k/dzeta_{k-1}) (u_{k-1} - u_{k-2}) with the
    new Dirichlet values, used only while the load keeps its direction
    (dzeta_k/dzeta_{k-1} > 0); a step that does not converge from the
    extrapolated start is solved again from the 'previous' one;
  * after convergence the trial internal variables of the last constitutive
    evaluation become the state of step k (Sections 2.1, 7.1, 7.2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse.linalg as spla

from . import constitutive as C
from .fem import Assembler, Geometry


@dataclass
class StepReport:
    newton_its: int
    rel_resid: float
    n_plastic: int
    resid_history: list = field(default_factory=list)
    energy_increments: list = field(default_factory=list)
    converged: bool = True


class OracleSolver:
    """Incremental elastoplastic solver on one mesh."""

    def __init__(self, problem, split: bool = True):
        self.p = problem
        m = problem.mesh
        self.dim = m.dim
        self.geom = Geometry(m.coords, m.elem, m.elem_type, m.dim)
        K, G = C.moduli(problem.material.E, problem.material.nu)
        De = C.elastic_tangent(K, G)
        if self.dim == 2:
            De = De[np.ix_(C.PLANE_INPLANE_IDX, C.PLANE_INPLANE_IDX)]
        self.asm = Assembler(self.geom, De)
        self.split = split
        nc = C.n_comp(self.dim)
        self.ep = np.zeros((nc, self.geom.n_int))
        self.hard = (np.zeros((nc, self.geom.n_int)) if problem.material.model == 1
                     else np.zeros(self.geom.n_int))
        self.stress = np.zeros((nc, self.geom.n_int))
        self.plastic = np.zeros(self.geom.n_int, dtype=np.int8)
        self.free = problem.dirichlet == 0
        self.u = np.zeros(problem.n_dof)
        self.u_prev = None
        self.zeta_done = []

    # -- one evaluation of T_k, F and K at u --------------------------------
    def evaluate(self, u, need_K=True):
        E = self.geom.strain(self.asm.B, u)
        res = C.constitutive(self.p.material, self.dim, E, self.ep, self.hard)
        F = self.asm.internal_force(res["S_in"])
        K = None
        if need_K:
            K = self.asm.tangent_split(res["DS_in"]) if self.split else self.asm.tangent_full(res["DS_in"])
        return res, F, K

    def energy_norm(self, v):
        return math.sqrt(max(0.0, float(v @ (self.asm.K_elast @ v))))

    def start_iterate(self, zeta, mode="extrapolate"):
        u = self.u.copy()
        if mode == "extrapolate" and self.u_prev is not None and len(self.zeta_done) >= 2:
            dz_prev = self.zeta_done[-1] - self.zeta_done[-2]
            dz = zeta - self.zeta_done[-1]
            if dz_prev != 0.0 and dz / dz_prev > 0.0:
                u = self.u + (dz / dz_prev) * (self.u - self.u_prev)
        fixed = ~self.free
        u[fixed] = zeta * self.p.u_D_unit[fixed]
        return u

    def solve_step(self, zeta, tol=None, maxit=50, mode="extrapolate") -> StepReport:
        rep = self._newton(zeta, tol, maxit, mode)
        if not rep[-1].converged and mode == "extrapolate":
            rep = self._newton(zeta, tol, maxit, "previous")
        u, res, report = rep
        # commit (state of step k)
        self.u_prev, self.u = self.u, u
        self.zeta_done.append(zeta)
        self.ep, self.hard = res["ep"], res["hard"]
        self.stress, self.plastic = res["S"], res["plastic"]
        return report

    def _newton(self, zeta, tol, maxit, mode):
        tol = self.p.newton_rtol if tol is None else tol
        f = zeta * self.p.f_unit
        u = self.start_iterate(zeta, mode)
        Q = self.free
        hist, einc = [], []
        converged = False
        it = 0
        while True:
            res, F, K = self.evaluate(u, need_K=True)
            if np.any(res["err"]):
                raise FloatingPointError("return mapping has no admissible stress (apex, K eta eta_bar + Hc = 0)")
            r = (f - F)[Q]
            scale = max(np.linalg.norm(f[Q]), np.linalg.norm(F))
            rel = np.linalg.norm(r) / scale if scale > 0 else np.linalg.norm(r)
            hist.append(rel)
            if rel <= tol:
                converged = True
                break
            if it >= maxit:
                break
            KQ = K[Q][:, Q].tocsc()
            du = np.zeros_like(u)
            du[Q] = spla.splu(KQ).solve(r)
            u_old = u
            u = u + du
            einc.append(self.energy_norm(du) / max(self.energy_norm(u_old) + self.energy_norm(u), 1e-300))
            it += 1
        return u, res, StepReport(it, hist[-1], int(np.count_nonzero(res["plastic"])), hist, einc, converged)

    def solve_path(self, zetas=None, **kw):
        zetas = self.p.zeta if zetas is None else zetas
        return [self.solve_step(float(z), **kw) for z in zetas]


def homogeneous_column(material, t_values, tol=1e-14, maxit=60):
    """One material point of the plane-strain column: sigma_xx = 0, sigma_yy = -t, e33 = 0.

    Unknowns (e11, e22) with 2e12 = 0.  Newton on the 2x2 block of the tangent,
    with the state carried from one load value to the next.  Returns per-load
    (strain [3], stored stress [4], plastic strain [4], hardening, plastic flag).
    """
    dim = 2
    nc = 4
    ep = np.zeros((nc, 1))
    hard = np.zeros((nc, 1)) if material.model == 1 else np.zeros(1)
    e = np.zeros(2)
    out = []
    for t in t_values:
        target = np.array([0.0, -t])
        for _ in range(maxit):
            E = np.array([[e[0]], [e[1]], [0.0]])
            res = C.constitutive(material, dim, E, ep, hard)
            s = res["S_in"][:2, 0]
            r = target - s
            if np.linalg.norm(r) <= tol * max(abs(t), 1.0):
                break
            D = res["DS_in"][:2, :2, 0]
            e = e + np.linalg.solve(D, r)
        E = np.array([[e[0]], [e[1]], [0.0]])
        res = C.constitutive(material, dim, E, ep, hard)
        ep, hard = res["ep"], res["hard"]
        out.append(dict(strain=E[:, 0].copy(), stress=res["S"][:, 0].copy(), ep=ep[:, 0].copy(),
                        hard=np.array(hard, copy=True).ravel(), plastic=int(res["plastic"][0])))
    return out
