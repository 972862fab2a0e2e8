"""Host-side load-stepping drivers for the paper's validation experiments (Section 8).

Everything is computed through the C ABI (ep_solve_load_path, ep_get); these
functions only choose the next load factor and read results back:

* footing_pressure: average pressure under a strip footing, from the reaction
  forces (the internal forces F = B^T(W S) at the prescribed footing DOFs).
* strip_footing_path: the displacement-controlled path of the strip-footing
  benchmark (Section 8.3) with the paper's adaptive increment: start with
  du = 0.001 and double it when the pressure has stopped growing.  The paper
  does not quantify "the pressure increment is sufficiently small"; here it is
  when the secant slope dp/du of the last step fell below 1/10 of the first
  step's (elastic) slope.  A step whose (undamped) Newton iteration fails is
  retried with half the increment (the failed step leaves the last converged
  state in place); the paper's method has no damping for large increments.
* external_work: f_max^T u_k, the ordinate of the hysteresis curve of the
  cyclic von Mises experiment (Section 8.2).
* autotune: picks the fastest solver schedule (precision, Krylov method,
  preconditioner) and then the fastest kernel schedule (assembly tile size,
  graph-replayed or directly launched Krylov iterations) for a context by
  timing each on the first load steps and restoring the state in between (the
  paper uses one direct solver; the schedule is this implementation's choice,
  Section 5's linear systems).
* sparse_lu_solve: one solve with the sparse LU on the benchmark mesh's elastic
  tangent (for timing and profiling its kernels outside a load path).
"""
from __future__ import annotations

import numpy as np

from . import ep


def footing_pressure(ctx, problem) -> float:
    """Average pressure under the footing: -(sum of the vertical reactions) / footing width."""
    F = ctx.get(ep.EP_F_INT).reshape(-1, ctx.dim)
    nodes = problem.extra["footing_nodes"]
    return float(-F[nodes, ctx.dim - 1].sum() / problem.extra["footing"])


def strip_footing_path(ctx, problem, u_max: float = 1.0, du0: float = 1e-3, soft: float = 0.1,
                       max_steps: int = 400, opts=None, du_min: float = 1e-6):
    """Adaptive displacement path of the strip footing; returns (u_D values, pressures, reports)."""
    opts = opts or ep.default_opts()
    u, du = 0.0, du0
    us, ps, reps = [], [], []
    slope0 = None
    p_prev = 0.0
    for _ in range(max_steps):
        if u >= u_max - 1e-12:
            break
        step = min(du, u_max - u)
        st, r = ctx.solve_load_path(np.array([u + step]), opts, raise_on_error=False)
        if st != ep.EP_OK:
            if step / 2.0 < du_min:
                raise ep.EPError(st, ep.lib().ep_last_error(ctx.h).decode())
            du = step / 2.0
            continue
        u += step
        p = footing_pressure(ctx, problem)
        slope = (p - p_prev) / step
        if slope0 is None:
            slope0 = slope
        elif slope < soft * slope0:
            du *= 2.0
        us.append(u)
        ps.append(p)
        reps.extend(r)
        p_prev = p
    return np.array(us), np.array(ps), reps


def external_work(ctx, problem) -> float:
    """f_max^T u_k with f_max the traction load at zeta = 1."""
    return float(problem.f_unit @ ctx.get(ep.EP_U))


# -- schedule autotuner ---------------------------------------------------------------------------
STATE_FIELDS = (ep.EP_U, ep.EP_PLASTIC_STRAIN, ep.EP_HARDENING, ep.EP_STRESS, ep.EP_PLASTIC_FLAG)


def schedule_candidates(symmetric: bool, base=None):
    """Solver schedules to try: precision x (Krylov method, preconditioner).  CG only for a symmetric
    tangent (von Mises, associated Drucker-Prager); GMRES and BiCGStab otherwise; block Jacobi and
    the AMG V-cycle as preconditioners.  Returns a list of dicts of ep_opts fields."""
    methods = [1, 3] if symmetric else [3, 2]
    out = []
    for prec in (ep.EP_FP64, ep.EP_MIXED):
        for m in methods:
            for pc in (2, 1):
                d = dict(base or {})
                d.update(precision=prec, krylov=m, precond=pc)
                out.append(d)
    return out


def kernel_schedule_candidates(solver_schedule):
    """Kernel schedules for a chosen solver schedule: the assembly tile (the element type's elements
    per CTA, or half of them: less shared memory per CTA, more CTAs per SM) x the launch form of the
    GMRES iterations (replayed CUDA graphs, or direct launches)."""
    out = []
    for tile in (1, 2):
        for graphs in (1, 0):
            d = dict(solver_schedule)
            d.update(asm_tile=tile, krylov_graphs=graphs)
            out.append(d)
    return out


def autotune(ctx, zeta, trial_steps: int = 3, candidates=None, base_opts=None, kernel_schedules: bool = True):
    """Time each candidate schedule on the first `trial_steps` load steps from the context's current
    state, restoring that state after every trial; returns (best opts, [(candidate, seconds or None)]).

    Two stages: the solver schedules (precision x Krylov method x preconditioner), then, on the
    fastest of them, the kernel schedules (assembly tile x graph-replayed or direct Krylov launches,
    kernel_schedule_candidates).  The time of a trial is the sum of its steps' t_step_ms (set-up work
    done once per context, such as the AMG hierarchy, is outside the steps).  A candidate whose trial
    fails is skipped; the trial paths of the others converge to the same tolerance, so their
    solutions agree."""
    import numpy as np
    base = dict(newton_rtol=1e-10) if base_opts is None else dict(base_opts)
    if candidates is None:
        sym = int(ctx.material.model) != ep.EP_DP or (ctx.material.phi == ctx.material.psi and ctx.material.Hc == 0.0)
        candidates = schedule_candidates(sym, base)
    saved = {f: ctx.get(f).copy() for f in STATE_FIELDS}
    z = np.asarray(zeta, dtype=np.float64)[:max(1, trial_steps)]
    results = []

    def trial(cand):
        opts = ep.default_opts(**cand)
        st, reps = ctx.solve_load_path(z, opts, raise_on_error=False)
        t = sum(r.t_step_ms for r in reps) / 1e3 if st == ep.EP_OK else None
        results.append((cand, t))
        for f, v in saved.items():
            ctx.set(f, v)
        return t

    for cand in candidates:
        trial(cand)
    ok = [(c, t) for c, t in results if t is not None]
    if not ok:
        raise ep.EPError(ep.EP_ERR_STATE, "autotune: every candidate schedule failed on the trial steps")
    best, t_best = min(ok, key=lambda ct: ct[1])
    if kernel_schedules:
        for cand in kernel_schedule_candidates(best):
            t = trial(cand)
            if t is not None and t < t_best:
                best, t_best = cand, t
    return ep.default_opts(**best), results


def sparse_lu_solve(n: int = 256, rtol: float = 1e-12, seed: int = 1):
    """One linear solve with the sparse LU (precond 3) on the elastic tangent of the n x n P2 column
    (the benchmark's mesh): one factorisation and the GMRES iterations its solves precondition.
    Returns (iterations, relative residual).  A small driver for timing and profiling the
    factorisation and solve kernels outside a load path."""
    from synthetic import p2_plane_dp
    prob = p2_plane_dp(n=n, n_steps=40)
    ctx = ep.Context.from_problem(prob)
    try:
        ctx.assemble(np.zeros(prob.n_dof))
        b = np.random.default_rng(seed).standard_normal(prob.n_dof) * (prob.dirichlet == 0)
        _, its, rel = ctx.linear_solve(b, ep.default_opts(krylov=3, krylov_rtol=rtol, krylov_maxit=50, precond=3,
                                                          krylov_graphs=0))
    finally:
        ctx.close()
    return its, rel
