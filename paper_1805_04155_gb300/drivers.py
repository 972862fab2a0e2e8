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
