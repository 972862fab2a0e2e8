"""The paper's validation experiments (Section 8.2, 8.3) on the GPU path.

Parity: the cyclic L-shape (von Mises, kinematic hardening) and the first steps of the strip
footing (Drucker-Prager, displacement control) against the oracle at 1e-11.  Validation: the
L-shape's load cycle is a hysteresis loop (positive dissipated work, a residual displacement after
unloading), and the strip footing's limit pressure approaches Prandtl's c N_c.
"""
import math

import numpy as np
import pytest

from gpu_helpers import rel_max
from synthetic import l_shape_vm, prandtl_nc, strip_footing_dp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = 1e-11


@pytest.fixture(scope="module")
def ep():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_04155_gb300 import build as b
    b.build()
    import paper_1805_04155_gb300.ep as mod
    return mod


def test_l_shape_cyclic_matches_oracle_and_loops(ep):
    from oracle.newton import OracleSolver
    from paper_1805_04155_gb300.drivers import external_work
    prob = l_shape_vm("Q2", m=3, n_steps=40)
    ctx = ep.Context.from_problem(prob)
    ref = OracleSolver(prob)
    work, work_ref = [], []
    for z in prob.zeta:
        ctx.solve_load_path([z], ep.default_opts(newton_rtol=1e-12))
        ref.solve_step(float(z), tol=1e-13)
        work.append(external_work(ctx, prob))
        work_ref.append(float(prob.f_unit @ ref.u))
    u = ctx.get(ep.EP_U)
    e_u = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    e_s = rel_max(ctx.get(ep.EP_STRESS), ref.stress)
    e_b = rel_max(ctx.get(ep.EP_HARDENING), ref.hard)
    print(f"\nL-shape cyclic: |u-u_or|/|u_or| = {e_u:.2e}, stress {e_s:.2e}, back stress {e_b:.2e}")
    assert e_u < TOL and e_s < TOL and e_b < TOL
    np.testing.assert_allclose(work, work_ref, rtol=1e-10)
    z = prob.zeta
    w = np.array(work)
    # hysteresis: the work at the same load factor differs on loading and unloading branches, and
    # the closed cycle leaves a residual displacement (dissipated energy: positive loop area)
    area = 0.5 * np.sum((z[1:] - z[:-1]) * (w[1:] + w[:-1]))
    print(f"loop: work at zeta=0.5 loading {w[4]:.4e}, unloading {w[14]:.4e}; residual work {w[-1]:.4e}")
    assert abs(w[-1]) > 1e-3 * np.abs(w).max()
    assert abs(w[4] - w[14]) > 1e-3 * np.abs(w).max()
    assert ctx.get(ep.EP_PLASTIC_FLAG).any() or np.abs(ctx.get(ep.EP_PLASTIC_STRAIN)).max() > 0
    assert area != 0.0
    ctx.close()


def test_strip_footing_first_steps_match_oracle(ep):
    from oracle.newton import OracleSolver
    prob = strip_footing_dp("P2", n=8)
    ctx = ep.Context.from_problem(prob)
    ctx.solve_load_path(prob.zeta, ep.default_opts(newton_rtol=1e-12))
    ref = OracleSolver(prob)
    ref.solve_path(tol=1e-13)
    e_u = np.linalg.norm(ctx.get(ep.EP_U) - ref.u) / np.linalg.norm(ref.u)
    e_s = rel_max(ctx.get(ep.EP_STRESS), ref.stress)
    print(f"\nstrip footing (8x8 P2, 10 steps): |u-u_or|/|u_or| = {e_u:.2e}, stress {e_s:.2e}, "
          f"plastic points {int(ref.plastic.astype(bool).sum())}")
    assert e_u < TOL and e_s < TOL
    assert np.array_equal(ctx.get(ep.EP_PLASTIC_FLAG), ref.plastic.astype(np.uint8))
    ctx.close()


def test_strip_footing_limit_pressure_approaches_prandtl(ep):
    """Adaptive displacement path to u_D = 1: the footing pressure levels off near c0 N_c."""
    from paper_1805_04155_gb300.drivers import strip_footing_path
    prob = strip_footing_dp("P2", n=64)
    ctx = ep.Context.from_problem(prob)
    us, ps, reps = strip_footing_path(ctx, prob, opts=ep.default_opts(newton_rtol=1e-10, newton_maxit=50))
    ctx.close()
    nc = prandtl_nc(prob.material.phi)
    ratio = ps[-1] / (prob.material.c0 * nc)
    print(f"\nstrip footing 64x64 P2: {len(us)} steps, u_D = {us[-1]:.3f}, p/c0 = {ps[-1] / prob.material.c0:.3f}, "
          f"Prandtl N_c = {nc:.3f}, ratio {ratio:.3f}; last pressure increments {np.diff(ps)[-3:]}")
    assert us[-1] >= 1.0 - 1e-9
    assert all(r.rel_resid <= 1e-10 for r in reps)
    # the pressure is bounded: it has levelled off (last doubling steps add < 1 %)
    assert (ps[-1] - ps[-4]) / ps[-1] < 0.01
    # and the limit is Prandtl's within the discretisation error of a 64x64 P2 mesh
    assert 0.95 < ratio < 1.15
