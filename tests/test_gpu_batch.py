"""Batched problems (one context over several independent meshes) vs the oracle, problem by problem.

Each problem of a batch must match the oracle solving it alone at the FP64 tolerance
(1e-11 relative on displacements and stresses, flags exact), and the batch must match
separate GPU contexts; the batch shares launches, not arithmetic, between problems.
"""
import numpy as np
import pytest

from gpu_helpers import rel_max
from synthetic import batch_problems, p2_plane_dp, q1_cube_vm, Material, DP

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


def _check_against_oracle(ep, probs, tol_newton, precision=None):
    from oracle.newton import OracleSolver
    ctx = ep.Context.from_batch(probs)
    opts = ep.default_opts(newton_rtol=tol_newton, newton_maxit=40,
                           precision=ep.EP_FP64 if precision is None else precision)
    reps = ctx.solve_load_path(probs[0].zeta, opts)
    us = ctx.split(ep.EP_U, ctx.get(ep.EP_U))
    sig = ctx.split(ep.EP_STRESS, ctx.get(ep.EP_STRESS))
    fl = ctx.split(ep.EP_PLASTIC_FLAG, ctx.get(ep.EP_PLASTIC_FLAG))
    ctx.close()
    for i, pb in enumerate(probs):
        ref = OracleSolver(pb)
        ref.solve_path(tol=min(tol_newton, 1e-13))
        e_u = np.linalg.norm(us[i] - ref.u) / np.linalg.norm(ref.u)
        e_s = rel_max(sig[i], ref.stress)
        print(f"\n{pb.name}: |u-u_or|/|u_or| = {e_u:.2e}, stress {e_s:.2e}")
        assert e_u < TOL and e_s < TOL, pb.name
        assert np.array_equal(fl[i], ref.plastic.astype(np.uint8)), pb.name
    assert all(r.rel_resid <= tol_newton for r in reps)
    return reps


def test_batch_p1_columns_uneven_sizes_and_materials(ep):
    probs = batch_problems(seed=7, n_problems=4, sizes=(4, 9), families=["P1"] * 4, n_steps=8)["P1"]
    assert len({pb.mesh.n_elem for pb in probs}) > 1
    _check_against_oracle(ep, probs, 1e-12)


def test_batch_p2_columns(ep):
    probs = batch_problems(seed=8, n_problems=3, sizes=(3, 6), families=["P2"] * 3, n_steps=8)["P2"]
    _check_against_oracle(ep, probs, 1e-12)


def test_batch_q1_cubes(ep):
    probs = batch_problems(seed=9, n_problems=3, sizes=(2, 4), families=["Q1"] * 3, n_steps=5)["Q1"]
    _check_against_oracle(ep, probs, 1e-12)


def test_batch_drucker_prager_gmres(ep):
    """Nonassociated DP (GMRES path), different cohesions and mesh sizes in one batch."""
    import math
    probs = []
    # the load is 0.8 of the limit traction of c0 = 450, below both problems' limits (the limit
    # traction of the column is proportional to c0 and does not depend on psi)
    for n, c0 in ((4, 450.0), (6, 520.0)):
        pb = p2_plane_dp(n=n, n_steps=10, load_fraction=0.8)
        pb.material = Material(DP, E=206900.0, nu=0.29, c0=c0, phi=math.radians(20.0), psi=math.radians(5.0))
        probs.append(pb)
    _check_against_oracle(ep, probs, 1e-12)


def test_batch_mixed_precision(ep):
    probs = batch_problems(seed=10, n_problems=3, sizes=(4, 8), families=["P1"] * 3, n_steps=8)["P1"]
    _check_against_oracle(ep, probs, 1e-12, precision=ep.EP_MIXED)


def test_batch_equals_separate_contexts(ep):
    probs = batch_problems(seed=11, n_problems=3, sizes=(6, 12), families=["Q1"] * 3, n_steps=4)["Q1"]
    ctx = ep.Context.from_batch(probs)
    ctx.solve_load_path(probs[0].zeta, ep.default_opts(newton_rtol=1e-12))
    us = ctx.split(ep.EP_U, ctx.get(ep.EP_U))
    ctx.close()
    for i, pb in enumerate(probs):
        c1 = ep.Context.from_problem(pb)
        c1.solve_load_path(pb.zeta, ep.default_opts(newton_rtol=1e-12))
        u1 = c1.get(ep.EP_U)
        c1.close()
        assert np.linalg.norm(us[i] - u1) / np.linalg.norm(u1) < 1e-10
