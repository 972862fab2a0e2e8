"""The schedule autotuner on the GPU: it restores the state after every trial, and the schedule it
picks solves the load path to the oracle's solution."""
import numpy as np
import pytest

from synthetic import p2_plane_dp, q1_cube_vm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ep():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_04155_gb300 import build as b
    b.build()
    import paper_1805_04155_gb300.ep as mod
    return mod


@pytest.mark.parametrize("make", [lambda: p2_plane_dp(n=10, n_steps=12, load_fraction=0.9),
                                  lambda: q1_cube_vm(n=4, n_steps=6)])
def test_autotuned_schedule_solves_to_the_oracle(ep, make):
    from oracle.newton import OracleSolver
    from paper_1805_04155_gb300 import drivers as D
    prob = make()
    ctx = ep.Context.from_problem(prob)
    best, table = D.autotune(ctx, prob.zeta, trial_steps=3, base_opts={"newton_rtol": 1e-12, "newton_maxit": 40})
    print("\n" + "\n".join(f"{c['precision']} krylov {c['krylov']} precond {c['precond']}: "
                           f"{'failed' if t is None else f'{t * 1e3:.2f} ms'}" for c, t in table))
    assert sum(t is not None for _, t in table) >= 4
    # the state was restored: the context is at its virgin state
    assert np.all(ctx.get(ep.EP_U) == 0.0) and np.all(ctx.get(ep.EP_PLASTIC_FLAG) == 0)
    reps = ctx.solve_load_path(prob.zeta, best)
    ref = OracleSolver(prob)
    ref.solve_path(tol=1e-13)
    u = ctx.get(ep.EP_U)
    e_u = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    print(f"best: precision {best.precision} krylov {best.krylov} precond {best.precond}; |u-u_or|/|u_or| {e_u:.2e}; "
          f"Newton its {[r.newton_its for r in reps]}")
    assert e_u < 1e-11
    ctx.close()
