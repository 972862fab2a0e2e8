"""Edge cases of the load path on the GPU: an empty path, a zero load, and meshes of one or two
elements (a CTA's element slots mostly empty), each against the oracle where it computes anything."""
import numpy as np
import pytest

from gpu_helpers import rel_max
from synthetic import p1_plane_vm, q1_cube_vm

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


def test_empty_load_path_leaves_the_state(ep):
    ctx = ep.Context.from_problem(p1_plane_vm(n=3, n_steps=2))
    assert ctx.solve_load_path([]) == []
    assert np.all(ctx.get(ep.EP_U) == 0.0) and np.all(ctx.get(ep.EP_PLASTIC_FLAG) == 0)
    ctx.close()


def test_zero_load_converges_at_once(ep):
    ctx = ep.Context.from_problem(p1_plane_vm(n=3, n_steps=2))
    reps = ctx.solve_load_path([0.0])
    assert reps[0].newton_its == 0 and reps[0].n_plastic == 0
    assert np.all(ctx.get(ep.EP_U) == 0.0)
    ctx.close()


@pytest.mark.parametrize("make", [lambda: p1_plane_vm(n=1, n_steps=6), lambda: q1_cube_vm(n=1, n_steps=4)],
                         ids=["p1_two_triangles", "q1_one_hexahedron"])
def test_smallest_meshes_match_the_oracle(ep, make):
    from oracle.newton import OracleSolver
    prob = make()
    ctx = ep.Context.from_problem(prob)
    reps = ctx.solve_load_path(prob.zeta, ep.default_opts(newton_rtol=1e-12))
    ref = OracleSolver(prob)
    ref.solve_path(tol=1e-13)
    u = ctx.get(ep.EP_U)
    e_u = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    e_s = rel_max(ctx.get(ep.EP_STRESS), ref.stress)
    print(f"\n{prob.name}: {prob.mesh.elem.shape[0]} elements, |u-u_or|/|u_or| {e_u:.2e}, stress {e_s:.2e}, "
          f"Newton its {[r.newton_its for r in reps]}, plastic {reps[-1].n_plastic}")
    assert e_u < TOL and e_s < TOL
    assert np.array_equal(ctx.get(ep.EP_PLASTIC_FLAG), ref.plastic.astype(np.uint8))
    ctx.close()
