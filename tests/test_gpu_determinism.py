"""Deterministic form (ep_opts.deterministic): coloured assembly without atomics, fixed-order
Galerkin products, per-step preconditioner.

K and F of the coloured assembly equal the atomic assembly's to 1e-14 (only the summation order
differs) and the oracle's to 1e-11; a load path repeats bit for bit; a run resumed from a saved state
equals the uninterrupted run bit for bit.
"""
import numpy as np
import pytest

from gpu_helpers import ALL_ELEMS, fed_iterate, oracle_eval, rel_fro, rel_max, small_problem
from synthetic import DP, VM_ISO

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
SIZES = {("P1", 2): 9, ("P2", 2): 7, ("Q1", 2): 9, ("Q2", 2): 5, ("P1", 3): 3, ("P2", 3): 3, ("Q1", 3): 3,
         ("Q2", 3): 2}


@pytest.fixture(scope="module")
def ep():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_04155_gb300 import build as b
    b.build()
    import paper_1805_04155_gb300.ep as mod
    return mod


def _set_det(ep, ctx, det):
    # n_steps = 0: applies the options (the deterministic mode stays with the context)
    ctx.solve_load_path(np.zeros(0), ep.default_opts(deterministic=det, precond=0))


@pytest.mark.parametrize("model", [DP, VM_ISO])
@pytest.mark.parametrize("elem,dim", ALL_ELEMS)
def test_coloured_assembly_equals_atomic_assembly(ep, elem, dim, model):
    prob = small_problem(elem, dim, SIZES[(elem, dim)] + 1, model, seed=21)
    u, ep_, hard = fed_iterate(prob, seed=22, dilate=(1.5e-3 if model == DP else 0.0))
    ctx = ep.Context.from_problem(prob)
    ctx.set(ep.EP_PLASTIC_STRAIN, ep_)
    ctx.set(ep.EP_HARDENING, hard)
    for split in (True, False):
        ref = oracle_eval(prob, u, ep_, hard, split=split)
        _set_det(ep, ctx, 0)
        n_a = ctx.assemble(u, split=split)
        Ka, Fa = ctx.K_csr(), ctx.get(ep.EP_F_INT)
        _set_det(ep, ctx, 1)
        n_c = ctx.assemble(u, split=split)
        Kc, Fc = ctx.K_csr(), ctx.get(ep.EP_F_INT)
        assert n_a == n_c > 0
        assert rel_fro(Kc, Ka) < 1e-14 and rel_max(Fc, Fa) < 1e-14
        assert rel_fro(Kc, ref["K"]) < 1e-11 and rel_max(Fc, ref["F"]) < 1e-11
        # the coloured assembly is bit-reproducible
        ctx.assemble(u, split=split)
        assert np.array_equal(ctx.K_csr().data, Kc.data) and np.array_equal(ctx.get(ep.EP_F_INT), Fc)
    ctx.close()


def _path(ep, prob, steps, det, state=None, **kw):
    ctx = ep.Context.from_problem(prob)
    if state is not None:
        for f, v in state.items():
            ctx.set(f, v)
    reps = ctx.solve_load_path(steps, ep.default_opts(newton_rtol=1e-10, deterministic=det, warm_start=0, **kw))
    fields = (ep.EP_U, ep.EP_STRESS, ep.EP_PLASTIC_STRAIN, ep.EP_HARDENING, ep.EP_PLASTIC_FLAG)
    out = {f: ctx.get(f) for f in fields}
    ctx.close()
    return out, reps


@pytest.mark.parametrize("which", ["p2_dp", "q1_vm"])
def test_deterministic_path_repeats_and_resumes_bit_for_bit(ep, which):
    from synthetic import problems as P
    prob = P.p2_plane_dp(n=16, n_steps=12, load_fraction=0.9) if which == "p2_dp" else P.q1_cube_vm(n=6, n_steps=8)
    z = prob.zeta
    a, reps = _path(ep, prob, z, 1)
    assert reps[-1].n_plastic > 0
    b, _ = _path(ep, prob, z, 1)
    for f in a:
        assert np.array_equal(a[f], b[f]), f
    k = len(z) // 2
    half, _ = _path(ep, prob, z[:k], 1)
    c, _ = _path(ep, prob, z[k:], 1, state=half)
    for f in a:
        assert np.array_equal(a[f], c[f]), f
    # the atomic form reaches the same converged path to the Newton tolerance
    d, _ = _path(ep, prob, z, 0)
    assert rel_max(d[ep.EP_U], a[ep.EP_U]) < 1e-8


def test_graph_replayed_krylov_iterations_equal_direct_launches(ep):
    """GMRES iterations replayed from captured CUDA graphs run the same kernels in the same order as
    direct launches: in the deterministic form the two load paths are identical bit for bit."""
    from synthetic import problems as P
    prob = P.p2_plane_dp(n=16, n_steps=12, load_fraction=0.9)
    a, reps = _path(ep, prob, prob.zeta, 1, krylov_graphs=1)
    assert sum(r.krylov_its for r in reps) > 0
    b, _ = _path(ep, prob, prob.zeta, 1, krylov_graphs=0)
    for f in a:
        assert np.array_equal(a[f], b[f]), f


@pytest.mark.parametrize("elem,dim", [("P2", 2), ("Q1", 3), ("P2", 3)])
def test_half_tile_assembly_schedule_equals_the_default(ep, elem, dim):
    """The autotuner's second assembly schedule (half the elements per CTA) computes the same K and F
    (coloured form: bit for bit)."""
    prob = small_problem(elem, dim, SIZES[(elem, dim)] + 1, DP, seed=23)
    u, ep_, hard = fed_iterate(prob, seed=24, dilate=1.5e-3)
    ctx = ep.Context.from_problem(prob)
    ctx.set(ep.EP_PLASTIC_STRAIN, ep_)
    ctx.set(ep.EP_HARDENING, hard)
    out = {}
    for tile in (1, 2):
        ctx.solve_load_path(np.zeros(0), ep.default_opts(deterministic=1, precond=0, asm_tile=tile))
        ctx.assemble(u, split=True)
        out[tile] = (ctx.K_csr().data.copy(), ctx.get(ep.EP_F_INT))
    assert np.array_equal(out[1][0], out[2][0]) and np.array_equal(out[1][1], out[2][1])
    ctx.close()
