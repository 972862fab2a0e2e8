"""GPU (C ABI) vs CPU oracle, element by element, for every step of the hot path.

Tolerance: 1e-11 relative for K, F, stresses and displacements (FP64 path);
plastic flags and integer outputs exact.  Meshes are small enough for the
oracle but span several CTA tiles with a ragged last tile.
"""
import math

import numpy as np
import pytest

from gpu_helpers import (ALL_ELEMS, fed_iterate, material, oracle_eval, rel_fro, rel_max, small_problem)
from oracle import constitutive as OC
from synthetic import DP, ELASTIC, VM_ISO, VM_KIN

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = 1e-11

# element counts chosen to leave a ragged last CTA tile (tiles: P1-2D 128, P2-2D 32, Q1-2D 64,
# Q2-2D 16, P1-3D 64, P2-3D 4, Q1-3D 8, Q2-3D 1 elements)
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


@pytest.mark.parametrize("elem,dim", ALL_ELEMS)
def test_geometry_and_elastic_stiffness(ep, elem, dim):
    prob = small_problem(elem, dim, SIZES[(elem, dim)], ELASTIC, seed=1)
    ctx = ep.Context.from_problem(prob)
    from oracle.fem import Geometry
    g = Geometry(prob.mesh.coords, prob.mesh.elem, elem, dim)
    w = ctx.get(ep.EP_WEIGHT)
    dphi = ctx.get(ep.EP_DPHI)                   # [n_int][n_p][dim]
    assert rel_max(w, g.WEIGHT) < TOL
    assert rel_max(dphi, np.transpose(g.DPhi, (2, 1, 0))) < TOL
    Kel = ctx.K_csr(elastic=True)
    from oracle.fem import Assembler
    K, G = OC.moduli(prob.material.E, prob.material.nu)
    De = OC.elastic_tangent(K, G)
    if dim == 2:
        De = De[np.ix_(OC.PLANE_INPLANE_IDX, OC.PLANE_INPLANE_IDX)]
    Kor = Assembler(g, De).K_elast
    assert rel_fro(Kel, Kor) < TOL
    ctx.close()


MODELS = [VM_KIN, VM_ISO, DP, ELASTIC]


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("elem,dim", ALL_ELEMS)
def test_fed_iterate_assembly(ep, elem, dim, model):
    """K (split and full forms), F and the plastic count at an oracle-fed iterate and state."""
    prob = small_problem(elem, dim, SIZES[(elem, dim)], model, seed=2)
    u, ep_, hard = fed_iterate(prob, seed=3, dilate=(1.5e-3 if model == DP else 0.0))
    ctx = ep.Context.from_problem(prob)
    ctx.set(ep.EP_PLASTIC_STRAIN, ep_)
    ctx.set(ep.EP_HARDENING, hard)
    for split in (True, False):
        ref = oracle_eval(prob, u, ep_, hard, split=split)
        n_pl = ctx.assemble(u, split=split)
        assert n_pl == int(np.count_nonzero(ref["res"]["plastic"]))
        if model != ELASTIC:
            assert n_pl > 0
        assert rel_fro(ctx.K_csr(), ref["K"]) < TOL
        assert rel_max(ctx.get(ep.EP_F_INT), ref["F"]) < TOL
    # commit: stress, plastic strain, hardening and flags of the new state
    ref = oracle_eval(prob, u, ep_, hard)
    ctx.commit(u)
    assert rel_max(ctx.get(ep.EP_STRESS), ref["res"]["S"]) < TOL
    assert rel_max(ctx.get(ep.EP_PLASTIC_STRAIN), ref["res"]["ep"]) < TOL
    if model != ELASTIC:
        h = ctx.get(ep.EP_HARDENING)
        assert rel_max(h, np.asarray(ref["res"]["hard"])) < TOL
    flags = ctx.get(ep.EP_PLASTIC_FLAG)
    assert np.array_equal(flags, ref["res"]["plastic"].astype(np.uint8))
    assert np.array_equal(ctx.get(ep.EP_U), u)
    ctx.close()


@pytest.mark.parametrize("model,elem,dim", [(DP, "P2", 2), (VM_ISO, "Q1", 3), (VM_KIN, "P1", 2), (DP, "P2", 3)])
def test_split_reset_follows_changing_plastic_sets(ep, model, elem, dim):
    """Eq. (K-split) across a sequence of split assemblies whose plastic sets differ: each one resets
    only the blocks the previous one moved away from K_elast, so every K must still equal the
    oracle's K_elast + sum over the current plastic points (large set, small set, none, large)."""
    prob = small_problem(elem, dim, SIZES[(elem, dim)] + 1, model, seed=7)
    u, ep_, hard = fed_iterate(prob, seed=8, dilate=(1.5e-3 if model == DP else 0.0))
    ctx = ep.Context.from_problem(prob)
    ctx.set(ep.EP_PLASTIC_STRAIN, ep_)
    ctx.set(ep.EP_HARDENING, hard)
    counts = []
    for scale in (1.0, 0.35, 0.0, 1.0, 0.6):
        us = u * scale
        ref = oracle_eval(prob, us, ep_, hard, split=True)
        n_pl = ctx.assemble(us, split=True)
        counts.append(n_pl)
        assert n_pl == int(np.count_nonzero(ref["res"]["plastic"]))
        assert rel_fro(ctx.K_csr(), ref["K"]) < TOL
        assert rel_max(ctx.get(ep.EP_F_INT), ref["F"]) < TOL
    assert counts[0] > counts[1] and len(set(counts)) >= 3, counts
    # a full assembly in between, then split again (the next split starts from a whole copy)
    ctx.assemble(u, split=False)
    ref = oracle_eval(prob, u * 0.35, ep_, hard, split=True)
    ctx.assemble(u * 0.35, split=True)
    assert rel_fro(ctx.K_csr(), ref["K"]) < TOL
    ctx.close()


def test_reset_returns_to_the_virgin_state(ep):
    """ep_reset: state fields zero, and a load path solved after it equals one from a new context."""
    from synthetic import p1_plane_vm
    prob = p1_plane_vm(n=8, n_steps=6)
    opts = ep.default_opts(newton_rtol=1e-12)
    ctx = ep.Context.from_problem(prob)
    ctx.solve_load_path(prob.zeta, opts)
    u1, s1 = ctx.get(ep.EP_U), ctx.get(ep.EP_STRESS)
    assert np.count_nonzero(ctx.get(ep.EP_PLASTIC_FLAG)) > 0
    ctx.reset()
    for f in (ep.EP_U, ep.EP_STRESS, ep.EP_PLASTIC_STRAIN, ep.EP_HARDENING, ep.EP_PLASTIC_FLAG):
        assert not np.any(ctx.get(f))
    reps = ctx.solve_load_path(prob.zeta, opts)
    assert reps[0].start == 0          # no extrapolation from the path before the reset
    assert rel_max(ctx.get(ep.EP_U), u1) < TOL and rel_max(ctx.get(ep.EP_STRESS), s1) < TOL
    ctx.close()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("model", MODELS)
def test_constitutive_fuzz(ep, dim, model):
    """Stand-alone return mapping on seeded states spanning elastic, smooth and apex returns."""
    n = 20000 + 37
    g = np.random.default_rng(100 + dim * 10 + model)
    ns = 3 if dim == 2 else 6
    nc = OC.n_comp(dim)
    E = g.standard_normal((ns, n)) * 2e-3
    E[:2 if dim == 2 else 3] += g.uniform(-3e-3, 4e-3, n)
    ep_prev = g.standard_normal((nc, n)) * 2e-4
    if model == VM_KIN:
        hard = OC.extract_state(OC.DEV @ OC.embed_state(g.standard_normal((nc, n)) * 50.0, dim), dim)
    else:
        hard = np.abs(g.standard_normal(n)) * 1e-3
    mat = material(model, dim)
    ref = OC.constitutive(mat, dim, E, ep_prev, hard)
    dev = torch.device("cuda:0")
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    S, DS, flag, ep_new, hard_new = ep.constitutive(mat, dim, T(E), T(ep_prev), T(hard))
    torch.cuda.synchronize()
    assert np.array_equal(flag.cpu().numpy(), ref["plastic"].astype(np.uint8))
    if model == DP:
        assert set(np.unique(ref["plastic"])) == {0, 1, 2}
    assert rel_max(S.cpu().numpy(), ref["S"]) < TOL
    assert rel_max(DS.cpu().numpy(), ref["DS_in"]) < TOL
    assert rel_max(ep_new.cpu().numpy(), ref["ep"]) < TOL
    assert rel_max(hard_new.cpu().numpy(), np.asarray(ref["hard"])) < TOL


@pytest.mark.parametrize("method", [1, 2, 3])
@pytest.mark.parametrize("model,elem,dim", [(VM_ISO, "P2", 2), (DP, "P2", 2), (VM_ISO, "Q1", 3), (DP, "P2", 3)])
def test_krylov_solve_matches_direct(ep, model, elem, dim, method):
    """CG (symmetric tangents only), BiCGStab and GMRES vs a sparse direct solve."""
    if method == 1 and model == DP:
        pytest.skip("CG needs a symmetric tangent")
    import scipy.sparse.linalg as spla
    prob = small_problem(elem, dim, SIZES[(elem, dim)] + 1, model, seed=4)
    u, ep_, hard = fed_iterate(prob, seed=5, dilate=(1.0e-3 if model == DP else 0.0))
    ctx = ep.Context.from_problem(prob)
    ctx.set(ep.EP_PLASTIC_STRAIN, ep_)
    ctx.set(ep.EP_HARDENING, hard)
    ctx.assemble(u)
    K = ctx.K_csr()
    free = prob.dirichlet == 0
    b = np.random.default_rng(6).standard_normal(prob.n_dof) * free
    for precond in (0, 1, 2):
        x, its, rel = ctx.linear_solve(b, ep.default_opts(krylov=method, krylov_rtol=1e-13, krylov_maxit=20000,
                                                         precond=precond))
        xr = np.zeros(prob.n_dof)
        xr[free] = spla.spsolve(K[free][:, free].tocsc(), b[free])
        assert its > 0 and rel <= 1e-13
        assert np.all(x[~free] == 0.0)
        assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-9
    ctx.close()


def _path_parity(ep, prob, tol_newton, opts=None):
    from oracle.newton import OracleSolver
    ctx = ep.Context.from_problem(prob)
    reps = ctx.solve_load_path(prob.zeta, opts or ep.default_opts(newton_rtol=tol_newton))
    ref = OracleSolver(prob)
    ref.solve_path(tol=min(tol_newton, 1e-13))
    u = ctx.get(ep.EP_U)
    assert np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u) < TOL
    assert rel_max(ctx.get(ep.EP_STRESS), ref.stress) < TOL
    assert rel_max(ctx.get(ep.EP_PLASTIC_STRAIN), ref.ep) < max(TOL, 1e-16 / max(np.abs(ref.ep).max(), 1e-300))
    assert np.array_equal(ctx.get(ep.EP_PLASTIC_FLAG), ref.plastic.astype(np.uint8))
    ctx.close()
    return reps


def test_load_path_p1_von_mises_column(ep):
    """Plane-strain P1 column, von Mises isotropic hardening, 20 steps to 1.5x first yield, 1e-12."""
    from synthetic import p1_plane_vm
    prob = p1_plane_vm()
    reps = _path_parity(ep, prob, 1e-12)
    assert reps[-1].n_plastic == prob.mesh.n_elem
    assert all(r.rel_resid <= 1e-12 for r in reps)


def test_load_path_p2_drucker_prager_column(ep):
    """Plane-strain P2 column, nonassociated DP, to 0.98 of the limit traction (reduced mesh)."""
    from synthetic import p2_plane_dp
    prob = p2_plane_dp(n=12, n_steps=20, load_fraction=0.98)
    # near the limit load the tangent is ill-conditioned: 1e-11 in u needs a 1e-13 residual
    reps = _path_parity(ep, prob, 1e-13, ep.default_opts(newton_rtol=1e-13, newton_maxit=40))
    assert reps[-1].n_plastic == prob.mesh.n_elem * 7


@pytest.mark.parametrize("model,prob_name", [(DP, "p2_dp"), (VM_ISO, "q1_vm")])
def test_precise_vcycle_load_path(ep, monkeypatch, model, prob_name):
    """The precise V-cycle (FP64 coarse correction and level-0 residuals, forced from the start of
    the path) reaches the oracle's load path; every step reports it."""
    from synthetic import p2_plane_dp, q1_cube_vm
    monkeypatch.setenv("EP_AMG_PRECISE", "1")
    prob = p2_plane_dp(n=12, n_steps=10, load_fraction=0.95) if prob_name == "p2_dp" else q1_cube_vm(n=5, n_steps=6)
    # near the limit load 1e-11 in eps^p needs a 1e-13 residual (as in the direct test above)
    reps = _path_parity(ep, prob, 1e-13, ep.default_opts(newton_rtol=1e-13, newton_maxit=40, precond=2))
    assert all(r.precise == 1 for r in reps if r.krylov_its > 0)
    assert reps[-1].n_plastic > 0


def test_load_path_p2_full_size_all_steps(ep):
    """The 256x256 P2 column to 0.95 t_lim (40 steps, V-cycle GMRES throughout) end to end, against the
    one-point oracle (0.98 t_lim: tests/test_gpu_direct.py)."""
    from oracle.newton import homogeneous_column
    from synthetic import p2_plane_dp
    prob = p2_plane_dp(load_fraction=0.95)
    ctx = ep.Context.from_problem(prob)
    reps = ctx.solve_load_path(prob.zeta, ep.default_opts(newton_rtol=1e-10))
    sig = ctx.get(ep.EP_STRESS)
    ctx.close()
    hom = homogeneous_column(prob.material, prob.zeta * prob.extra["load_fraction"] * prob.extra["t_lim"])
    assert rel_max(sig, np.repeat(hom[-1]["stress"][:, None], sig.shape[1], axis=1)) < 1e-9
    assert all(r.rel_resid <= 1e-10 for r in reps) and reps[-1].n_plastic == sig.shape[1]


def test_load_path_q1_cube_fixed_base(ep):
    from synthetic import q1_cube_vm
    prob = q1_cube_vm(n=4, n_steps=6)
    _path_parity(ep, prob, 1e-12)


def test_load_path_p2_tet_strip(ep):
    from synthetic import p2_tet_strip_dp
    prob = p2_tet_strip_dp(n=3, n_steps=6)
    _path_parity(ep, prob, 1e-12)


def test_homogeneous_column_full_size_p2(ep):
    """Full-size P2 column (256x256, 917504 points) to 0.95 t_lim in 10 steps: every point equals the
    one-point oracle."""
    from oracle.newton import homogeneous_column
    from synthetic import p2_plane_dp
    prob = p2_plane_dp(load_fraction=0.95)
    ctx = ep.Context.from_problem(prob)
    zs = prob.zeta[::4]           # 10 of the 40 steps, same end point
    reps = ctx.solve_load_path(zs, ep.default_opts(newton_rtol=1e-10))
    sig = ctx.get(ep.EP_STRESS)
    flags = ctx.get(ep.EP_PLASTIC_FLAG)
    ctx.close()
    hom = homogeneous_column(prob.material, zs * prob.extra["load_fraction"] * prob.extra["t_lim"])
    want = hom[-1]["stress"]
    assert rel_max(sig, np.repeat(want[:, None], sig.shape[1], axis=1)) < 1e-9
    assert np.all(flags == hom[-1]["plastic"])
    assert all(r.rel_resid <= 1e-10 for r in reps)


# ---------------------------------------------------------------------------
# Error paths (host-made failures; nothing faults the GPU)
# ---------------------------------------------------------------------------
def test_inverted_element_is_rejected(ep):
    prob = small_problem("Q1", 2, 3, ELASTIC, perturb=0.0)
    elem = prob.mesh.elem.copy()
    elem[4] = elem[4][[1, 0, 3, 2]]          # reversed orientation
    with pytest.raises(ep.EPError) as e:
        ep.Context(prob.mesh.coords, elem, "Q1", prob.material, prob.dirichlet, None, prob.f_unit)
    assert e.value.status == ep.EP_ERR_BAD_ELEMENT


def test_bad_node_index_is_rejected(ep):
    prob = small_problem("P1", 2, 3, ELASTIC, perturb=0.0)
    elem = prob.mesh.elem.copy()
    elem[0, 0] = prob.mesh.n_nodes
    with pytest.raises(ep.EPError) as e:
        ep.Context(prob.mesh.coords, elem, "P1", prob.material, prob.dirichlet)
    assert e.value.status == ep.EP_ERR_INVALID_ARG


def test_apex_without_dilatancy_reports_return_map_error(ep):
    from synthetic import Material
    prob = small_problem("P1", 2, 4, DP, perturb=0.0)
    prob.material = Material(DP, E=E_MOD_, nu=0.3, c0=10.0, phi=math.radians(20), psi=0.0, Hc=0.0)
    ctx = ep.Context.from_problem(prob)
    u = prob.mesh.coords.ravel() * 1e-2                 # strong dilation -> apex
    with pytest.raises(ep.EPError) as e:
        ctx.assemble(u)
    assert e.value.status == ep.EP_ERR_RETURN_MAP
    ctx.close()


E_MOD_ = 1e4


def test_newton_cap_and_nan_are_reported(ep):
    from synthetic import p1_plane_vm
    prob = p1_plane_vm(n=6, n_steps=4)
    ctx = ep.Context.from_problem(prob)
    st, reps = ctx.solve_load_path([1.0], ep.default_opts(newton_maxit=1, krylov_rtol=0.5), raise_on_error=False)
    assert st == ep.EP_ERR_NEWTON_NO_CONVERGENCE
    # the failed step left the state at the last converged step (virgin)
    assert np.all(ctx.get(ep.EP_U) == 0.0)
    bad = np.zeros((4, prob.mesh.n_elem))
    bad[0, 3] = np.nan
    ctx.set(ep.EP_PLASTIC_STRAIN, bad)
    st, reps = ctx.solve_load_path([0.5], ep.default_opts(), raise_on_error=False)
    assert st == ep.EP_ERR_NAN
    ctx.close()


def test_krylov_cap_is_reported(ep):
    prob = small_problem("Q1", 3, 4, VM_ISO)
    ctx = ep.Context.from_problem(prob)
    ctx.assemble(np.zeros(prob.n_dof))
    b = np.ones(prob.n_dof) * (prob.dirichlet == 0)
    with pytest.raises(ep.EPError) as e:
        ctx.linear_solve(b, ep.default_opts(krylov_rtol=1e-14, krylov_maxit=2, precond=1))
    assert e.value.status == ep.EP_ERR_KRYLOV
    ctx.close()


def test_resume_from_saved_state(ep):
    """Checkpoint after k steps, restore into a fresh context, continue: the same solution.

    FP64 atomics make the summation order, hence the last bits, differ from run to run, so the
    two runs agree to the accuracy the Newton tolerance fixes (tight here), not bit for bit."""
    from synthetic import p2_plane_dp
    prob = p2_plane_dp(n=6, n_steps=10, load_fraction=0.95)
    opts = ep.default_opts(newton_rtol=1e-13, newton_maxit=40, warm_start=0)
    a = ep.Context.from_problem(prob)
    a.solve_load_path(prob.zeta, opts)
    b = ep.Context.from_problem(prob)
    b.solve_load_path(prob.zeta[:6], opts)
    saved = {f: b.get(f) for f in (ep.EP_U, ep.EP_PLASTIC_STRAIN, ep.EP_HARDENING, ep.EP_STRESS, ep.EP_PLASTIC_FLAG)}
    b.close()
    c = ep.Context.from_problem(prob)
    for f, v in saved.items():
        c.set(f, v)
    c.solve_load_path(prob.zeta[6:], opts)
    for f in (ep.EP_U, ep.EP_STRESS, ep.EP_PLASTIC_STRAIN):
        assert rel_max(c.get(f), a.get(f)) < 1e-11
    assert np.array_equal(a.get(ep.EP_PLASTIC_FLAG), c.get(ep.EP_PLASTIC_FLAG))
    a.close()
    c.close()
