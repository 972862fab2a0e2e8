"""Mixed-precision path (FP32 tangent and inner Krylov, FP64 residual) vs the FP64 oracle.

What stays FP64 (strains, return mapping, F, Newton residual) is held to the
FP64 tolerance 1e-11.  The FP32 tangent is held to a componentwise forward
error bound: every entry of K is formed by at most n_r = 2*NS + 2*NQ*NS +
N_SHARE sequential FP32 roundings (NS rows of D and of H = D G, the sum over
the NQ points of one element, the atomic sum over the elements sharing a node
pair), so |K32 - K| <= gamma(n_r) * K_abs with gamma(n) = n u / (1 - n u),
u = 2^-24, and K_abs = B_abs^T |W| S B_abs (the same assembly over absolute
values) with the per-point scale S = |D| + 2|C| + 4(K + 2G) at plastic points:
the tangent's coefficients (Section 2) are each bounded by 4(K + 2G) and the
terms of one entry may cancel, and split mode adds the rounded K_elast.  Load paths must
reach the same Newton tolerance as the FP64 path, so their displacements and
stresses are held to the FP64 tolerance too; each test prints its error
against the oracle.
"""
import math

import numpy as np
import pytest

from gpu_helpers import ALL_ELEMS, fed_iterate, oracle_eval, rel_fro, rel_max, small_problem
from oracle import constitutive as OC
from synthetic import DP, ELASTIC, VM_ISO, VM_KIN

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = 1e-11
U32 = 2.0 ** -24
NQ = {("P1", 2): 1, ("P2", 2): 7, ("Q1", 2): 4, ("Q2", 2): 9, ("P1", 3): 1, ("P2", 3): 11, ("Q1", 3): 8,
      ("Q2", 3): 27}
N_SHARE = 32          # more than the elements sharing a node pair in any of the test meshes
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


def _gamma(n):
    return n * U32 / (1.0 - n * U32)


def _abs_bound(ref, DS_abs):
    """B_abs^T |W| |D| B_abs summed over all points (the scale of the FP32 rounding errors)."""
    B = abs(ref["asm"].B).tocsr()
    g = ref["geom"]
    return (B.T @ g.block_diag(DS_abs * np.abs(g.WEIGHT), weighted=False) @ B).tocsr()


@pytest.mark.parametrize("model", [VM_KIN, VM_ISO, DP, ELASTIC])
@pytest.mark.parametrize("elem,dim", ALL_ELEMS)
def test_mixed_assembly(ep, elem, dim, model):
    """F, plastic count and flags as FP64; the FP32 tangent within its rounding bound."""
    prob = small_problem(elem, dim, SIZES[(elem, dim)], model, seed=2)
    u, ep_, hard = fed_iterate(prob, seed=3, dilate=(1.5e-3 if model == DP else 0.0))
    ctx = ep.Context.from_problem(prob)
    ctx.set(ep.EP_PLASTIC_STRAIN, ep_)
    ctx.set(ep.EP_HARDENING, hard)
    ns = 3 if dim == 2 else 6
    n_r = 2 * ns + 2 * NQ[(elem, dim)] * ns + N_SHARE
    K_b, G_b = OC.moduli(prob.material.E, prob.material.nu)
    C = OC.elastic_tangent(K_b, G_b)
    if dim == 2:
        C = C[np.ix_(OC.PLANE_INPLANE_IDX, OC.PLANE_INPLANE_IDX)]
    for split in (True, False):
        ref = oracle_eval(prob, u, ep_, hard, split=split)
        n_pl = ctx.assemble(u, split=split, precision=ep.EP_MIXED)
        assert n_pl == int(np.count_nonzero(ref["res"]["plastic"]))
        assert rel_max(ctx.get(ep.EP_F_INT), ref["F"]) < TOL
        K32 = ctx.K_csr(f32=True)
        DS = ref["res"]["DS_in"]
        # scale of the rounded terms per point: |D| + 2|C|, plus 4(K + 2G) at plastic points (every
        # tangent coefficient of Section 2 is bounded by that, and the terms of one entry may cancel)
        plastic = (ref["res"]["plastic"] != 0).astype(float)
        scale = np.abs(DS) + 2 * np.abs(C)[:, :, None] + 4 * (K_b + 2 * G_b) * plastic[None, None, :]
        bound = _abs_bound(ref, scale)
        err = abs(K32 - ref["K"]).tocsr()
        # plus FP64-level differences of the inputs (GPU and oracle geometry agree to ~1e-16, so an
        # entry that is exactly zero in the oracle can be ~1e-17 |K| on the GPU)
        lim = (_gamma(n_r) * bound).tocsr()
        slack = 1e-13 * np.abs(ref["K"]).max()
        excess = (err - lim).tocsr()
        ratio = (err.multiply(lim.power(-1))).max() if lim.nnz else 0.0
        assert excess.nnz == 0 or excess.data.max() <= slack, (elem, dim, model, split, ratio)
        e_rel = rel_fro(K32, ref["K"])
        print(f"\n{elem}{dim}d model {model} split {split}: |K32-K|_F/|K|_F = {e_rel:.2e}, "
              f"max err/bound = {ratio:.2e}")
        assert e_rel < 1e-5
    ctx.close()


@pytest.mark.parametrize("method", [1, 2, 3])
@pytest.mark.parametrize("model,elem,dim", [(VM_ISO, "P2", 2), (DP, "P2", 2), (VM_ISO, "Q1", 3), (DP, "P2", 3)])
def test_mixed_krylov_solve(ep, model, elem, dim, method):
    """FP32 CG / BiCGStab / GMRES on the FP32 tangent vs a direct solve of that same matrix."""
    if method == 1 and model == DP:
        pytest.skip("CG needs a symmetric tangent")
    import scipy.sparse.linalg as spla
    prob = small_problem(elem, dim, SIZES[(elem, dim)] + 1, model, seed=4)
    u, ep_, hard = fed_iterate(prob, seed=5, dilate=(1.0e-3 if model == DP else 0.0))
    ctx = ep.Context.from_problem(prob)
    ctx.set(ep.EP_PLASTIC_STRAIN, ep_)
    ctx.set(ep.EP_HARDENING, hard)
    ctx.assemble(u, precision=ep.EP_MIXED)
    K32 = ctx.K_csr(f32=True)
    free = prob.dirichlet == 0
    b = np.random.default_rng(6).standard_normal(prob.n_dof) * free
    xr = np.zeros(prob.n_dof)
    xr[free] = spla.spsolve(K32[free][:, free].tocsc(), b[free])
    for precond in (0, 1, 2):
        x, its, rel = ctx.linear_solve(b, ep.default_opts(krylov=method, krylov_rtol=1e-5, krylov_maxit=20000,
                                                         precond=precond, precision=ep.EP_MIXED))
        assert its > 0 and rel <= 1e-5
        assert np.all(x[~free] == 0.0)
        true_rel = np.linalg.norm((b - K32 @ x)[free]) / np.linalg.norm(b[free])
        print(f"\n{elem}{dim}d model {model} method {method} precond {precond}: its {its} "
              f"true residual {true_rel:.2e} error {np.linalg.norm(x - xr) / np.linalg.norm(xr):.2e}")
        # the recursively updated residual of BiCGStab drifts from the true one by O(u32) times
        # its largest intermediate residual (Jacobi: erratic convergence), so its bound is looser
        assert true_rel < (1e-3 if method == 2 else 1e-4)
    ctx.close()


def _mixed_path_parity(ep, prob, tol_newton, **kw):
    from oracle.newton import OracleSolver
    ctx = ep.Context.from_problem(prob)
    reps = ctx.solve_load_path(prob.zeta, ep.default_opts(newton_rtol=tol_newton, precision=ep.EP_MIXED, **kw))
    ref = OracleSolver(prob)
    ref.solve_path(tol=min(tol_newton, 1e-13))
    u = ctx.get(ep.EP_U)
    e_u = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    e_s = rel_max(ctx.get(ep.EP_STRESS), ref.stress)
    print(f"\n{prob.name} mixed: |u-u_or|/|u_or| = {e_u:.2e}, max|sig-sig_or|/max|sig_or| = {e_s:.2e}, "
          f"Newton its {[r.newton_its for r in reps]}")
    assert e_u < TOL and e_s < TOL
    assert np.array_equal(ctx.get(ep.EP_PLASTIC_FLAG), ref.plastic.astype(np.uint8))
    assert all(r.rel_resid <= tol_newton for r in reps)
    ctx.close()
    return reps


def test_mixed_load_path_p1_von_mises_column(ep):
    from synthetic import p1_plane_vm
    prob = p1_plane_vm()
    reps = _mixed_path_parity(ep, prob, 1e-12)
    assert reps[-1].n_plastic == prob.mesh.n_elem


def test_mixed_load_path_p2_drucker_prager_column(ep):
    from synthetic import p2_plane_dp
    prob = p2_plane_dp(n=12, n_steps=20, load_fraction=0.98)
    _mixed_path_parity(ep, prob, 1e-13, newton_maxit=40)


def test_mixed_load_path_q1_cube(ep):
    from synthetic import q1_cube_vm
    _mixed_path_parity(ep, q1_cube_vm(n=4, n_steps=6), 1e-12)


def test_mixed_load_path_p2_tet_strip(ep):
    from synthetic import p2_tet_strip_dp
    _mixed_path_parity(ep, p2_tet_strip_dp(n=3, n_steps=6), 1e-12)


def test_mixed_full_size_p2_matches_fp64(ep):
    """The 256x256 P2 column to 0.95 t_lim (40 steps) in both precisions: the same converged path."""
    from oracle.newton import homogeneous_column
    from synthetic import p2_plane_dp
    prob = p2_plane_dp(load_fraction=0.95)
    out = {}
    for prec in (ep.EP_FP64, ep.EP_MIXED):
        ctx = ep.Context.from_problem(prob)
        reps = ctx.solve_load_path(prob.zeta, ep.default_opts(newton_rtol=1e-10, precision=prec))
        out[prec] = (ctx.get(ep.EP_U), ctx.get(ep.EP_STRESS), reps)
        ctx.close()
        assert all(r.rel_resid <= 1e-10 for r in reps)
    u64, s64, r64 = out[ep.EP_FP64]
    u32, s32, r32 = out[ep.EP_MIXED]
    hom = homogeneous_column(prob.material, prob.zeta * prob.extra["load_fraction"] * prob.extra["t_lim"])
    want = np.repeat(hom[-1]["stress"][:, None], s32.shape[1], axis=1)
    e_u = np.linalg.norm(u32 - u64) / np.linalg.norm(u64)
    print(f"\nmixed vs FP64: |du|/|u| = {e_u:.2e}; stress vs one-point oracle: FP64 {rel_max(s64, want):.2e}, "
          f"mixed {rel_max(s32, want):.2e}; Newton its FP64 {sum(r.newton_its for r in r64)}, "
          f"mixed {sum(r.newton_its for r in r32)}; Krylov its FP64 {sum(r.krylov_its for r in r64)}, "
          f"mixed {sum(r.krylov_its for r in r32)}")
    assert rel_max(s32, want) < 1e-9
    assert e_u < 1e-8
