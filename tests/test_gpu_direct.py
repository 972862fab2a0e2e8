"""The sparse LU (precond 3: multifrontal, nested-dissection order, FP64 fronts with static
pivoting, refined by FP64 GMRES) against sparse direct solves and the oracle, and the Newton loop's
switch to it near the limit load of the nonassociated Drucker-Prager column (Section 2.3)."""
import numpy as np
import pytest

from gpu_helpers import ALL_ELEMS, fed_iterate, rel_max, small_problem
from synthetic import DP, VM_ISO

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


SIZES = {("P1", 2): 10, ("P2", 2): 8, ("Q1", 2): 10, ("Q2", 2): 6, ("P1", 3): 4, ("P2", 3): 3, ("Q1", 3): 4,
         ("Q2", 3): 3}


@pytest.mark.parametrize("model", [VM_ISO, DP])
@pytest.mark.parametrize("elem,dim", ALL_ELEMS)
def test_sparse_lu_solve_matches_a_direct_solve(ep, elem, dim, model):
    """GMRES with the sparse LU reaches 1e-13 within a few iterations on a plastic tangent of every
    element type and matches scipy's sparse direct solve."""
    import scipy.sparse.linalg as spla
    prob = small_problem(elem, dim, SIZES[(elem, dim)], model, seed=11)
    u, ep_, hard = fed_iterate(prob, seed=12, dilate=(1.0e-3 if model == DP else 0.0))
    ctx = ep.Context.from_problem(prob)
    ctx.set(ep.EP_PLASTIC_STRAIN, ep_)
    ctx.set(ep.EP_HARDENING, hard)
    ctx.assemble(u)
    K = ctx.K_csr()
    free = prob.dirichlet == 0
    b = np.random.default_rng(13).standard_normal(prob.n_dof) * free
    x, its, rel = ctx.linear_solve(b, ep.default_opts(krylov=3, krylov_rtol=1e-13, krylov_maxit=200, precond=3))
    xr = np.zeros(prob.n_dof)
    xr[free] = spla.spsolve(K[free][:, free].tocsc(), b[free])
    print(f"\n{elem}-{dim}d: {its} GMRES iterations, |x - x_direct|/|x_direct| = "
          f"{np.linalg.norm(x - xr) / np.linalg.norm(xr):.2e}")
    assert 0 < its <= 12 and rel <= 1e-13
    assert np.all(x[~free] == 0.0)
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-9
    ctx.close()


def test_sparse_lu_on_a_batch_of_disconnected_problems(ep):
    """A batch context (disconnected meshes with overlapping coordinates in one pattern)."""
    import scipy.sparse.linalg as spla
    from synthetic import batch_problems
    probs = batch_problems(seed=14, n_problems=3, sizes=(5, 9), families=["P2"] * 3, n_steps=4)["P2"]
    ctx = ep.Context.from_batch(probs)
    n = sum(pb.n_dof for pb in probs)
    ctx.assemble(np.zeros(n))
    K = ctx.K_csr()
    free = np.concatenate([pb.dirichlet == 0 for pb in probs])
    b = np.random.default_rng(15).standard_normal(n) * free
    x, its, rel = ctx.linear_solve(b, ep.default_opts(krylov=3, krylov_rtol=1e-13, krylov_maxit=200, precond=3))
    xr = np.zeros(n)
    xr[free] = spla.spsolve(K[free][:, free].tocsc(), b[free])
    assert 0 < its <= 12 and rel <= 1e-13
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-9
    ctx.close()


def _path_vs_oracle(ep, prob, opts, tol_newton, tol_ep=TOL):
    from oracle.newton import OracleSolver
    ctx = ep.Context.from_problem(prob)
    reps = ctx.solve_load_path(prob.zeta, opts)
    ref = OracleSolver(prob)
    ref.solve_path(tol=tol_newton)
    u, sig, epl = ctx.get(ep.EP_U), ctx.get(ep.EP_STRESS), ctx.get(ep.EP_PLASTIC_STRAIN)
    fl = ctx.get(ep.EP_PLASTIC_FLAG)
    ctx.close()
    e_u = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    print(f"\n{prob.name}: |u - u_oracle|/|u_oracle| = {e_u:.2e}, stress {rel_max(sig, ref.stress):.2e}, "
          f"direct steps {sum(r.direct for r in reps)}, Krylov iterations {sum(r.krylov_its for r in reps)}")
    assert e_u < TOL
    assert rel_max(sig, ref.stress) < TOL
    assert rel_max(epl, ref.ep) < tol_ep
    assert np.array_equal(fl, ref.plastic.astype(np.uint8))
    assert all(r.rel_resid <= tol_newton for r in reps)
    return reps


def test_load_path_p2_column_to_098_with_the_sparse_lu(ep):
    """precond 3 from the first step: the nonassociated column to 0.98 of the limit traction."""
    from synthetic import p2_plane_dp
    prob = p2_plane_dp(n=12, n_steps=20, load_fraction=0.98)
    reps = _path_vs_oracle(ep, prob, ep.default_opts(newton_rtol=1e-13, newton_maxit=40, precond=3), 1e-13)
    assert all(r.direct == 1 for r in reps if r.krylov_its > 0)
    assert reps[-1].n_plastic == prob.mesh.n_elem * 7


def test_newton_switches_to_the_sparse_lu_where_the_vcycle_stalls(ep):
    """Default options (V-cycle GMRES): near the limit load the V-cycle stalls and the rest of the path
    is solved with the sparse LU; the path matches the oracle.  At 32x32 cells the FP64 residual of
    the last step's nearly singular state does not go below about 1.3e-13 (measured), so both sides
    solve to 1e-12 here; the plastic strain, the difference of the total strain and the elastic
    strain of the stress, keeps 1e-10 of its largest entry at that residual (measured 3e-11)."""
    from synthetic import p2_plane_dp
    prob = p2_plane_dp(n=32, n_steps=40, load_fraction=0.98)
    reps = _path_vs_oracle(ep, prob, ep.default_opts(newton_rtol=1e-12, newton_maxit=40), 1e-12, tol_ep=1e-10)
    assert reps[-1].direct == 1
    assert reps[0].direct == 0


def test_full_size_p2_column_to_098_of_the_limit_load(ep):
    """The 256x256 P2 column (917 504 points) to 0.98 t_lim in 40 steps: the last step is solved with
    the sparse LU after the V-cycle stalls, again from its start iterate, every Newton system to
    1e-13 like the oracle's direct solves (the last step's Newton residuals then equal the oracle's:
    5.3e-3, 1.8e-3, 2.1e-4, 3.1e-6, 7.1e-10, measured).

    Near the limit load the state's distance from the homogeneous column is set by the residuals the
    load history was solved to (plasticity remembers them through the plastic strains, and the nearly
    singular tangent amplifies them): at 1e-10 it is 1.4e-8 (measured), and it falls with the
    residual.  So at 1e-10 the check is the solution branch (an inexact start of the last step once
    led Newton to a branch 4.5e-3 away), and at 5e-12 every point equals the one-point oracle to 1e-9."""
    from oracle.newton import homogeneous_column
    from synthetic import p2_plane_dp
    prob = p2_plane_dp(n=256, n_steps=40, load_fraction=0.98)
    hom = homogeneous_column(prob.material, prob.zeta * prob.extra["load_fraction"] * prob.extra["t_lim"])
    want = hom[-1]["stress"]
    ctx = ep.Context.from_problem(prob)
    errs = []
    for tol, bound in ((1e-10, 1e-7), (5e-12, 1e-9)):
        ctx.reset()
        reps = ctx.solve_load_path(prob.zeta, ep.default_opts(newton_rtol=tol, newton_maxit=40))
        sig = ctx.get(ep.EP_STRESS)
        flags = ctx.get(ep.EP_PLASTIC_FLAG)
        err = rel_max(sig, np.repeat(want[:, None], sig.shape[1], axis=1))
        errs.append(err)
        print(f"\nnewton_rtol {tol:.0e}: stress vs the one-point oracle {err:.2e}; Newton "
              f"{sum(r.newton_its for r in reps)} (last step {reps[-1].newton_its}), Krylov "
              f"{sum(r.krylov_its for r in reps)}, sparse-LU steps {sum(r.direct for r in reps)}, last residual "
              f"{reps[-1].rel_resid:.2e}")
        assert all(r.rel_resid <= tol for r in reps)
        assert err < bound
        assert np.all(flags == hom[-1]["plastic"])
        assert reps[-1].direct == 1 and reps[0].direct == 0
    ctx.close()
    assert errs[1] < 0.2 * errs[0]


def test_sparse_lu_refused_when_its_factors_do_not_fit(ep, monkeypatch):
    """precond 3 with the factors capped below their size: ep_linear_solve reports EP_ERR_STATE with
    the reason, and the context stays usable (a block-Jacobi solve afterwards succeeds)."""
    monkeypatch.setenv("EP_DIRECT_MAX_MB", "0")
    prob = small_problem("P2", 2, 12, DP, seed=21)
    ctx = ep.Context.from_problem(prob)
    ctx.assemble(np.zeros(prob.n_dof))
    b = np.random.default_rng(22).standard_normal(prob.n_dof) * (prob.dirichlet == 0)
    with pytest.raises(ep.EPError) as ei:
        ctx.linear_solve(b, ep.default_opts(krylov=3, krylov_rtol=1e-10, krylov_maxit=200, precond=3))
    assert ei.value.status == ep.EP_ERR_STATE and "MiB" in str(ei.value)
    x, its, rel = ctx.linear_solve(b, ep.default_opts(krylov=3, krylov_rtol=1e-10, krylov_maxit=5000, precond=1))
    assert rel <= 1e-10
    ctx.close()


def test_sparse_lu_path_repeats_bit_for_bit_in_the_deterministic_form(ep):
    """The factorisation sums in a fixed order (extend-add by child rank, no atomics): with the
    deterministic form a load path solved with the sparse LU repeats bit for bit."""
    from synthetic import p2_plane_dp
    prob = p2_plane_dp(n=12, n_steps=10, load_fraction=0.98)
    out = []
    for _ in range(2):
        ctx = ep.Context.from_problem(prob)
        ctx.solve_load_path(prob.zeta, ep.default_opts(newton_rtol=1e-12, newton_maxit=40, precond=3,
                                                       deterministic=1))
        out.append((ctx.get(ep.EP_U), ctx.get(ep.EP_STRESS)))
        ctx.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
