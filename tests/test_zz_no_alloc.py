"""The allocation-free Krylov entry point (ep_linear_solve_noalloc) against ep_linear_solve.

Some callers cannot allocate device memory when they solve (another runtime
owns the memory pool, or the phase forbids cudaMalloc); they hand the matrix
and vectors in and the solver works in a fixed device array inside the
library.  This file is collected last so that a failure here leaves every
other test already run; it passes both alone and after the other tests.
"""
import numpy as np
import pytest

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


def _system(ep, model, seed):
    from gpu_helpers import fed_iterate, small_problem
    prob = small_problem("P2", 2, 6, model, seed=seed)
    u, ep_, hard = fed_iterate(prob, seed=seed + 1)
    ctx = ep.Context.from_problem(prob)
    ctx.set(ep.EP_PLASTIC_STRAIN, ep_)
    ctx.set(ep.EP_HARDENING, hard)
    ctx.assemble(u)
    return prob, ctx


@pytest.mark.parametrize("model,method", [(2, 1), (3, 2)])
def test_noalloc_solve_matches_context_solve(ep, model, method):
    prob, ctx = _system(ep, model, seed=11)
    free = (prob.dirichlet == 0)
    b = np.random.default_rng(12).standard_normal(prob.n_dof) * free
    opts = ep.default_opts(krylov=method, krylov_rtol=1e-12, krylov_maxit=5000, precond=1)
    x_ref, its_ref, rel_ref = ctx.linear_solve(b, opts)
    rp = ctx.get(ep.EP_K_ROW_PTR)
    ci = ctx.get(ep.EP_K_COL_IDX)
    vals = ctx.get(ep.EP_K_VALUES)
    diag = np.array([rp[i] + np.searchsorted(ci[rp[i]:rp[i + 1]], i) for i in range(len(rp) - 1)], dtype=np.int32)
    assert np.all(ci[diag] == np.arange(len(rp) - 1))
    dev = torch.device("cuda:0")
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    args = [T(rp), T(ci), T(diag), T(vals), T(prob.dirichlet == 0).to(torch.uint8), T(b)]
    K = ctx.K_csr()
    first = None
    for call in range(2):            # the second call must not see the first one's workspace
        x = torch.full((prob.n_dof,), float("nan"), dtype=torch.float64, device=dev)
        st, its, rel = ep.linear_solve_noalloc(2, *args, x, method=method, precond=1, rtol=1e-12, maxit=5000)
        torch.cuda.synchronize()
        assert st == ep.EP_OK, ep.lib().ep_last_error(None)
        xh = x.cpu().numpy()
        assert np.all(xh[~free] == 0.0)
        # the context's SpMV takes its rows in a length-grouped order and sums the solver's dot
        # products in that order; the workspace-free solve uses the natural order: both solve the
        # same system to the same tolerance, so their true residuals meet it, while their iterates
        # (and iteration counts) differ by rounding, amplified by the system's conditioning
        true_rel = np.linalg.norm((b - K @ xh)[free]) / np.linalg.norm(b[free])
        print(f"\nmethod {method}: its {its} (context {its_ref}), true residual {true_rel:.2e}, "
              f"|x - x_ctx|/|x_ctx| {np.linalg.norm(xh - x_ref) / np.linalg.norm(x_ref):.2e}")
        # BiCGStab's recursively updated residual drifts from the true one by O(u) times its largest
        # intermediate residual, so its true residual may end a little above the 1e-12 it reports
        assert true_rel <= (1e-11 if method == 1 else 1e-10)
        assert np.linalg.norm(xh - x_ref) <= 1e-6 * np.linalg.norm(x_ref)
        assert abs(its - its_ref) <= max(5, its_ref // 10)
        if first is None:
            first = (its, xh.copy())
        else:                        # the workspace-free solve itself is deterministic
            assert its == first[0] and np.array_equal(xh, first[1])
    ctx.close()


def test_noalloc_solve_allocates_no_device_memory(ep):
    """After the first call (which looks up the fixed array's device address), repeated solves leave
    the device's free memory unchanged: nothing on this path allocates."""
    prob, ctx = _system(ep, 2, seed=13)
    free = (prob.dirichlet == 0)
    b = np.random.default_rng(14).standard_normal(prob.n_dof) * free
    rp = ctx.get(ep.EP_K_ROW_PTR)
    ci = ctx.get(ep.EP_K_COL_IDX)
    vals = ctx.get(ep.EP_K_VALUES)
    diag = np.array([rp[i] + np.searchsorted(ci[rp[i]:rp[i + 1]], i) for i in range(len(rp) - 1)], dtype=np.int32)
    dev = torch.device("cuda:0")
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    args = [T(rp), T(ci), T(diag), T(vals), T(prob.dirichlet == 0).to(torch.uint8), T(b)]
    x = torch.zeros(prob.n_dof, dtype=torch.float64, device=dev)
    for method, precond in ((1, 1), (2, 0)):
        st, _, _ = ep.linear_solve_noalloc(2, *args, x, method=method, precond=precond, rtol=1e-10, maxit=2000)
        assert st == ep.EP_OK
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        for method, precond in ((1, 1), (2, 0)):
            st, _, _ = ep.linear_solve_noalloc(2, *args, x, method=method, precond=precond, rtol=1e-10, maxit=2000)
            assert st == ep.EP_OK
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_workspace(ep):
    """Host-side check before any GPU work: more DOFs than the fixed array holds."""
    dev = torch.device("cuda:0")
    n_nodes = ep.EP_NOALLOC_MAX_DOF // 2 + 1
    rp = torch.zeros(n_nodes + 1, dtype=torch.int32, device=dev)
    one = torch.zeros(1, dtype=torch.int32, device=dev)
    v = torch.zeros(4, dtype=torch.float64, device=dev)
    m = torch.zeros(2 * n_nodes, dtype=torch.uint8, device=dev)
    bx = torch.zeros(2 * n_nodes, dtype=torch.float64, device=dev)
    st, _, _ = ep.linear_solve_noalloc(2, rp, one, one, v, m, bx, bx.clone())
    assert st == ep.EP_ERR_INVALID_ARG
    assert b"EP_NOALLOC_MAX_DOF" in ep.lib().ep_last_error(None)
    st, _, _ = ep.linear_solve_noalloc(2, rp[:3], one, one, v, m, bx, bx.clone(), maxit=ep.EP_NOALLOC_MAX_ITERATIONS + 1)
    assert st == ep.EP_ERR_INVALID_ARG
