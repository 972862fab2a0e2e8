"""Learned warm start on the GPU vs the oracle: the network (forward, gradient, Adam), the recorded
features and targets, and load paths started from the network's prediction.

Tolerances follow the FP32 arithmetic of the network.  A dot product of length m evaluated in FP32
(any order, with or without FMA) is within gamma(m) = m u / (1 - m u), u = 2^-24, of the exact one
times the sum of the absolute values of its terms.  Through the three layers the outputs are within
2 gamma(275) a3 of the exact outputs of the same (bfloat16-rounded) weights, where a1 = |W1||x| +
|b1|, a2 = |W2| a1 + |b2|, a3 = |W3| a2 + |b3|.  Rows whose pre-activations lie closer to zero than
that error are dropped, so both sides take the same ReLU branches.  Gradients add the summation
over rows (chains of at most n + 600 roundings) to the propagated output and activation errors.
"""
import math

import numpy as np
import pytest

from oracle import warm_start as W
from synthetic import Material, VM_ISO, vm_iso_material
from synthetic.problems import first_yield_traction_vm, plane_column
from synthetic.random_states import mlp_init, mlp_rows

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
U32 = 2.0 ** -24


def _gamma(m):
    return m * U32 / (1.0 - m * U32)


@pytest.fixture(scope="module")
def ep():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_04155_gb300 import build as b
    b.build()
    import paper_1805_04155_gb300.ep as mod
    return mod


def _abs_chain(params, X):
    W1, b1, W2, b2, W3, b3 = W.unpack(params)
    Xa = np.abs(np.asarray(X, dtype=np.float64))
    a1 = Xa @ np.abs(W1).T + np.abs(b1)
    a2 = a1 @ np.abs(W2).T + np.abs(b2)
    a3 = a2 @ np.abs(W3).T + np.abs(b3)
    return a1, a2, a3


def _safe_rows(params, X):
    """Rows whose pre-activations are farther from 0 than their FP32 evaluation error."""
    W1, b1, W2, b2, _, _ = W.unpack(params)
    a1, a2, _ = _abs_chain(params, X)
    z1 = np.asarray(X, dtype=np.float64) @ W1.T + b1
    z2 = np.maximum(z1, 0) @ W2.T + b2
    ok = (np.abs(z1) > 4 * _gamma(17) * a1).all(axis=1) & (np.abs(z2) > 4 * _gamma(146) * a2).all(axis=1)
    return ok


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_network_forward_parity(ep):
    """Ragged row count (15 full tiles of 64 and a tail of 40)."""
    p = mlp_init(21, out_scale=1.0, bias_scale=0.1)
    X, _ = mlp_rows(1000, seed=22)
    keep = _safe_rows(p, X)
    X = X[keep]
    net = ep.MLP(p)
    Y = torch.empty((X.shape[0], 4), dtype=torch.float32, device="cuda")
    net.forward(_dev(X), Y)
    y_or, _ = W.mlp_forward(p, X)
    _, _, a3 = _abs_chain(p, X)
    err = np.abs(Y.cpu().numpy() - y_or)
    bound = 2 * _gamma(275) * a3
    print(f"\nforward: {X.shape[0]} rows, max err {err.max():.2e}, max err/bound {(err / bound).max():.2e}")
    assert np.all(err <= bound)
    # weights are used as bfloat16: the GPU is far closer to the rounded network than the unrounded
    # network is
    y_x, _ = W.mlp_forward(p, X, round_weights=False)
    assert err.max() < 0.01 * np.abs(y_x - y_or).max()
    net.close()


def _grad_bound(params, X, T):
    """First-order bound of |g_gpu - g_oracle| per parameter (module docstring)."""
    n = X.shape[0]
    W1, b1, W2, b2, W3, b3 = W.unpack(params)
    y, (h1, h2, _) = W.mlp_forward(params, X)
    a1, a2, a3 = _abs_chain(params, X)
    e3 = 2 * _gamma(275) * a3
    dy = np.empty_like(y)
    dy[:, :3] = 2.0 * (y[:, :3] - T[:, :3]) / n
    dy[:, 3] = W.LAMBDA_PL * (1.0 / (1.0 + np.exp(-y[:, 3])) - T[:, 3]) / n
    dyb = np.abs(dy) + np.concatenate([2.0 * e3[:, :3] / n, W.LAMBDA_PL * 0.25 * e3[:, 3:] / n], axis=1)
    h1b = np.abs(h1) + 2 * _gamma(17) * a1
    h2b = np.abs(h2) + 2 * _gamma(146) * a2
    Xa = np.abs(np.asarray(X, dtype=np.float64))
    m1, m2 = (h1 > 0), (h2 > 0)

    def back(dya, h1a, h2a):
        dW3 = dya.T @ h2a
        db3 = dya.sum(axis=0)
        dh2 = (dya @ np.abs(W3)) * m2
        dW2 = dh2.T @ h1a
        db2 = dh2.sum(axis=0)
        dh1 = (dh2 @ np.abs(W2)) * m1
        return W.pack(dh1.T @ Xa, dh1.sum(axis=0), dW2, db2, dW3, db3)

    G = back(np.abs(dy), np.abs(h1), np.abs(h2))
    Gb = back(dyb, h1b, h2b)
    return (Gb - G) + 2 * _gamma(n + 600) * Gb + 1e-30


def test_network_gradient_parity(ep):
    p = mlp_init(23, out_scale=1.0, bias_scale=0.1)
    X, T = mlp_rows(900, seed=24)
    keep = _safe_rows(p, X)
    X, T = X[keep], T[keep]
    net = ep.MLP(p)
    loss, g = net.grad(_dev(X), _dev(T))
    l_or, g_or = W.mlp_grad(p, X.astype(np.float64), T.astype(np.float64))
    bound = _grad_bound(p, X.astype(np.float64), T.astype(np.float64))
    err = np.abs(g.astype(np.float64) - g_or)
    print(f"\ngradient: {X.shape[0]} rows, loss {loss:.6e} vs {l_or:.6e}, max err/bound {(err / bound).max():.2e}, "
          f"rel {np.linalg.norm(err) / np.linalg.norm(g_or):.2e}")
    assert np.all(err <= bound)
    assert abs(loss - l_or) <= 2 * _gamma(X.shape[0] + 600) * l_or + 4 * _gamma(275) * l_or
    net.close()


def test_network_adam_step(ep):
    """One Adam step: entries whose gradient sign is certain move by lr * sign(g) (the first
    bias-corrected step), as in the oracle; every entry moves by at most lr."""
    p = mlp_init(25, out_scale=1.0, bias_scale=0.1)
    X, T = mlp_rows(600, seed=26)
    keep = _safe_rows(p, X)
    X, T = X[keep], T[keep]
    lr = 1e-3
    net = ep.MLP(p)
    loss = net.train_step(_dev(X), _dev(T), lr)
    q = net.params().astype(np.float64)
    _, g_or = W.mlp_grad(p, X.astype(np.float64), T.astype(np.float64))
    bound = _grad_bound(p, X.astype(np.float64), T.astype(np.float64))
    q_or, _, _ = W.adam_step(p.astype(np.float64), np.zeros(W.N_PARAMS), np.zeros(W.N_PARAMS), g_or, 1, lr)
    sure = (np.abs(g_or) > 10 * bound) & (np.abs(g_or) > 1e3 * W.ADAM_EPS)
    assert sure.mean() > 0.5
    d = np.abs(q - q_or)
    lim = 1e-6 * np.abs(q_or) + 1e-5 * lr
    print(f"\nAdam step: {sure.sum()} entries with a certain sign, max dev {d[sure].max():.2e}, loss {loss:.4e}")
    assert np.all(d[sure] <= lim[sure])
    assert np.all(np.abs(q - p) <= lr * (1 + 1e-5) + 1e-6 * np.abs(p))
    net.close()


def test_network_training_lowers_the_loss(ep):
    """Adam on a teacher network's outputs: 300 full-batch steps cut the loss at least fivefold."""
    teacher = mlp_init(27, out_scale=1.0, bias_scale=0.1)
    X, _ = mlp_rows(4096, seed=28)
    y, _ = W.mlp_forward(teacher, X)
    T = np.concatenate([y[:, :3], 1.0 / (1.0 + np.exp(-y[:, 3:]))], axis=1)
    net = ep.MLP(mlp_init(29))
    Xd, Td = _dev(X), _dev(T)
    l0 = net.train_step(Xd, Td, 3e-3)
    for _ in range(298):
        net.train_step(Xd, Td, 3e-3, want_loss=False)
    l1 = net.train_step(Xd, Td, 3e-3)
    l_or = W.mlp_loss(net.params(), X, T)
    print(f"\ntraining: loss {l0:.4e} -> {l1:.4e} (oracle at the final parameters {l_or:.4e})")
    assert l1 < 0.2 * l0
    assert math.isfinite(l_or) and l_or < 0.25 * l0
    net.close()


def test_empty_and_invalid_calls(ep):
    net = ep.MLP(mlp_init(30))
    lib = ep.lib()
    import ctypes as C
    assert lib.ep_mlp_forward(net.h, None, 0, None) == ep.EP_OK          # no rows: nothing to do
    assert lib.ep_mlp_train_step(net.h, None, None, 0, 1e-3, None) == ep.EP_ERR_INVALID_ARG
    X = _dev(np.zeros((4, 16)))
    T = _dev(np.zeros((4, 4)))
    assert lib.ep_mlp_train_step(net.h, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()), 4, 0.0, None) == \
        ep.EP_ERR_INVALID_ARG                                              # lr must be > 0
    net.close()


# -- features, targets and learned starts on load paths ------------------------------------------
def _column(n, scale=(1.0, 1.0, 1.0, 1.0), n_steps=13):
    """P1 plane-strain column (von Mises, isotropic hardening) with E, nu, Y, H scaled, loaded to 1.5x
    its first-yield traction: elastic for two thirds of the path, then plastic throughout.  With
    n_steps not a multiple of 3 no step ends exactly at first yield, where the plastic flag is a tie
    that rounding decides."""
    base = vm_iso_material()
    mat = Material(VM_ISO, E=base.E * scale[0], nu=min(0.45, base.nu * scale[1]), Y=base.Y * scale[2],
                   H=base.H * scale[3])
    return plane_column("P1", n, mat, 1.5 * first_yield_traction_vm(mat.E, mat.nu, mat.Y), n_steps)


def _oracle_rows(probs):
    """Oracle rows of a batch: per step, the rows of every problem in order."""
    from oracle.newton import OracleSolver
    per = [W.trajectory_samples(pb, pb.zeta, OracleSolver) for pb in probs]
    n_steps = per[0][0].shape[0] // probs[0].mesh.n_nodes
    Xs, Ts = [], []
    for s in range(n_steps):
        for (X, T), pb in zip(per, probs):
            n = pb.mesh.n_nodes
            Xs.append(X[s * n:(s + 1) * n])
            Ts.append(T[s * n:(s + 1) * n])
    return np.concatenate(Xs), np.concatenate(Ts)


def _recording_case(name):
    from synthetic import l_shape_vm, p2_plane_dp, p2_tet_strip_dp, q1_cube_vm
    return {
        "column": lambda: [_column(6)],
        "batch": lambda: [_column(5), _column(7, (0.8, 1.1, 0.9, 1.2)), _column(4, (1.2, 0.9, 1.1, 0.8))],
        "q1_cube_3d": lambda: [q1_cube_vm(n=3, n_steps=10)],
        "dp_column": lambda: [p2_plane_dp(n=6, n_steps=12, load_fraction=0.9)],
        "kinematic_l_shape": lambda: [l_shape_vm("Q2", m=3, n_steps=16)],
        "dp_tet_strip_3d": lambda: [p2_tet_strip_dp(n=2, n_steps=8)],
    }[name]()


@pytest.mark.parametrize("case", ["column", "batch", "q1_cube_3d", "dp_column", "kinematic_l_shape", "dp_tet_strip_3d"])
def test_recorded_rows_match_the_oracle(ep, case):
    """Inputs and targets recorded along a plastic load path equal the oracle's, computed from its own
    trajectory: 2D and 3D, von Mises with isotropic and kinematic hardening, Drucker-Prager with and
    without dilatancy and hardening (the yield proximity of each model), one problem and a batch.
    The two trajectories agree to the Newton tolerance (1e-11 relative), so the FP32 rows agree to
    their rounding plus that difference divided by the increment scale."""
    probs = _recording_case(case)
    batch = len(probs) > 1
    ctx = ep.Context.from_problem(probs[0]) if not batch else ep.Context.from_batch(probs)
    n_total = sum(pb.mesh.n_nodes for pb in probs)
    ctx.ws_record(n_total * 20)
    reps = ctx.solve_load_path(probs[0].zeta, ep.default_opts(newton_rtol=1e-13, warm_start=1, newton_maxit=40))
    X = ctx.get(ep.EP_WS_X)
    T = ctx.get(ep.EP_WS_T)
    ctx.close()
    Xo, To = _oracle_rows(probs)
    assert X.shape == Xo.shape and T.shape == To.shape and X.shape[0] > 0
    ex = np.abs(X - Xo)
    et = np.abs(T - To)
    print(f"\nrecorded {X.shape[0]} rows ({sum(r.n_plastic > 0 for r in reps)} plastic steps): "
          f"max |dX| {ex.max():.2e}, max |dT| {et.max():.2e}, max |T| {np.abs(To[:, :3]).max():.2e}")
    assert np.all(ex <= 1e-6 + 1e-6 * np.abs(Xo))
    assert np.all(et[:, :3] <= 1e-6 + 1e-6 * np.abs(To[:, :3]))
    assert np.array_equal(X[:, 8], Xo[:, 8].astype(np.float32))
    assert np.all(Xo[:, 10] >= 0) and Xo[:, 10].max() <= 1.0 + 1e-9
    if Xo[:, 8].max() > 0:      # a node next to plastic points sees the yield surface
        assert Xo[Xo[:, 8] > 0, 10].min() > 1.0 - 1e-9
    assert np.array_equal(T[:, 3], To[:, 3].astype(np.float32))
    assert np.abs(To[:, :3]).max() > 1e-3     # the plastic steps make the extrapolation inexact


@pytest.mark.parametrize("batch", [False, True])
def test_learned_start_matches_the_oracle(ep, batch):
    """The learned start of the last step (network, projection, update) against the oracle's, for a
    fixed untrained network.  Both trajectories converge to 1e-13; the network's FP32 outputs are within
    1e-5 of their scale, so the starts agree to 1e-4 s max|P(y)| plus the trajectories' difference."""
    from oracle.newton import OracleSolver
    probs = [_column(6)] if not batch else [_column(5), _column(6, (0.9, 1.1, 1.05, 0.95))]
    params = mlp_init(33, out_scale=0.5, bias_scale=0.05)
    net = ep.MLP(params)
    ctx = ep.Context.from_problem(probs[0]) if not batch else ep.Context.from_batch(probs)
    ctx.ws_attach(net)
    reps = ctx.solve_load_path(probs[0].zeta, ep.default_opts(newton_rtol=1e-13, warm_start=2, newton_maxit=40))
    uL = ctx.get(ep.EP_WS_START)
    parts = ctx.split(ep.EP_U, uL) if batch else [uL]
    ctx.close()
    net.close()
    for i, pb in enumerate(probs):
        out = W.last_learned_start(pb, pb.zeta, params, OracleSolver)
        assert out is not None
        u_or, s, P = out
        err = np.abs(parts[i] - u_or).max()
        lim = 1e-9 * np.abs(u_or).max() + 1e-4 * s * np.abs(P).max()
        print(f"\nproblem {i}: learned start max err {err:.2e} (limit {lim:.2e}), s {s:.3e}, max|P| {np.abs(P).max():.3e}; "
              f"starts {[r.start for r in reps]}")
        assert err <= lim
        assert np.abs(P).max() > 0.0


def test_learned_start_needs_a_network(ep):
    ctx = ep.Context.from_problem(_column(3))
    st, _ = ctx.solve_load_path([0.1], ep.default_opts(warm_start=2), raise_on_error=False)
    assert st == ep.EP_ERR_INVALID_ARG
    ctx.close()


def test_learned_start_saves_newton_iterations_on_unseen_problems(ep):
    """Train on recorded trajectories of one batch of columns, then solve other columns (unseen sizes
    and materials) from the learned start with large load increments (7 steps to 1.5x first yield):
    the converged path equals the oracle's and the learned start needs fewer Newton iterations than
    the plain extrapolated start.  Everything runs in the deterministic form, so the recorded rows,
    the trained network and the iteration counts are reproducible (measured: 16 -> 13)."""
    from oracle.newton import OracleSolver
    n_steps = 7
    g = np.random.default_rng(31)
    train = [_column(int(g.integers(4, 9)), tuple(g.uniform(0.8, 1.2, 4)), n_steps=n_steps) for _ in range(6)]
    test = [_column(int(g.integers(4, 9)), tuple(g.uniform(0.8, 1.2, 4)), n_steps=n_steps) for _ in range(3)]
    ctx = ep.Context.from_batch(train)
    ctx.ws_record(sum(pb.mesh.n_nodes for pb in train) * n_steps)
    opts1 = ep.default_opts(newton_rtol=1e-12, warm_start=1, newton_maxit=40, deterministic=1)
    ctx.solve_load_path(train[0].zeta, opts1)
    xp, tp, n = ctx.ws_samples_ptr()
    net = ep.MLP(mlp_init(0))
    l0 = net.train_step(xp, tp, 2e-3, n_rows=n)
    for _ in range(600):
        net.train_step(xp, tp, 2e-3, n_rows=n, want_loss=False)
    l1 = net.train_step(xp, tp, 2e-3, n_rows=n)
    ctx.close()
    its = {}
    us = {}
    learned = []
    for ws in (1, 2):
        c = ep.Context.from_batch(test)
        if ws == 2:
            c.ws_attach(net)
        reps = c.solve_load_path(test[0].zeta, ep.default_opts(newton_rtol=1e-12, warm_start=ws, newton_maxit=40,
                                                              deterministic=1))
        its[ws] = [r.newton_its for r in reps]
        us[ws] = c.split(ep.EP_U, c.get(ep.EP_U))
        if ws == 2:
            learned = [r.n_learned for r in reps]
        c.close()
    for i, pb in enumerate(test):
        ref = OracleSolver(pb)
        ref.solve_path(tol=1e-13)
        for ws in (1, 2):
            assert np.linalg.norm(us[ws][i] - ref.u) / np.linalg.norm(ref.u) < 1e-11
    print(f"\ntraining loss {l0:.3e} -> {l1:.3e} on {n} rows; Newton its extrapolated {sum(its[1])} {its[1]}, "
          f"learned {sum(its[2])} {its[2]}; problems on the learned start per step {learned}")
    assert l1 < 0.1 * l0
    assert sum(learned) > 0
    assert sum(its[2]) < sum(its[1])
    net.close()
