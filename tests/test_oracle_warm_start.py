"""Pins of the learned-warm-start oracle (features, targets, MLP, Adam) on the CPU."""
import math

import numpy as np
import pytest

from oracle import warm_start as W
from oracle.newton import OracleSolver
from synthetic import p1_plane_vm, q1_cube_vm
from synthetic.random_states import mlp_init, mlp_rows


def test_bf16_rounding_ties_to_even():
    one = 1.0
    cases = [
        (one, one),
        (one + 2.0 ** -8, one),                      # halfway between 1 and 1 + 2^-7: the even one
        (one + 3 * 2.0 ** -8, one + 2.0 ** -6),      # halfway between 1 + 2^-7 and 1 + 2^-6: the even one
        (one + 2.0 ** -8 + 2.0 ** -20, one + 2.0 ** -7),
        (-(one + 2.0 ** -8 + 2.0 ** -20), -(one + 2.0 ** -7)),
        (0.0, 0.0),
        (2.0 ** -130, 2.0 ** -130),                  # a subnormal that bfloat16 holds exactly
    ]
    x = np.array([c[0] for c in cases], dtype=np.float32)
    want = np.array([c[1] for c in cases], dtype=np.float32)
    assert np.array_equal(W.bf16_round(x), want)


def test_bf16_rounding_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(20000).astype(np.float32) * 10.0 ** np.random.default_rng(1).integers(-20, 20, 20000)
    x = x.astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(W.bf16_round(x), ref)


def test_parameter_layout():
    assert W.N_PARAMS == 19204
    p = mlp_init(0)
    assert p.shape == (W.N_PARAMS,) and p.dtype == np.float32
    W1, b1, W2, b2, W3, b3 = W.unpack(p, round_weights=False)
    assert W1.shape == (128, 16) and W2.shape == (128, 128) and W3.shape == (4, 128)
    assert np.array_equal(W.pack(W1, b1, W2, b2, W3, b3), p.astype(np.float64))


def test_forward_matches_explicit_loops():
    p = mlp_init(3, out_scale=1.0, bias_scale=0.1)
    X, _ = mlp_rows(3, seed=4)
    y, _ = W.mlp_forward(p, X)
    W1, b1, W2, b2, W3, b3 = W.unpack(p)
    for r in range(3):
        h1 = [max(0.0, sum(W1[j][i] * float(X[r][i]) for i in range(16)) + b1[j]) for j in range(128)]
        h2 = [max(0.0, sum(W2[j][i] * h1[i] for i in range(128)) + b2[j]) for j in range(128)]
        for o in range(4):
            yo = sum(W3[o][i] * h2[i] for i in range(128)) + b3[o]
            assert abs(yo - y[r, o]) <= 1e-12 * max(1.0, abs(yo))


def test_weights_are_rounded_in_the_forward_pass():
    p = mlp_init(5, out_scale=1.0)
    X, _ = mlp_rows(8, seed=6)
    y_r, _ = W.mlp_forward(p, X, round_weights=True)
    y_x, _ = W.mlp_forward(p, X, round_weights=False)
    assert np.abs(y_r - y_x).max() > 0.0
    # bfloat16 keeps 8 significant bits: the two differ by about 2^-9 of the output scale
    assert np.abs(y_r - y_x).max() < 0.05 * np.abs(y_x).max()


def test_gradient_matches_central_differences():
    p = mlp_init(7, out_scale=1.0, bias_scale=0.2).astype(np.float64)
    X, T = mlp_rows(6, seed=8)
    loss, g = W.mlp_grad(None, X, T, params_f64=p)
    assert abs(loss - W.mlp_loss(None, X, T, params_f64=p)) <= 1e-14 * abs(loss)
    rng = np.random.default_rng(9)
    blocks = [(W.OFF_W1, W.OFF_B1), (W.OFF_B1, W.OFF_W2), (W.OFF_W2, W.OFF_B2), (W.OFF_B2, W.OFF_W3),
              (W.OFF_W3, W.OFF_B3), (W.OFF_B3, W.N_PARAMS)]
    idx = np.concatenate([rng.choice(np.arange(a, b), size=min(12, b - a), replace=False) for a, b in blocks])
    gmax = np.abs(g).max()
    for i in idx:
        h = 1e-6 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (W.mlp_loss(None, X, T, params_f64=pp) - W.mlp_loss(None, X, T, params_f64=pm)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * gmax + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_adam_constant_gradient_closed_form():
    """With a constant gradient the bias-corrected moments are g and g^2 at every step, so each step
    moves a parameter by lr * g / (|g| + eps)."""
    g = np.array([1e-3, -2.0, 5e-9, 0.0, 30.0])
    p = np.array([0.5, -1.0, 2.0, 3.0, 0.0])
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    lr = 1e-2
    q = p.copy()
    for t in range(1, 8):
        q, m, v = W.adam_step(q, m, v, g, t, lr)
        want = p - lr * t * g / (np.abs(g) + W.ADAM_EPS)
        assert np.allclose(q, want, rtol=0, atol=1e-15 * t)


def test_plastic_fraction_brute_force():
    prob = p1_plane_vm(n=4, n_steps=2)
    elem = prob.mesh.elem
    n_q = 1
    rng = np.random.default_rng(10)
    flags = rng.integers(0, 3, elem.shape[0] * n_q).astype(np.int8)
    pf = W.node_plastic_fraction(elem, flags, n_q, prob.mesh.n_nodes)
    for node in range(prob.mesh.n_nodes):
        pl = tot = 0
        for e in range(elem.shape[0]):
            if node in list(elem[e]):
                pl += sum(1 for q in range(n_q) if flags[e * n_q + q] != 0)
                tot += n_q
        assert pf[node] == (pl / tot if tot else 0.0)
    assert np.all(W.node_plastic_fraction(elem, np.ones(elem.shape[0]), 1, prob.mesh.n_nodes) == 1.0)


def _elastic_path(prob, zetas):
    return W.trajectory_samples(prob, zetas, OracleSolver)


@pytest.mark.parametrize("make,dim", [(lambda: p1_plane_vm(n=4, n_steps=2), 2), (lambda: q1_cube_vm(n=2, n_steps=2), 3)])
def test_features_and_targets_on_an_elastic_path(make, dim):
    """Linear elasticity: u is linear in zeta, so the extrapolation is exact (target 0), the scaled
    increments of unequal steps stand in the ratio of their load increments, and the scaled last
    increment has unit RMS over the DOFs."""
    prob = make()
    zetas = [0.05, 0.1, 0.2, 0.25, 0.4]     # at most 0.4 x (1.5 x first yield): elastic
    X, T = _elastic_path(prob, zetas)
    n = prob.mesh.n_nodes
    assert X.shape == (2 * n, 16) and T.shape == (2 * n, 4)
    for step, (r_k, r_k1, ratio) in enumerate([(0.05 / 0.1, 0.1 / 0.05, 0.05 / 0.1), (0.15 / 0.05, 0.05 / 0.1, 0.1 / 0.05)]):
        Xs, Ts = X[step * n:(step + 1) * n], T[step * n:(step + 1) * n]
        assert np.allclose(Xs[:, 6], r_k, rtol=1e-14) and np.allclose(Xs[:, 7], r_k1, rtol=1e-14)
        # the increment before the last one is (its load increment / the last one's) times the last one
        assert np.allclose(Xs[:, 3:3 + dim], Xs[:, 0:dim] * ratio, rtol=1e-8, atol=1e-9)
        assert abs((Xs[:, 0:dim] ** 2).sum() / (n * dim) - 1.0) < 1e-12
        assert np.all(Xs[:, dim:3] == 0.0) if dim == 2 else True
        assert np.abs(Ts[:, :3]).max() < 1e-8
        assert np.all(Ts[:, 3] == 0.0) and np.all(Xs[:, 8:10] == 0.0)
        # loaded but elastic: every node sees stress below the yield limit
        assert np.all(Xs[:, 10] > 0.0) and np.all(Xs[:, 10] < 1.0)
        stat = W.static_features(prob.material, prob.dirichlet, dim)
        assert np.array_equal(Xs[:, 11:], stat)


def test_static_features_values():
    prob = p1_plane_vm(n=2, n_steps=2)
    st = W.static_features(prob.material, prob.dirichlet, 2)
    m = prob.material
    assert np.allclose(st[:, 0], m.nu) and np.allclose(st[:, 1], m.Y / m.E * 1e3)
    assert np.allclose(st[:, 2], m.H / m.E * 10) and np.all(st[:, 3] == 0) and st.shape[1] == 5
    # node 0 at the origin has both components prescribed, the top-right corner none
    assert st[0, 4] == 1.0 and st[-1, 4] == 0.0


def test_targets_and_learned_start_round_trip():
    """Feeding the targets back as the network output reproduces the converged solution."""
    prob = p1_plane_vm(n=4, n_steps=8)
    rng = np.random.default_rng(11)
    n, dim = prob.mesh.n_nodes, 2
    free = prob.dirichlet == 0
    u_k, u_ex = rng.standard_normal(n * dim) * free, rng.standard_normal(n * dim) * free
    s = 0.37
    T = W.targets(u_k, u_ex, s, np.zeros(n), free, dim)
    u_L = W.learned_start(u_ex, T, s, free, dim)
    assert np.allclose(u_L[free], u_k[free], rtol=0, atol=1e-15)
    assert np.all(u_L[~free] == u_ex[~free])


def test_adam_training_reduces_the_loss():
    p = mlp_init(12).astype(np.float64)
    X, T = mlp_rows(256, seed=13)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0 = W.mlp_loss(p.astype(np.float32), X, T)
    for t in range(1, 31):
        _, g = W.mlp_grad(p.astype(np.float32), X, T)
        p, m, v = W.adam_step(p, m, v, g, t, 1e-3)
    assert W.mlp_loss(p.astype(np.float32), X, T) < 0.9 * l0
    assert math.isfinite(l0)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("model", [0, 1, 2, 3])
def test_yield_proximity_is_one_on_the_yield_surface(model, dim):
    """After a return mapping, plastic points lie on the (current) yield surface, so their
    proximity is 1; elastic points lie inside it (Sections 2.2, 2.3 and the hardening extensions)."""
    import math as m_
    from oracle import constitutive as OC
    from synthetic import Material
    mats = {0: Material(0, E=206900.0, nu=0.29),
            1: Material(1, E=206900.0, nu=0.29, Y=450.0 * m_.sqrt(2 / 3), H=1e4),
            2: Material(2, E=206900.0, nu=0.29, Y=450.0 * m_.sqrt(2 / 3), H=1e4),
            3: Material(3, E=206900.0, nu=0.29, c0=450.0, phi=m_.radians(30.0), psi=m_.radians(10.0), Hc=1e3)}
    mat = mats[model]
    n = 4000
    rng = np.random.default_rng(40 + model + 10 * dim)
    ns = 3 if dim == 2 else 6
    nc = 4 if dim == 2 else 6
    E = rng.standard_normal((ns, n)) * 4e-3
    ep = rng.standard_normal((nc, n)) * 5e-4
    if model == 1:
        beta6 = OC.DEV @ OC.embed_state(rng.standard_normal((nc, n)) * 40.0, dim)
        hard = OC.extract_state(beta6, dim)
    else:
        hard = np.abs(rng.standard_normal(n)) * 1e-3
    res = OC.constitutive(mat, dim, E, ep, hard)
    q = W.yield_proximity(mat, dim, res["S"], res["hard"])
    pl = res["plastic"] != 0
    if model == 0:
        assert np.all(q == 0.0)
        return
    assert pl.any() and (~pl).any()
    assert np.abs(q[pl] - 1.0).max() < 1e-10
    assert np.all(q[~pl] <= 1.0 + 1e-12)
    # a stress scaled up by 10 % from an elastic point inside the von Mises cylinder moves outward
    if model == 2:
        q2 = W.yield_proximity(mat, dim, 1.1 * res["S"], res["hard"])
        assert np.all(q2[~pl] > q[~pl] - 1e-15)


def test_node_max_brute_force():
    prob = p1_plane_vm(n=3, n_steps=2)
    elem = prob.mesh.elem
    vals = np.random.default_rng(41).uniform(0, 2, elem.shape[0])
    out = W.node_max(elem, vals, 1, prob.mesh.n_nodes)
    for node in range(prob.mesh.n_nodes):
        assert out[node] == max(vals[e] for e in range(elem.shape[0]) if node in list(elem[e]))


def test_projection_keeps_fields_in_the_span_and_removes_an_orthogonal_part():
    rng = np.random.default_rng(42)
    n, dim = 50, 3
    X = rng.standard_normal((n, 16))
    free = np.ones(n * dim, dtype=bool)
    free[:6] = False
    fr = free.reshape(n, dim)
    a, b = rng.standard_normal(dim), rng.standard_normal(dim)
    y_in = np.stack([a[c] * X[:, c] + b[c] * X[:, 3 + c] for c in range(dim)], 1)
    P = W.project_correction(X, y_in, free, dim)
    assert np.allclose(P[fr], y_in[fr], rtol=0, atol=1e-12) and np.all(P[~fr] == 0.0)
    y = rng.standard_normal((n, 4))
    P = W.project_correction(X, y, free, dim)
    for c in range(dim):
        r = (y[:, c] - P[:, c]) * fr[:, c]
        assert abs(r @ (X[:, c] * fr[:, c])) < 1e-10 and abs(r @ (X[:, 3 + c] * fr[:, c])) < 1e-10
    # a vanishing older increment: the fit falls back to the last increment alone
    X0 = X.copy()
    X0[:, 3:6] = 0.0
    P0 = W.project_correction(X0, y, free, dim)
    for c in range(dim):
        x1 = X0[:, c] * fr[:, c]
        assert np.allclose(P0[:, c], (x1 @ (y[:, c] * fr[:, c])) / (x1 @ x1) * x1)
    assert np.all(W.project_correction(np.zeros((n, 16)), y, free, dim) == 0.0)
