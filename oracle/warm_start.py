"""Learned warm start of the Newton iteration: features, targets and the per-node MLP (plain numpy, FP64).

Test infrastructure: part of the CPU oracle; never used by the product path.

The paper starts Newton at step k from the prescribed values u_{D,k} (ALG-NEWTON,
Section 4); the build's default start is the linear extrapolation
    u_ex = u_{k-1} + r_k (u_{k-1} - u_{k-2}),  r_k = (zeta_k - zeta_{k-1}) / (zeta_{k-1} - zeta_{k-2}),
with the Dirichlet values of step k.  The learned start adds a per-node
correction predicted by a small MLP from the node's recent history:
    u_L = u_ex + s * P(y[:dim])  on free DOFs,
where s is the problem's RMS increment of the last step and P projects the
per-node prediction, per problem and displacement component, onto the span of
the last two increments (least squares over the free DOFs).  The projection
keeps the correction as smooth as the increments: per-node predictions carry
independent errors of a few percent, whose roughness the stiffness turns into
residuals larger than those of the plain extrapolation.  The definitions here
are the ones the CUDA path must reproduce:

  node_plastic_fraction  fraction of the integration points of the elements
                         adjacent to a node that are plastic (flag != 0)
  yield_proximity        yield-function ratio of a committed stress (1 on the
                         yield surface), and node_max its maximum over the
                         points of the adjacent elements
  static_features        material and boundary scalars of a node
  features               the 16 inputs of a node for step k
  targets                the 4 outputs the MLP is trained on after step k converged
  project_correction     the projection P above
  mlp_forward / mlp_loss / mlp_grad   3 linear layers 16 -> 128 -> 128 -> 4, ReLU,
                         weights rounded to bfloat16, biases and activations
                         kept exact (FP64 here, FP32 on the device)
  adam_step              Adam (Kingma & Ba, 2015) with bias correction

Parameter layout (flat float32 vector, EP_WS_N_PARAMS = 19204 entries):
  W1 [128][16], b1 [128], W2 [128][128], b2 [128], W3 [4][128], b3 [4],
each weight matrix [out][in] (y_j = sum_i W[j][i] x_i + b_j).

Loss (per batch of n rows): (1/n) sum_rows [ sum_{c<3} (y_c - t_c)^2 + LAMBDA_PL * bce(y_3, t_3) ],
bce(z, t) = max(z, 0) - z t + log(1 + exp(-|z|)) (the logistic loss of the
plastic-fraction logit z against the fraction t).

Pins (tests/test_oracle_warm_start.py): bfloat16 rounding on exact halfway cases
and against torch's conversion; forward pass against explicit loops; gradient
against central finite differences; Adam against the constant-gradient closed
form; plastic fractions against a brute-force scan; features and targets
against the homogeneous elastic column, whose equally spaced steps make the
extrapolation exact; the proximity against the return mappings (exactly 1 at
plastic points, below 1 at elastic ones); the projection against fields that
lie in the span and the orthogonality of what it removes.
"""
from __future__ import annotations

import math

import numpy as np

from . import constitutive as C

N_IN, WIDTH, N_OUT = 16, 128, 4
OFF_W1 = 0
OFF_B1 = OFF_W1 + WIDTH * N_IN
OFF_W2 = OFF_B1 + WIDTH
OFF_B2 = OFF_W2 + WIDTH * WIDTH
OFF_W3 = OFF_B2 + WIDTH
OFF_B3 = OFF_W3 + N_OUT * WIDTH
N_PARAMS = OFF_B3 + N_OUT
LAMBDA_PL = 0.1
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


# -- bfloat16 -----------------------------------------------------------------------------------
def bf16_round(x) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even) -> float32: keep the upper 16 bits after adding
    0x7FFF plus the lowest kept bit (finite inputs)."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return (b << 16).astype(np.uint32).view(np.float32)


# -- parameters ---------------------------------------------------------------------------------
def unpack(params, round_weights: bool = True):
    """(W1, b1, W2, b2, W3, b3) in FP64; the weights rounded to bfloat16 when round_weights."""
    p = np.asarray(params, dtype=np.float32)
    assert p.shape == (N_PARAMS,)
    rw = bf16_round if round_weights else (lambda a: a)
    W1 = rw(p[OFF_W1:OFF_B1]).astype(np.float64).reshape(WIDTH, N_IN)
    b1 = p[OFF_B1:OFF_W2].astype(np.float64)
    W2 = rw(p[OFF_W2:OFF_B2]).astype(np.float64).reshape(WIDTH, WIDTH)
    b2 = p[OFF_B2:OFF_W3].astype(np.float64)
    W3 = rw(p[OFF_W3:OFF_B3]).astype(np.float64).reshape(N_OUT, WIDTH)
    b3 = p[OFF_B3:].astype(np.float64)
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, np.ravel(W3), b3]).astype(np.float64)


# -- network --------------------------------------------------------------------------------------
def mlp_forward(params, X, round_weights: bool = True, params_f64=None):
    """Y [n][4] and the hidden activations (h1, h2); X [n][16].  params_f64 (FP64, unrounded)
    replaces params when given (finite-difference checks)."""
    if params_f64 is not None:
        p = np.asarray(params_f64, dtype=np.float64)
        W1 = p[OFF_W1:OFF_B1].reshape(WIDTH, N_IN)
        b1 = p[OFF_B1:OFF_W2]
        W2 = p[OFF_W2:OFF_B2].reshape(WIDTH, WIDTH)
        b2 = p[OFF_B2:OFF_W3]
        W3 = p[OFF_W3:OFF_B3].reshape(N_OUT, WIDTH)
        b3 = p[OFF_B3:]
    else:
        W1, b1, W2, b2, W3, b3 = unpack(params, round_weights)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    y = h2 @ W3.T + b3
    return y, (h1, h2, (W1, W2, W3))


def _bce(z, t):
    return np.maximum(z, 0.0) - z * t + np.log1p(np.exp(-np.abs(z)))


def mlp_loss(params, X, T, round_weights: bool = True, params_f64=None) -> float:
    y, _ = mlp_forward(params, X, round_weights, params_f64)
    T = np.asarray(T, dtype=np.float64)
    n = X.shape[0]
    return float(((y[:, :3] - T[:, :3]) ** 2).sum() / n + LAMBDA_PL * _bce(y[:, 3], T[:, 3]).sum() / n)


def mlp_grad(params, X, T, round_weights: bool = True, params_f64=None):
    """(loss, gradient [N_PARAMS]) by backpropagation through the three layers; the gradient with
    respect to a rounded weight is taken as the gradient with respect to its FP32 master copy."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    n = X.shape[0]
    y, (h1, h2, (W1, W2, W3)) = mlp_forward(params, X, round_weights, params_f64)
    loss = float(((y[:, :3] - T[:, :3]) ** 2).sum() / n + LAMBDA_PL * _bce(y[:, 3], T[:, 3]).sum() / n)
    dy = np.empty_like(y)
    dy[:, :3] = 2.0 * (y[:, :3] - T[:, :3]) / n
    dy[:, 3] = LAMBDA_PL * (1.0 / (1.0 + np.exp(-y[:, 3])) - T[:, 3]) / n
    dW3 = dy.T @ h2
    db3 = dy.sum(axis=0)
    dh2 = (dy @ W3) * (h2 > 0)
    dW2 = dh2.T @ h1
    db2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (h1 > 0)
    dW1 = dh1.T @ X
    db1 = dh1.sum(axis=0)
    return loss, pack(dW1, db1, dW2, db2, dW3, db3)


def adam_step(p, m, v, g, t: int, lr: float):
    """One Adam update (step t >= 1); returns (p, m, v), all FP64."""
    m = ADAM_B1 * m + (1.0 - ADAM_B1) * g
    v = ADAM_B2 * v + (1.0 - ADAM_B2) * g * g
    mh = m / (1.0 - ADAM_B1 ** t)
    vh = v / (1.0 - ADAM_B2 ** t)
    return p - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


# -- features and targets ----------------------------------------------------------------------
def node_plastic_fraction(elem, plastic, n_q: int, n_nodes: int) -> np.ndarray:
    """Per node: plastic points / all points of the elements containing it (integration point
    e*n_q + q belongs to element e)."""
    elem = np.asarray(elem)
    pl = (np.asarray(plastic).reshape(-1, n_q) != 0).sum(axis=1)
    cnt_pl = np.zeros(n_nodes)
    cnt_ip = np.zeros(n_nodes)
    for p in range(elem.shape[1]):
        np.add.at(cnt_pl, elem[:, p], pl)
        np.add.at(cnt_ip, elem[:, p], n_q)
    return np.where(cnt_ip > 0, cnt_pl / np.maximum(cnt_ip, 1), 0.0)


def yield_proximity(material, dim: int, stress, hard) -> np.ndarray:
    """Per integration point, the ratio of the yield function's stress part to its current limit
    for a committed stress (stored layout: (11, 22, 12, 33) in 2D, Voigt in 3D), clamped at 0:
      von Mises, isotropic:  |dev s| / (Y + H alpha)           (Section 2.2, with the extension)
      von Mises, kinematic:  |dev s - beta| / Y
      Drucker-Prager:        (|dev s| / sqrt(2) + eta p) / (c + Hc alpha),  p = tr(s)/3  (Section 2.3)
      elastic:               0
    with |x|^2 = x11^2 + x22^2 + x33^2 + 2 (x12^2 + x23^2 + x13^2) (tensor norm of a stress-type vector)."""
    m = material
    model = int(m.model)
    S = C.embed_state(np.asarray(stress, dtype=np.float64), dim)
    n = S.shape[1]
    if model == 0:
        return np.zeros(n)
    mean = (S[0] + S[1] + S[2]) / 3.0
    dev = S.copy()
    dev[0:3] -= mean
    if model == 1:
        dev = dev - C.embed_state(np.asarray(hard, dtype=np.float64), dim)
    nrm = np.sqrt(dev[0] ** 2 + dev[1] ** 2 + dev[2] ** 2 + 2.0 * (dev[3] ** 2 + dev[4] ** 2 + dev[5] ** 2))
    if model == 1:
        q = nrm / m.Y
    elif model == 2:
        q = nrm / (m.Y + m.H * np.asarray(hard, dtype=np.float64))
    else:
        eta, c, _ = C.dp_parameters(m.c0, m.phi, m.psi, dim)
        q = (nrm / math.sqrt(2.0) + eta * mean) / (c + m.Hc * np.asarray(hard, dtype=np.float64))
    return np.maximum(q, 0.0)


def node_max(elem, values, n_q: int, n_nodes: int) -> np.ndarray:
    """Per node: the largest value over the integration points of the elements containing it."""
    elem = np.asarray(elem)
    ve = np.asarray(values).reshape(-1, n_q).max(axis=1)
    out = np.zeros(n_nodes)
    for p in range(elem.shape[1]):
        np.maximum.at(out, elem[:, p], ve)
    return out


def static_features(material, dirichlet, dim: int) -> np.ndarray:
    """[n_nodes][5]: nu, yield strain x 1e3 (Y/E for von Mises, c0/E for Drucker-Prager), hardening
    ratio x 10 (H/E or Hc/E), 1 for Drucker-Prager, fraction of prescribed components."""
    mask = np.asarray(dirichlet).reshape(-1, dim)
    n = mask.shape[0]
    m = material
    is_dp = int(m.model) == 3
    ys = (m.c0 if is_dp else m.Y) / m.E * 1e3 if int(m.model) != 0 else 0.0
    hr = ((m.Hc if is_dp else m.H) / m.E * 10.0) if int(m.model) != 0 else 0.0
    out = np.zeros((n, 5))
    out[:, 0] = m.nu
    out[:, 1] = ys
    out[:, 2] = hr
    out[:, 3] = 1.0 if is_dp else 0.0
    out[:, 4] = (mask != 0).sum(axis=1) / dim
    return out


def increment_scale(u1, u2) -> float:
    """s = RMS of the last increment over all DOFs of a problem."""
    d = np.asarray(u1) - np.asarray(u2)
    return float(np.sqrt((d * d).mean())) if d.size else 0.0


def features(u1, u2, u3, zetas, pf1, pf2, prox1, stat, dim: int):
    """Inputs for step k [n_nodes][16] and the scale s.

    u1, u2, u3 = u_{k-1}, u_{k-2}, u_{k-3}; zetas = (zeta_k, zeta_{k-1}, zeta_{k-2}, zeta_{k-3});
    pf1, pf2 = plastic fractions after steps k-1 and k-2; prox1 = node_max of the yield proximity
    after step k-1.  Columns: the last two increments / s (3 each, zero-padded in 2D), r_k, r_{k-1},
    pf1, pf1 - pf2, prox1, the five static features."""
    z0, z1, z2, z3 = zetas
    s = increment_scale(u1, u2)
    inv_s = 1.0 / s if s > 0 else 0.0
    n = stat.shape[0]
    X = np.zeros((n, N_IN))
    d1 = (np.asarray(u1) - np.asarray(u2)).reshape(n, dim) * inv_s
    d2 = (np.asarray(u2) - np.asarray(u3)).reshape(n, dim) * inv_s
    X[:, 0:dim] = d1
    X[:, 3:3 + dim] = d2
    X[:, 6] = (z0 - z1) / (z1 - z2)
    X[:, 7] = (z1 - z2) / (z2 - z3) if z2 != z3 else 0.0
    X[:, 8] = pf1
    X[:, 9] = np.asarray(pf1) - np.asarray(pf2)
    X[:, 10] = prox1
    X[:, 11:16] = stat
    return X, s


def extrapolated_start(u1, u2, zetas, free, uD_unit):
    """u_ex: the linear extrapolation with the Dirichlet values of step k."""
    z0, z1, z2 = zetas[:3]
    u = np.asarray(u1) + (z0 - z1) / (z1 - z2) * (np.asarray(u1) - np.asarray(u2))
    u = u.copy()
    u[~free] = z0 * np.asarray(uD_unit)[~free]
    return u


def targets(u_k, u_ex, s: float, pf_k, free, dim: int):
    """Training targets [n_nodes][4]: (u_k - u_ex)/s on free DOFs (0 on prescribed ones, padded to 3
    components) and the plastic fraction after step k."""
    inv_s = 1.0 / s if s > 0 else 0.0
    d = (np.asarray(u_k) - np.asarray(u_ex)) * inv_s * np.asarray(free)
    n = d.size // dim
    T = np.zeros((n, N_OUT))
    T[:, :dim] = d.reshape(n, dim)
    T[:, 3] = pf_k
    return T


def project_correction(X, y, free, dim: int):
    """P(y): per displacement component c, the least-squares fit of y[:, c] over the free DOFs by
    a x1 + b x2 with x1 = X[:, c], x2 = X[:, 3 + c] (the scaled last two increments), from the 2x2
    normal equations; when they are singular (det <= 1e-12 S11 S22) the fit uses x1 alone, and
    nothing when x1 vanishes on the free DOFs.  Prescribed DOFs get 0.  Returns [n][dim]."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    fr = np.asarray(free).reshape(-1, dim).astype(np.float64)
    out = np.zeros((X.shape[0], dim))
    for c in range(dim):
        x1 = X[:, c] * fr[:, c]
        x2 = X[:, 3 + c] * fr[:, c]
        yc = y[:, c] * fr[:, c]
        s11, s12, s22 = x1 @ x1, x1 @ x2, x2 @ x2
        b1, b2 = x1 @ yc, x2 @ yc
        det = s11 * s22 - s12 * s12
        if det > 1e-12 * s11 * s22 and det > 0:
            a, b = (s22 * b1 - s12 * b2) / det, (s11 * b2 - s12 * b1) / det
        elif s11 > 0:
            a, b = b1 / s11, 0.0
        else:
            a, b = 0.0, 0.0
        out[:, c] = a * x1 + b * x2
    return out


def learned_start(u_ex, y, s: float, free, dim: int):
    """u_L = u_ex + s y[:dim] on free DOFs."""
    u = np.asarray(u_ex, dtype=np.float64).copy()
    corr = (s * np.asarray(y, dtype=np.float64)[:, :dim]).ravel()
    u[free] += corr[free]
    return u


def trajectory_samples(problem, zetas, solver_factory, free=None):
    """Solve the load path with the oracle (extrapolated start) and return the (X, T) rows of every
    step k >= 4 (three earlier converged steps): the features before the step, the targets after."""
    sol = solver_factory(problem)
    dim = problem.mesh.dim
    n_nodes = problem.mesh.n_nodes
    n_q = sol.geom.n_q
    free = problem.dirichlet == 0 if free is None else free
    stat = static_features(problem.material, problem.dirichlet, dim)
    us = [sol.u.copy()]
    zs = [0.0]
    pfs = [np.zeros(n_nodes)]
    prox = [np.zeros(n_nodes)]
    Xs, Ts = [], []
    for z in zetas:
        z = float(z)
        if len(us) >= 4 and zs[-1] != zs[-2] and (z - zs[-1]) / (zs[-1] - zs[-2]) > 0:
            X, s = features(us[-1], us[-2], us[-3], (z, zs[-1], zs[-2], zs[-3]), pfs[-1], pfs[-2], prox[-1],
                            stat, dim)
        else:
            X = None
        if not sol.solve_step(z, tol=1e-13).converged:
            raise RuntimeError(f"oracle Newton did not converge at zeta = {z}")
        pf = node_plastic_fraction(problem.mesh.elem, sol.plastic, n_q, n_nodes)
        if X is not None:
            u_ex = extrapolated_start(us[-1], us[-2], (z, zs[-1], zs[-2]), free, problem.u_D_unit)
            Xs.append(X)
            Ts.append(targets(sol.u, u_ex, s, pf, free, dim))
        us.append(sol.u.copy())
        zs.append(z)
        pfs.append(pf)
        prox.append(node_max(problem.mesh.elem, yield_proximity(problem.material, dim, sol.stress, sol.hard), n_q,
                             n_nodes))
    if not Xs:
        return np.zeros((0, N_IN)), np.zeros((0, N_OUT))
    return np.concatenate(Xs), np.concatenate(Ts)


def last_learned_start(problem, zetas, params, solver_factory):
    """The learned start of the last step of a load path, from the oracle's own trajectory (extrapolated
    starts; the converged steps do not depend on the start): (u_L, s, P(y)) with P(y) [n][dim], or None
    when that step has no inputs (fewer than three earlier steps, or a reversed load)."""
    sol = solver_factory(problem)
    dim = problem.mesh.dim
    n_nodes = problem.mesh.n_nodes
    n_q = sol.geom.n_q
    free = problem.dirichlet == 0
    stat = static_features(problem.material, problem.dirichlet, dim)
    us, zs, pfs, prox = [sol.u.copy()], [0.0], [np.zeros(n_nodes)], [np.zeros(n_nodes)]
    for z in zetas[:-1]:
        if not sol.solve_step(float(z), tol=1e-13).converged:
            raise RuntimeError(f"oracle Newton did not converge at zeta = {z}")
        us.append(sol.u.copy())
        zs.append(float(z))
        pfs.append(node_plastic_fraction(problem.mesh.elem, sol.plastic, n_q, n_nodes))
        prox.append(node_max(problem.mesh.elem, yield_proximity(problem.material, dim, sol.stress, sol.hard), n_q,
                             n_nodes))
    z = float(zetas[-1])
    if len(us) < 4 or zs[-1] == zs[-2] or (z - zs[-1]) / (zs[-1] - zs[-2]) <= 0:
        return None
    X, s = features(us[-1], us[-2], us[-3], (z, zs[-1], zs[-2], zs[-3]), pfs[-1], pfs[-2], prox[-1], stat, dim)
    X = X.astype(np.float32)       # the network reads FP32 inputs
    y, _ = mlp_forward(params, X)
    P = project_correction(X, y, free, dim)
    u_ex = extrapolated_start(us[-1], us[-2], (z, zs[-1], zs[-2]), free, problem.u_D_unit)
    return learned_start(u_ex, P, s, free, dim), s, P
