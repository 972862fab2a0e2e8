"""Pins for the oracle's assembly, loads and Newton solver (Sections 4, 6, 7, 9).

Independent checks: quadrature weights sum to the domain measure; the elastic
patch test (affine fields reproduced exactly on perturbed meshes); rigid-body
modes in the kernel of K for any D; symmetry and semi-definiteness of
K_elast; the textbook constant-strain-triangle stiffness; per-element brute
force = split form = one-product form; consistent loads equal the closed-form
face distributions; the FEM solution of the plane-strain column equals the
one-material-point solve at every step; Newton converges locally
quadratically for von Mises.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import constitutive as C
from oracle.fem import Assembler, Geometry, element_matrices_bruteforce, scatter_elements, surface_load
from oracle.newton import OracleSolver, homogeneous_column
from synthetic import Material, structured_mesh, traction_load, VM_ISO, DP
from synthetic import p1_plane_vm, p2_plane_dp, generic_box, q1_cube_vm

ALL = [(e, d) for d in (2, 3) for e in ("P1", "P2", "Q1", "Q2")]
E_MOD, NU = 206900.0, 0.29
K_B, G_S = C.moduli(E_MOD, NU)


def _De(dim):
    D = C.elastic_tangent(K_B, G_S)
    return D[np.ix_(C.PLANE_INPLANE_IDX, C.PLANE_INPLANE_IDX)] if dim == 2 else D


def _mesh(elem, dim, n=None, perturb=0.0, seed=0):
    n = n if n is not None else (4 if dim == 2 else 2)
    m = structured_mesh(elem, dim, (n,) * dim, (10.0,) * dim)
    if perturb:
        g = np.random.default_rng(seed)
        h = 10.0 / n
        inner = np.all((m.coords > 1e-9) & (m.coords < 10 - 1e-9), axis=1)
        m.coords[inner] += g.uniform(-perturb * h, perturb * h, (inner.sum(), dim))
    return m


@pytest.mark.parametrize("elem,dim", ALL)
def test_weights_sum_to_measure(elem, dim):
    m = _mesh(elem, dim, perturb=0.1)
    g = Geometry(m.coords, m.elem, elem, dim)
    assert abs(g.WEIGHT.sum() - 10.0 ** dim) < 1e-10 * 10.0 ** dim
    assert (g.DET > 0).all()


@pytest.mark.parametrize("elem,dim", ALL)
def test_patch_test(elem, dim):
    m = _mesh(elem, dim, perturb=0.12, seed=1)
    g = Geometry(m.coords, m.elem, elem, dim)
    asm = Assembler(g, _De(dim))
    rng = np.random.default_rng(2)
    A = rng.standard_normal((dim, dim)) * 1e-3
    b = rng.standard_normal(dim) * 1e-2
    u_exact = (m.coords @ A.T + b).ravel()
    bnd = np.any((m.coords < 1e-9) | (m.coords > 10 - 1e-9), axis=1)
    fixed = np.repeat(bnd, dim)
    free = ~fixed
    K = asm.K_elast
    u = np.zeros_like(u_exact)
    u[fixed] = u_exact[fixed]
    rhs = -(K[free][:, fixed] @ u[fixed])
    u[free] = spla.spsolve(K[free][:, free].tocsc(), rhs)
    np.testing.assert_allclose(u, u_exact, atol=1e-12 * np.abs(u_exact).max() * 10)
    E = g.strain(asm.B, u)
    eps = 0.5 * (A + A.T)
    if dim == 2:
        want = np.array([eps[0, 0], eps[1, 1], 2 * eps[0, 1]])
    else:
        want = np.array([eps[0, 0], eps[1, 1], eps[2, 2], 2 * eps[0, 1], 2 * eps[1, 2], 2 * eps[0, 2]])
    np.testing.assert_allclose(E, want[:, None] * np.ones((1, g.n_int)), atol=1e-12)


def _rigid_modes(coords, dim):
    n = coords.shape[0]
    modes = []
    for a in range(dim):
        r = np.zeros((n, dim))
        r[:, a] = 1.0
        modes.append(r.ravel())
    x = coords
    if dim == 2:
        modes.append(np.stack([-x[:, 1], x[:, 0]], axis=1).ravel())
    else:
        for (i, j) in [(0, 1), (1, 2), (0, 2)]:
            r = np.zeros((n, 3))
            r[:, i], r[:, j] = -x[:, j], x[:, i]
            modes.append(r.ravel())
    return modes


@pytest.mark.parametrize("elem,dim", ALL)
def test_rigid_modes_and_symmetry(elem, dim):
    m = _mesh(elem, dim, perturb=0.1, seed=3)
    g = Geometry(m.coords, m.elem, elem, dim)
    asm = Assembler(g, _De(dim))
    B = asm.B
    ns = g.n_strain
    DS = np.random.default_rng(4).standard_normal((ns, ns, g.n_int)) * 1e5     # arbitrary, nonsymmetric
    Kt = asm.tangent_full(DS)
    for r in _rigid_modes(m.coords, dim):
        assert np.abs(B @ r).max() < 1e-12 * np.abs(r).max()
        assert np.abs(Kt @ r).max() < 1e-9 * abs(Kt).max() * np.abs(r).max()
    Ke = asm.K_elast
    assert abs(Ke - Ke.T).max() < 1e-10 * abs(Ke).max()
    x = np.random.default_rng(5).standard_normal((Ke.shape[0], 8))
    assert (np.einsum("ik,ik->k", x, Ke @ x) > 0).all()


def test_cst_triangle_closed_form():
    """P1 triangle: K_e = A B^T D B with the textbook constant-strain B."""
    x = np.array([[0.3, 0.1], [2.1, 0.4], [0.7, 1.9]])
    g = Geometry(x, np.array([[0, 1, 2]]), "P1", 2)
    D = _De(2)
    Ke = element_matrices_bruteforce(g, D[:, :, None] * np.ones((1, 1, 1)))[0]
    (x1, y1), (x2, y2), (x3, y3) = x
    A2 = (x2 - x1) * (y3 - y1) - (x3 - x1) * (y2 - y1)
    Bm = np.array([[y2 - y3, 0, y3 - y1, 0, y1 - y2, 0],
                   [0, x3 - x2, 0, x1 - x3, 0, x2 - x1],
                   [x3 - x2, y2 - y3, x1 - x3, y3 - y1, x2 - x1, y1 - y2]]) / A2
    want = (A2 / 2) * Bm.T @ D @ Bm
    np.testing.assert_allclose(Ke, want, rtol=1e-13, atol=1e-8)


@pytest.mark.parametrize("elem,dim", ALL)
def test_split_equals_full_equals_bruteforce(elem, dim):
    m = _mesh(elem, dim, n=(3 if dim == 2 else 2), perturb=0.1, seed=6)
    g = Geometry(m.coords, m.elem, elem, dim)
    asm = Assembler(g, _De(dim))
    ns = g.n_strain
    rng = np.random.default_rng(7)
    DS = np.repeat(_De(dim)[:, :, None], g.n_int, axis=2)
    plastic = rng.random(g.n_int) < 0.4
    DS[:, :, plastic] += rng.standard_normal((ns, ns, plastic.sum())) * 3e4
    K1 = asm.tangent_split(DS)
    K2 = asm.tangent_full(DS)
    K3 = scatter_elements(g, element_matrices_bruteforce(g, DS))
    nrm = np.sqrt((K3.multiply(K3)).sum())
    for Kx in (K1, K2):
        d = (Kx - K3)
        assert math.sqrt(d.multiply(d).sum()) <= 1e-13 * nrm


def test_internal_force_elastic_identity():
    """Elastic regime: F(u) = K_elast u - B^T W C eps^p."""
    m = _mesh("Q2", 2, n=3, perturb=0.1, seed=8)
    mat = Material(VM_ISO, E=E_MOD, nu=NU, Y=1e12, H=0.0)
    g = Geometry(m.coords, m.elem, "Q2", 2)
    asm = Assembler(g, _De(2))
    rng = np.random.default_rng(9)
    u = rng.standard_normal(m.n_nodes * 2) * 1e-3
    ep = rng.standard_normal((4, g.n_int)) * 1e-4
    res = C.constitutive(mat, 2, g.strain(asm.B, u), ep, np.zeros(g.n_int))
    F = asm.internal_force(res["S_in"])
    sig_p = (C.elastic_tangent(K_B, G_S) @ C.embed_state(ep, 2))[C.PLANE_INPLANE_IDX]
    want = asm.K_elast @ u - asm.BT @ (sig_p * g.WEIGHT).T.ravel()
    np.testing.assert_allclose(F, want, atol=1e-9 * np.abs(want).max())


@pytest.mark.parametrize("elem,dim", ALL)
def test_consistent_loads_match_closed_form(elem, dim):
    m = _mesh(elem, dim, n=3)
    t = np.array([0.3, -1.7] if dim == 2 else [0.2, 0.5, -1.3])
    f_closed = traction_load(m, t)
    f_quad = surface_load(m.coords, m.elem, elem, dim, lambda X: np.abs(X[:, dim - 1] - 10.0) < 1e-9, t)
    np.testing.assert_allclose(f_quad, f_closed, atol=1e-12)
    # total force = traction * area of the top face
    np.testing.assert_allclose(f_closed.reshape(-1, dim).sum(0), t * 10.0 ** (dim - 1), rtol=1e-13)


def _column_check(problem, t_max):
    s = OracleSolver(problem)
    hom = homogeneous_column(problem.material, problem.zeta * t_max)
    for k, z in enumerate(problem.zeta):
        rep = s.solve_step(float(z))
        assert rep.converged
        h = hom[k]
        smax = max(1.0, np.abs(h["stress"]).max())
        assert np.abs(s.stress - h["stress"][:, None]).max() <= 1e-10 * smax
        assert np.abs(s.ep - h["ep"][:, None]).max() <= 1e-12
        assert (s.plastic == h["plastic"]).all()
    return s


def test_column_p1_von_mises_matches_point_solve():
    p = p1_plane_vm(n=6)
    s = _column_check(p, 1.5 * p.extra["t_first_yield"])
    assert s.plastic.all()


def test_column_p2_drucker_prager_matches_point_solve():
    p = p2_plane_dp(n=3, n_steps=12, load_fraction=0.98)
    s = _column_check(p, 0.98 * p.extra["t_lim"])
    assert s.plastic.all()


def test_newton_quadratic_convergence_von_mises():
    mat = Material(VM_ISO, E=E_MOD, nu=NU, Y=450.0 * math.sqrt(2 / 3), H=1e4)
    p = q1_cube_vm(n=3, n_steps=4)
    p.material = mat
    s = OracleSolver(p)
    reps = s.solve_path(tol=1e-14, mode="previous")
    hist = max(reps, key=lambda r: r.newton_its).resid_history
    assert len(hist) >= 4
    # once in the local regime the error exponent roughly doubles per iteration
    good = [h for h in hist if h > 1e-13]
    ratios = [math.log(good[i + 1]) / math.log(good[i]) for i in range(len(good) - 1) if good[i] < 1e-2]
    assert ratios and max(ratios) > 1.6, hist


def test_batch_problem_generator_is_seeded_and_uneven():
    """The batched sweep's inputs: deterministic in the seed, sizes and materials within range."""
    from synthetic import batch_problems, vm_iso_material
    a = batch_problems(seed=1805, n_problems=8, sizes=(2, 5), n_steps=3)
    b = batch_problems(seed=1805, n_problems=8, sizes=(2, 5), n_steps=3)
    assert sorted(a) == ["P1", "P2", "Q1"] and sum(len(v) for v in a.values()) == 8
    base = vm_iso_material()
    for fam in a:
        for pa, pb in zip(a[fam], b[fam]):
            assert pa.mesh.n_elem == pb.mesh.n_elem and pa.material == pb.material
            assert 0.7 * base.E <= pa.material.E <= 1.3 * base.E
            assert 0.7 * base.Y <= pa.material.Y <= 1.3 * base.Y


def test_l_shape_and_strip_footing_inputs():
    """The validation workloads' meshes and loads: L-shape area 75 and total traction; footing nodes."""
    from synthetic import l_shape_vm, strip_footing_dp
    p = l_shape_vm("Q2", m=3, n_steps=40)
    g = Geometry(p.mesh.coords, p.mesh.elem, "Q2", 2)
    assert abs(g.WEIGHT.sum() - 75.0) < 1e-10
    np.testing.assert_allclose(p.f_unit.reshape(-1, 2).sum(0), [0.0, 2000.0], rtol=1e-13)
    assert p.zeta.max() == 1.0 and p.zeta.min() == -1.0 and abs(p.zeta[-1]) < 1e-12
    q = strip_footing_dp("P2", n=10)
    xs = q.mesh.coords[q.extra["footing_nodes"]]
    assert np.all(xs[:, 0] <= 1.0 + 1e-9) and np.all(np.abs(xs[:, 1] - 10.0) < 1e-9)
    assert len(xs) == 3          # x = 0, 0.5, 1 on a 10x10 P2 mesh


def test_prandtl_factor_closed_form():
    """N_c -> 2 + pi as phi -> 0 (Prandtl's cohesive limit) and N_c(30 deg) = 30.14 (textbook)."""
    from synthetic import prandtl_nc
    assert abs(prandtl_nc(1e-6) - (2.0 + math.pi)) < 1e-4
    assert abs(prandtl_nc(math.radians(30.0)) - 30.14) < 0.01


def test_oracle_l_shape_cycle_dissipates():
    """The oracle on the cyclic L-shape: plastic flow on loading, a residual state after the cycle."""
    from synthetic import l_shape_vm
    p = l_shape_vm("Q1", m=2, n_steps=8)
    s = OracleSolver(p)
    work = []
    for z in p.zeta:
        s.solve_step(float(z), tol=1e-12)
        work.append(float(p.f_unit @ s.u))
    assert np.abs(s.ep).max() > 0
    assert abs(work[-1]) > 1e-3 * max(abs(w) for w in work)


def test_oracle_newton_start_across_load_reversals():
    """Reading R24 of ALG-NEWTON's start: the extrapolation is used only while the load keeps its
    direction.  With the negative ratio at the second reversal of the 16-step cyclic L-shape (zeta
    -1 -> -0.75) the extrapolation predicts the loading branch, not the elastic unloading, and Newton
    did not converge in 50 iterations; with the reading every step converges."""
    from synthetic import l_shape_vm
    p = l_shape_vm("Q2", m=3, n_steps=16)
    s = OracleSolver(p)
    reps = s.solve_path(tol=1e-13)
    assert all(r.converged for r in reps)
    rev = [k for k in range(2, len(p.zeta)) if (p.zeta[k] - p.zeta[k - 1]) * (p.zeta[k - 1] - p.zeta[k - 2]) < 0]
    assert len(rev) == 2
    # after the first reversal two elastic unloading steps make the extrapolation exact: 0 iterations
    assert p.zeta[5] == 0.5 and reps[5].newton_its == 0
