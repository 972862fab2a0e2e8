"""Pins for the oracle's reference elements and quadrature (Appendix).

Checks against facts fixed by mathematics: partition of unity, Kronecker
property at the reference nodes, derivatives against central differences of
the basis, exactness of each rule on monomials (closed-form integrals), and
the 11-point rule's digits as printed in the paper.
"""
import math
import os

import numpy as np
import pytest

from oracle import elements

ALL = [(e, d) for d in (2, 3) for e in ("P1", "P2", "Q1", "Q2")]
N_P = {("P1", 2): 3, ("P2", 2): 6, ("Q1", 2): 4, ("Q2", 2): 8,
       ("P1", 3): 4, ("P2", 3): 10, ("Q1", 3): 8, ("Q2", 3): 20}
N_Q = {("P1", 2): 1, ("P2", 2): 7, ("Q1", 2): 4, ("Q2", 2): 9,
       ("P1", 3): 1, ("P2", 3): 11, ("Q1", 3): 8, ("Q2", 3): 27}


def _random_points(elem, dim, n, seed):
    g = np.random.default_rng(seed)
    if elem.startswith("P"):
        x = g.dirichlet(np.ones(dim + 1), size=n)[:, 1:].T
    else:
        x = g.uniform(-1, 1, size=(dim, n))
    return x


@pytest.mark.parametrize("elem,dim", ALL)
def test_partition_of_unity_and_kronecker(elem, dim):
    N = elements.nodes(elem, dim)
    assert N.shape == (N_P[(elem, dim)], dim)
    P, D = elements.basis(elem, dim, N.T)
    np.testing.assert_allclose(P, np.eye(N.shape[0]), atol=1e-14)
    x = _random_points(elem, dim, 50, 1)
    P, D = elements.basis(elem, dim, x)
    np.testing.assert_allclose(P.sum(axis=0), 1.0, atol=1e-13)
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-13)


@pytest.mark.parametrize("elem,dim", ALL)
def test_gradients_match_central_differences(elem, dim):
    x = _random_points(elem, dim, 20, 2) * 0.9
    P, D = elements.basis(elem, dim, x)
    h = 1e-6
    for i in range(dim):
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd = (elements.basis(elem, dim, xp)[0] - elements.basis(elem, dim, xm)[0]) / (2 * h)
        np.testing.assert_allclose(D[i], fd, atol=1e-8)


@pytest.mark.parametrize("elem,dim", ALL)
def test_linear_completeness(elem, dim):
    """sum_p x_p Phi_p(xi) = xi for the reference nodes (isoparametric identity)."""
    N = elements.nodes(elem, dim)
    x = _random_points(elem, dim, 30, 3)
    P, D = elements.basis(elem, dim, x)
    np.testing.assert_allclose(N.T @ P, x, atol=1e-13)
    for i in range(dim):
        np.testing.assert_allclose(N.T @ D[i], np.eye(dim)[:, [i]] * np.ones((1, x.shape[1])), atol=1e-13)


def _exact_simplex(exps):
    # int over the unit simplex of prod xi^a = prod a! / (sum a + dim)!
    num = np.prod([math.factorial(a) for a in exps])
    return num / math.factorial(sum(exps) + len(exps))


def _exact_cube(exps):
    return np.prod([0.0 if a % 2 else 2.0 / (a + 1) for a in exps])


DEGREE = {("P1", 2): 1, ("P2", 2): 5, ("P1", 3): 1, ("P2", 3): 4}


@pytest.mark.parametrize("elem,dim", ALL)
def test_quadrature_exactness(elem, dim):
    Xi, w = elements.quadrature(elem, dim)
    assert w.size == N_Q[(elem, dim)]
    if elem.startswith("P"):
        deg = DEGREE[(elem, dim)]
        for exps in np.ndindex(*([deg + 1] * dim)):
            if sum(exps) > deg:
                continue
            val = np.sum(w * np.prod([Xi[i] ** exps[i] for i in range(dim)], axis=0))
            assert abs(val - _exact_simplex(exps)) < 1e-15, exps
        # the rule is not exact one degree higher (it is a degree-`deg` rule)
        exps = (deg + 1,) + (0,) * (dim - 1)
        val = np.sum(w * Xi[0] ** (deg + 1))
        if deg > 1:
            assert abs(val - _exact_simplex(exps)) > 1e-8
    else:
        per = 3 if elem == "Q1" else 5
        for exps in np.ndindex(*([per + 2] * dim)):
            val = np.sum(w * np.prod([Xi[i] ** exps[i] for i in range(dim)], axis=0))
            exact = _exact_cube(exps)
            if max(exps) <= per:
                assert abs(val - exact) < 1e-14, exps
        assert abs(np.sum(w * Xi[0] ** (per + 1)) - _exact_cube((per + 1,) + (0,) * (dim - 1))) > 1e-6


def test_keast_rule_matches_printed_digits():
    path = os.path.join(os.path.dirname(__file__), "golden", "keast_11pt_printed.txt")
    printed = np.loadtxt(path)
    Xi, w = elements.quadrature("P2", 3)
    np.testing.assert_allclose(Xi.T, printed[:, :3], atol=1e-14)
    np.testing.assert_allclose(w, printed[:, 3], atol=1e-14)
    assert abs(w.sum() - 1.0 / 6.0) < 1e-16


@pytest.mark.parametrize("kind", ["L1", "L2", "T1", "T2", "S1", "S2"])
def test_face_rules_partition_of_unity(kind):
    fb, pts, w = elements.face_rule(kind)
    P, dP = fb(pts)
    np.testing.assert_allclose(P.sum(axis=0), 1.0, atol=1e-14)
    np.testing.assert_allclose(dP.sum(axis=1), 0.0, atol=1e-13)
