"""The library's host-side builders on the CPU (no GPU): the block-CSR pattern and element-to-slot map
against a brute-force adjacency, and the reference-element tables against the oracle's elements.

The builders' sources are compiled here with a small C wrapper (tests/host_shim.cpp); nothing of
the device code is involved.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import elements as OE
from synthetic import structured_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1805_04155_gb300", "csrc")
FAMILY = {"P1": 0, "P2": 1, "Q1": 2, "Q2": 3}
ALL = [(e, d) for d in (2, 3) for e in ("P1", "P2", "Q1", "Q2")]


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("shim") / "libhostshim.so")
    cmd = [nvcc, "-std=c++17", "-O1", "-Xcompiler", "-fPIC,-fopenmp", "-shared", "-x", "c++",
           os.path.join(ROOT, "tests", "host_shim.cpp"), os.path.join(SRC, "pattern_host.cpp"),
           os.path.join(SRC, "elements_host.cpp"), os.path.join(SRC, "amg_host.cpp"), os.path.join(SRC, "direct_host.cpp"),
           "-I", os.path.join(ROOT, "include"),
           "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = C.CDLL(out)
    lib.shim_build_pattern.argtypes = [C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                       C.c_void_p, C.POINTER(C.c_int64)]
    lib.shim_reference_tables.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64]
    lib.shim_color_elements.argtypes = [C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.shim_amg_setup.argtypes = [C.c_int, C.c_int64] + [C.c_void_p] * 5
    lib.shim_amg_setup.restype = C.c_void_p
    lib.shim_amg_free.argtypes = [C.c_void_p]
    lib.shim_amg_levels.argtypes = [C.c_void_p]
    lib.shim_amg_level.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_double)]
    lib.shim_amg_mat_shape.argtypes = [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                       C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int64)]
    lib.shim_amg_mat_copy.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.shim_amg_inv_sizes.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.shim_amg_inv_copy.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    lib.shim_direct_analyse.argtypes = [C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    lib.shim_direct_analyse.restype = C.c_void_p
    lib.shim_direct_free.argtypes = [C.c_void_p]
    lib.shim_direct_sizes.argtypes = [C.c_void_p, C.c_void_p]
    lib.shim_direct_copy.argtypes = [C.c_void_p] + [C.c_void_p] * 12
    return lib


def _pattern(shim, n_nodes, elem):
    elem = np.ascontiguousarray(elem, dtype=np.int32)
    n_e, n_p = elem.shape
    cap = n_nodes * 200
    rp = np.zeros(n_nodes + 1, dtype=np.int32)
    ci = np.zeros(cap, dtype=np.int32)
    sl = np.zeros(n_e * n_p * n_p, dtype=np.int32)
    nnzb = C.c_int64(0)
    st = shim.shim_build_pattern(n_nodes, n_e, n_p, elem.ctypes.data, rp.ctypes.data, cap, ci.ctypes.data,
                                 sl.ctypes.data, C.byref(nnzb))
    return st, rp, ci[:nnzb.value], sl.reshape(n_e, n_p, n_p)


@pytest.mark.parametrize("elem_type,dim", ALL)
def test_pattern_is_the_node_adjacency_and_slots_point_at_their_pairs(shim, elem_type, dim):
    mesh = structured_mesh(elem_type, dim, (3,) * dim, (10.0,) * dim)
    st, rp, ci, sl = _pattern(shim, mesh.n_nodes, mesh.elem)
    assert st == 1
    adj = [set() for _ in range(mesh.n_nodes)]
    for e in mesh.elem:
        for a in e:
            adj[a].update(int(b) for b in e)
    assert rp[0] == 0 and np.all(np.diff(rp) > 0)
    for n in range(mesh.n_nodes):
        row = ci[rp[n]:rp[n + 1]]
        assert np.all(np.diff(row) > 0)                     # sorted, unique
        assert set(row.tolist()) == adj[n]                  # exactly the nodes sharing an element
    n_p = mesh.elem.shape[1]
    for e, nodes in enumerate(mesh.elem):
        for p in range(n_p):
            for q in range(n_p):
                k = sl[e, p, q]
                assert rp[nodes[p]] <= k < rp[nodes[p] + 1] and ci[k] == nodes[q]


@pytest.mark.parametrize("elem_type,dim", ALL)
def test_element_colouring_separates_elements_sharing_a_node(shim, elem_type, dim):
    """Deterministic assembly: within a colour no two elements share a node (so plain adds into F and
    K cannot collide), every element has exactly one colour, and each colour lists its elements in
    increasing order."""
    m = structured_mesh(elem_type, dim, (5, 4) if dim == 2 else (3, 3, 2), (10.0,) * dim)
    elem = np.ascontiguousarray(m.elem, dtype=np.int32)
    n_e, n_p = elem.shape
    cp = np.zeros(n_e + 1, dtype=np.int32)
    ce = np.zeros(n_e, dtype=np.int32)
    nc = shim.shim_color_elements(m.n_nodes, n_e, n_p, elem.ctypes.data, cp.ctypes.data, ce.ctypes.data)
    assert nc >= 2
    cp = cp[:nc + 1]
    assert cp[0] == 0 and cp[-1] == n_e
    assert np.array_equal(np.sort(ce), np.arange(n_e))
    for c in range(nc):
        els = ce[cp[c]:cp[c + 1]]
        assert np.all(np.diff(els) > 0)
        nodes = elem[els].ravel()
        assert len(np.unique(nodes)) == len(nodes), f"colour {c} has elements sharing a node"
    # greedy bound: at most (elements sharing a node with one element) + 1 colours
    adj = max(len(set(np.nonzero(np.isin(elem, elem[e]).any(axis=1))[0])) for e in range(n_e))
    assert nc <= adj


def test_pattern_rejects_a_node_index_out_of_range(shim):
    mesh = structured_mesh("P1", 2, (2, 2), (10.0, 10.0))
    bad = mesh.elem.copy()
    bad[1, 2] = mesh.n_nodes
    assert _pattern(shim, mesh.n_nodes, bad)[0] == 0
    bad[1, 2] = -1
    assert _pattern(shim, mesh.n_nodes, bad)[0] == 0


@pytest.mark.parametrize("elem_type,dim", ALL)
def test_reference_tables_match_the_oracle_elements(shim, elem_type, dim):
    pts, w = OE.quadrature(elem_type, dim)
    _, D = OE.basis(elem_type, dim, pts)             # D [dim][n_p][n_q]
    n_p, n_q = D.shape[1], D.shape[2]
    dhat = np.zeros(n_q * n_p * dim)
    wq = np.zeros(n_q)
    assert shim.shim_reference_tables(FAMILY[elem_type], dim, dhat.ctypes.data, dhat.size, wq.ctypes.data, n_q) == n_q
    want = np.transpose(D, (2, 1, 0)).ravel()        # [n_q][n_p][dim]
    assert np.abs(wq - w).max() <= 1e-15 * np.abs(w).max()
    assert np.abs(dhat - want).max() <= 1e-14 * max(1.0, np.abs(want).max())


def _amg_mat(shim, h, level, which):
    import scipy.sparse as sp
    nr, nc, rb, cb, nnzb = C.c_int64(), C.c_int64(), C.c_int(), C.c_int(), C.c_int64()
    shim.shim_amg_mat_shape(h, level, which, C.byref(nr), C.byref(nc), C.byref(rb), C.byref(cb), C.byref(nnzb))
    rp = np.zeros(nr.value + 1, dtype=np.int32)
    ci = np.zeros(nnzb.value, dtype=np.int32)
    v = np.zeros(nnzb.value * rb.value * cb.value)
    shim.shim_amg_mat_copy(h, level, which, rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
    return sp.bsr_matrix((v.reshape(-1, rb.value, cb.value), ci, rp),
                         shape=(nr.value * rb.value, nc.value * cb.value)).tocsr()


@pytest.mark.parametrize("make", ["p2_column", "q1_cube"])
def test_amg_setup_galerkin_hierarchy(shim, make):
    """Smoothed-aggregation setup on K_elast (from the oracle): every coarse operator is the Galerkin
    product R A P with R = P^T (coarse DOFs whose near-null column was dropped get an identity row),
    the stored block-diagonal inverses invert the diagonal blocks, the coarsest dense inverse inverts
    the coarsest operator, and the spectral bound lies near the largest eigenvalue of D^-1 A."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    from oracle import constitutive as OC
    from oracle.fem import Assembler, Geometry
    from synthetic import p2_plane_dp, q1_cube_vm
    prob = p2_plane_dp(n=32, n_steps=2) if make == "p2_column" else q1_cube_vm(n=12, n_steps=2)
    m = prob.mesh
    d = m.dim
    g = Geometry(m.coords, m.elem, m.elem_type, d)
    K_b, G_b = OC.moduli(prob.material.E, prob.material.nu)
    Ce = OC.elastic_tangent(K_b, G_b)
    if d == 2:
        Ce = Ce[np.ix_(OC.PLANE_INPLANE_IDX, OC.PLANE_INPLANE_IDX)]
    Kel = Assembler(g, Ce).K_elast.tocsr()
    st, rp, ci, _ = _pattern(shim, m.n_nodes, m.elem)
    assert st == 1
    vals = np.zeros((len(ci), d, d))
    for n in range(m.n_nodes):
        for k in range(rp[n], rp[n + 1]):
            vals[k] = Kel[n * d:(n + 1) * d, ci[k] * d:(ci[k] + 1) * d].toarray()
    free = (prob.dirichlet == 0).astype(np.uint8)
    coords = np.ascontiguousarray(m.coords, dtype=np.float64)
    h = shim.shim_amg_setup(d, m.n_nodes, rp.ctypes.data, ci.ctypes.data, vals.ctypes.data, free.ctypes.data,
                            coords.ctypes.data)
    assert h
    try:
        nl = shim.shim_amg_levels(h)
        assert nl >= 2
        fr = free.astype(bool)
        A = Kel.multiply(np.outer(fr, fr)).tocsr() + sp.diags((~fr).astype(float))
        sizes = []
        for l in range(nl):
            bs, n, lam = C.c_int(), C.c_int64(), C.c_double()
            shim.shim_amg_level(h, l, C.byref(bs), C.byref(n), C.byref(lam))
            sizes.append(n.value)
            assert A.shape == (n.value, n.value)
            nd, nden = C.c_int64(), C.c_int64()
            shim.shim_amg_inv_sizes(h, l, C.byref(nd), C.byref(nden))
            dinv = np.zeros(max(1, nd.value))
            dense = np.zeros(max(1, nden.value))
            shim.shim_amg_inv_copy(h, l, dinv.ctypes.data, dense.ctypes.data)
            if l == nl - 1:                               # coarsest: dense inverse
                Ad = A.toarray()
                assert np.abs(dense.reshape(n.value, n.value) @ Ad - np.eye(n.value)).max() < 1e-8
                break
            b = bs.value
            Dinv = dinv.reshape(-1, b, b)
            for I in range(0, n.value // b, max(1, n.value // b // 50)):
                blk = A[I * b:(I + 1) * b, I * b:(I + 1) * b].toarray()
                assert np.abs(Dinv[I] @ blk - np.eye(b)).max() < 1e-10
            nb = n.value // b
            DA = sp.bsr_matrix((Dinv, np.arange(nb), np.arange(nb + 1)), shape=(n.value, n.value)).tocsr() @ A
            rho = abs(spla.eigs(DA, k=1, which="LM", return_eigenvectors=False)[0])
            assert 0.8 * rho <= lam.value <= 1.3 * rho, (l, lam.value, rho)
            P = _amg_mat(shim, h, l, 1)
            R = _amg_mat(shim, h, l, 2)
            assert abs(R - P.T).max() == 0.0
            G = (P.T @ A @ P).tocsr()
            Anext = _amg_mat(shim, h, l + 1, 0)
            ident = np.nonzero(G.diagonal() == 0.0)[0]
            Gf = G.tolil()
            for i in ident:
                Gf[i, :] = 0.0
                Gf[i, i] = 1.0
            err = abs(Anext - Gf.tocsr()).max() / abs(Anext).max()
            assert err < 1e-12, (l, err)
            A = Anext
        print(f"\n{make}: levels {sizes}")
        assert all(a > b for a, b in zip(sizes, sizes[1:])) and sizes[-1] <= 600
    finally:
        shim.shim_amg_free(h)


# -- sparse LU: symbolic analysis ----------------------------------------------------------------

def _direct_plan(shim, dim, n_nodes, rp, ci, coords, leaf):
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    h = shim.shim_direct_analyse(dim, n_nodes, rp.ctypes.data, ci.ctypes.data, coords.ctypes.data, leaf)
    assert h
    try:
        sz = np.zeros(5, dtype=np.int64)
        shim.shim_direct_sizes(h, sz.ctypes.data)
        nf, nl, nlist = int(sz[0]), int(sz[1]), int(sz[2])
        P = dict(level_ptr=np.zeros(nl + 1, np.int32), parent=np.zeros(nf, np.int32), npiv=np.zeros(nf, np.int32),
                 nupd=np.zeros(nf, np.int32), node_off=np.zeros(nf + 1, np.int64), nodes=np.zeros(nlist, np.int32),
                 umap=np.zeros(nlist, np.int32), blk_front=np.zeros(len(ci), np.int32),
                 blk_row=np.zeros(len(ci), np.int32), blk_col=np.zeros(len(ci), np.int32),
                 pos=np.zeros(n_nodes, np.int32))
        flops = C.c_double(0.0)
        shim.shim_direct_copy(h, *[P[k].ctypes.data for k in ("level_ptr", "parent", "npiv", "nupd", "node_off",
                                                               "nodes", "umap", "blk_front", "blk_row", "blk_col",
                                                               "pos")], C.byref(flops))
        P["flops"] = flops.value
    finally:
        shim.shim_direct_free(h)
    P["n_fronts"] = nf
    return P


def _direct_cases():
    from synthetic import structured_mesh
    out = []
    for et, dim, n in (("P2", 2, (7, 5)), ("P1", 2, (9, 9)), ("Q1", 3, (4, 3, 3)), ("P2", 3, (2, 2, 2))):
        m = structured_mesh(et, dim, n, (10.0,) * dim)
        out.append((f"{et}-{dim}d", dim, m.n_nodes, m.elem, m.coords))
    # two meshes with overlapping coordinates in one graph (a batch): disconnected components
    m = structured_mesh("Q2", 2, (3, 4), (10.0, 10.0))
    elem = np.vstack([m.elem, m.elem + m.n_nodes])
    out.append(("batch-Q2", 2, 2 * m.n_nodes, elem, np.vstack([m.coords, m.coords + 0.5])))
    return out


@pytest.mark.parametrize("case", _direct_cases(), ids=lambda c: c[0])
@pytest.mark.parametrize("leaf", [1, 8, 40])
def test_direct_analysis_fronts_are_the_filled_graph(shim, case, leaf):
    """The nested-dissection plan against brute-force symbolic elimination: the order is a permutation,
    every front's update set is exactly the set of later nodes its pivots are joined to in the filled
    graph, children precede parents and fit into them, and every block lands in the front of its
    first-eliminated node."""
    _, dim, n, elem, coords = case
    st, rp, ci, _ = _pattern(shim, n, elem)
    assert st == 1
    P = _direct_plan(shim, dim, n, rp, ci, coords, leaf)
    pos = P["pos"]
    assert sorted(pos.tolist()) == list(range(n))
    # filled graph by elimination in pos order
    order = np.argsort(pos)
    higher = [set(int(w) for w in ci[rp[v]:rp[v + 1]] if pos[w] > pos[v]) for v in range(n)]
    for v in order:
        hv = sorted(higher[v], key=lambda w: pos[w])
        for i, a in enumerate(hv):
            higher[a].update(hv[i + 1:])
    nf = P["n_fronts"]
    lists = [P["nodes"][P["node_off"][s]:P["node_off"][s + 1]] for s in range(nf)]
    assert P["level_ptr"][0] == 0 and P["level_ptr"][-1] == nf
    seen = 0
    for s in range(nf):
        k, u = P["npiv"][s], P["nupd"][s]
        piv, upd = lists[s][:k].tolist(), lists[s][k:].tolist()
        assert k >= 1 and len(upd) == u
        assert sorted(pos[piv].tolist()) == list(range(seen, seen + k))    # processing order = elimination order
        seen += k
        want = set().union(*[higher[v] for v in piv]) - set(piv)
        assert set(upd) == want
        assert all(pos[a] < pos[b] for a, b in zip(upd, upd[1:]))
        p = P["parent"][s]
        if p >= 0:
            assert p > s
            plist = lists[p].tolist()
            for a, w in enumerate(upd):
                assert plist[P["umap"][P["node_off"][s] + k + a]] == w
        else:
            assert u == 0
    assert seen == n
    # blocks
    for r in range(n):
        for b in range(rp[r], rp[r + 1]):
            c = ci[b]
            s = P["blk_front"][b]
            lst = lists[s]
            assert lst[P["blk_row"][b]] == r and lst[P["blk_col"][b]] == c
            first = r if pos[r] <= pos[c] else c
            assert first in lst[:P["npiv"][s]].tolist()


def test_direct_plan_factorises_exactly(shim):
    """A plain numpy multifrontal pass over the plan (assemble the blocks, partial LU without row
    exchanges, extend-add into the parent) gives factors with L U = P A P^T for a nonsymmetric,
    diagonally dominant matrix on a P2 pattern; nested dissection beats the natural order on fill."""
    from synthetic import structured_mesh
    dim = 2
    m = structured_mesh("P2", 2, (6, 6), (10.0, 10.0))
    n = m.n_nodes
    st, rp, ci, _ = _pattern(shim, n, m.elem)
    rng = np.random.default_rng(7)
    nnzb = len(ci)
    vals = rng.uniform(-1.0, 1.0, (nnzb, dim, dim))
    A = np.zeros((n * dim, n * dim))
    for r in range(n):
        for b in range(rp[r], rp[r + 1]):
            A[r * dim:(r + 1) * dim, ci[b] * dim:(ci[b] + 1) * dim] = vals[b]
    A += np.diag(np.abs(A).sum(axis=1) + 1.0)
    for r in range(n):
        for b in range(rp[r], rp[r + 1]):
            if ci[b] == r:
                vals[b] = A[r * dim:(r + 1) * dim, r * dim:(r + 1) * dim]
    P = _direct_plan(shim, dim, n, rp, ci, m.coords, 8)
    nf = P["n_fronts"]
    F = []
    for s in range(nf):
        sz = (P["npiv"][s] + P["nupd"][s]) * dim
        F.append(np.zeros((sz, sz)))
    for r in range(n):
        for b in range(rp[r], rp[r + 1]):
            s = P["blk_front"][b]
            i, j = P["blk_row"][b] * dim, P["blk_col"][b] * dim
            F[s][i:i + dim, j:j + dim] = vals[b]
    dof = lambda node, c: node * dim + c
    L = np.eye(n * dim)
    U = np.zeros((n * dim, n * dim))
    gpos = np.zeros(n * dim, dtype=np.int64)   # global DOF -> position in the permuted order
    for v in range(n):
        for c in range(dim):
            gpos[dof(v, c)] = P["pos"][v] * dim + c
    for s in range(nf):
        lst = P["nodes"][P["node_off"][s]:P["node_off"][s + 1]]
        gl = np.array([gpos[dof(v, c)] for v in lst for c in range(dim)])
        k = P["npiv"][s] * dim
        Fs = F[s]
        for t in range(k):
            Fs[t + 1:, t] /= Fs[t, t]
            Fs[t + 1:, t + 1:] -= np.outer(Fs[t + 1:, t], Fs[t, t + 1:])
        for t in range(k):
            U[gl[t], gl[t:]] = Fs[t, t:]
            L[gl[t + 1:], gl[t]] = Fs[t + 1:, t]
        p = P["parent"][s]
        if p >= 0:
            um = P["umap"][P["node_off"][s] + P["npiv"][s]:P["node_off"][s + 1]]
            idx = np.array([a * dim + c for a in um for c in range(dim)])
            F[p][np.ix_(idx, idx)] += Fs[k:, k:]
    perm = np.argsort(gpos)
    Ap = A[np.ix_(perm, perm)]
    assert np.abs(L @ U - Ap).max() <= 1e-12 * np.abs(A).max()
    assert np.allclose(np.triu(U), U) and np.allclose(np.tril(L), L)
    # fill: nested dissection against the natural order's band
    fill_nd = np.count_nonzero(np.abs(L) > 0) + np.count_nonzero(np.abs(U) > 0)
    assert P["flops"] > 0 and fill_nd < (n * dim) ** 2 / 2


def test_direct_plan_of_the_benchmark_mesh(shim):
    """The nested-dissection plan of the 256x256 P2 column with the library's leaves of 16 nodes: the
    structure the factorisation's cost follows (32 767 fronts on 15 levels, the root a separator of
    513 nodes, 41.6 GFLOP; leaves of 64 nodes gave 50.7)."""
    from synthetic import structured_mesh
    m = structured_mesh("P2", 2, (256, 256), (10.0, 10.0))
    st, rp, ci, _ = _pattern(shim, m.n_nodes, m.elem)
    assert st == 1
    P = _direct_plan(shim, 2, m.n_nodes, rp, ci, m.coords, 16)
    nf = P["n_fronts"]
    assert nf == 32767 and len(P["level_ptr"]) - 1 == 15
    root = nf - 1
    assert P["parent"][root] == -1 and P["npiv"][root] == 513 and P["nupd"][root] == 0
    order = (P["npiv"] + P["nupd"]) * 2
    assert order.max() == 1538
    assert abs(P["flops"] / 1e9 - 41.6) < 0.1
