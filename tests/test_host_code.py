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
    cmd = [nvcc, "-std=c++17", "-O1", "-Xcompiler", "-fPIC", "-shared", "-x", "c++",
           os.path.join(ROOT, "tests", "host_shim.cpp"), os.path.join(SRC, "pattern_host.cpp"),
           os.path.join(SRC, "elements_host.cpp"), "-I", os.path.join(ROOT, "include"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = C.CDLL(out)
    lib.shim_build_pattern.argtypes = [C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                       C.c_void_p, C.POINTER(C.c_int64)]
    lib.shim_reference_tables.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64]
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
