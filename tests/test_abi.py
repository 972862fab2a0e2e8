"""The C-ABI library builds, loads and exports every function include/ep.h declares.

No compute calls: these run on a machine without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "ep.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(ep_[a-z_]+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1805_04155_gb300 import build as b
    return b.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ep_create", "ep_destroy", "ep_solve_load_path", "ep_get", "ep_set", "ep_assemble",
                 "ep_commit", "ep_linear_solve", "ep_constitutive", "ep_status_str", "ep_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(libpath):
    import paper_1805_04155_gb300.ep as ep
    assert sorted(ep.EXPORTED) == _declared()
    lib = ep.lib()
    assert lib.ep_status_str(0) == b"ok"
    assert lib.ep_status_str(4) == b"element with det J <= 0"


def test_struct_layouts_match_header(libpath):
    """ctypes structures have the C sizes implied by the header's field lists."""
    import paper_1805_04155_gb300.ep as ep
    assert ctypes.sizeof(ep.ep_mesh) == 4 + 4 + 8 + 8 + 8 + 8
    assert ctypes.sizeof(ep.ep_material) == 8 + 8 * 8
    # ..., asm_tile, krylov_graphs, direct_fallback and 4 bytes of padding to the struct's 8-byte alignment
    assert ctypes.sizeof(ep.ep_opts) == 4 + 4 + 8 + 4 + 4 + 8 + 4 + 4 + 4 + 4 + 4 + 4 + 4 + 4 + 4 + 4
    assert ctypes.sizeof(ep.ep_step_report) == 4 + 4 + 8 + 8 * 4 + 4 * 4 + 8 * 2 + 8 + 4 * 4 + 8 + 8 + 4 + 4 + 4 + 4 + 8 * 4
    o = ep.default_opts()   # calls into the library (host only)
    assert o.newton_rtol == 1e-10 and o.precond == 2 and o.split_elastic_cache == 1 and o.direct_fallback == 1


def test_create_rejects_bad_input_without_gpu_work(libpath):
    """Argument validation happens before any CUDA call."""
    import numpy as np
    import paper_1805_04155_gb300.ep as ep
    lib = ep.lib()
    h = ctypes.c_void_p()
    coords = np.zeros((3, 2))
    elem = np.array([[0, 1, 2]], dtype=np.int32)
    mesh = ep.ep_mesh(4, 0, 3, 1, coords.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      elem.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    mat = ep.ep_material(0, 1.0, 0.3, 0, 0, 0, 0, 0, 0)
    mask = np.zeros(6, dtype=np.uint8)
    bc = ep.ep_bc(mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), None, None)
    st = lib.ep_create(ctypes.byref(h), ctypes.byref(mesh), ctypes.byref(mat), ctypes.byref(bc), 0, None)
    assert st == ep.EP_ERR_INVALID_ARG      # dim = 4
    assert lib.ep_create(None, None, None, None, 0, None) == ep.EP_ERR_INVALID_ARG


def test_batch_rejects_mixed_element_types_without_gpu_work(libpath):
    """ep_create_batch validates the problems before any CUDA call."""
    import numpy as np
    import paper_1805_04155_gb300.ep as ep
    lib = ep.lib()
    c2 = np.zeros((3, 2)); e2 = np.array([[0, 1, 2]], dtype=np.int32)
    c3 = np.zeros((4, 3)); e3 = np.array([[0, 1, 2, 3]], dtype=np.int32)
    P = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t))
    meshes = (ep.ep_mesh * 2)(ep.ep_mesh(2, 0, 3, 1, P(c2, ctypes.c_double), P(e2, ctypes.c_int32)),
                              ep.ep_mesh(3, 0, 4, 1, P(c3, ctypes.c_double), P(e3, ctypes.c_int32)))
    mats = (ep.ep_material * 2)(ep.ep_material(0, 1.0, 0.3, 0, 0, 0, 0, 0, 0), ep.ep_material(0, 1.0, 0.3, 0, 0, 0, 0, 0, 0))
    m2 = np.zeros(6, dtype=np.uint8); m3 = np.zeros(12, dtype=np.uint8)
    bcs = (ep.ep_bc * 2)(ep.ep_bc(P(m2, ctypes.c_uint8), None, None), ep.ep_bc(P(m3, ctypes.c_uint8), None, None))
    h = ctypes.c_void_p()
    assert lib.ep_create_batch(ctypes.byref(h), 2, meshes, mats, bcs, 0, None) == ep.EP_ERR_INVALID_ARG
    assert b"different element type" in lib.ep_last_error(None)


def test_warm_start_calls_reject_bad_input_without_gpu_work(libpath):
    """The network and recording entry points validate their arguments before any CUDA call."""
    import paper_1805_04155_gb300.ep as ep
    lib = ep.lib()
    h = ctypes.c_void_p()
    assert lib.ep_mlp_create(ctypes.byref(h), None, 0, None) == ep.EP_ERR_INVALID_ARG
    assert lib.ep_mlp_create(None, None, 0, None) == ep.EP_ERR_INVALID_ARG
    assert lib.ep_mlp_forward(None, None, 4, None) == ep.EP_ERR_INVALID_ARG
    assert lib.ep_mlp_train_step(None, None, None, 4, 1e-3, None) == ep.EP_ERR_INVALID_ARG
    assert lib.ep_ws_record(None, 10) == ep.EP_ERR_INVALID_ARG
    assert lib.ep_ws_attach(None, None) == ep.EP_ERR_INVALID_ARG
    assert lib.ep_mlp_destroy(None) == ep.EP_OK


def test_warm_start_sizes_match_the_oracle():
    import paper_1805_04155_gb300.ep as ep
    from oracle import warm_start as W
    text = open(os.path.join(ROOT, "include", "ep.h")).read()
    for name, val in (("EP_WS_N_IN", W.N_IN), ("EP_WS_WIDTH", W.WIDTH), ("EP_WS_N_OUT", W.N_OUT),
                      ("EP_WS_N_PARAMS", W.N_PARAMS)):
        assert re.search(rf"#define {name} {val}\b", text), name
        assert getattr(ep, name) == val


def test_network_binding_checks_the_parameter_count(libpath):
    """The binding rejects a parameter vector of the wrong length before calling the library."""
    import numpy as np
    import paper_1805_04155_gb300.ep as ep
    with pytest.raises(ValueError):
        ep.MLP(np.zeros(ep.EP_WS_N_PARAMS - 1, dtype=np.float32))


def test_constitutive_with_no_points_returns_ok_without_gpu_work(libpath):
    """n = 0 is a valid empty call: it returns before touching any pointer or the device."""
    import paper_1805_04155_gb300.ep as ep
    lib = ep.lib()
    mat = ep.ep_material(1, 206900.0, 0.29, 367.4, 1e4, 0, 0, 0, 0)
    args = [None] * 8
    assert lib.ep_constitutive(ctypes.byref(mat), 2, 0, *args, None) == ep.EP_OK
    assert lib.ep_constitutive(ctypes.byref(mat), 4, 0, *args, None) == ep.EP_ERR_INVALID_ARG   # dim
