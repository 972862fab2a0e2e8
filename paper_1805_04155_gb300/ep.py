"""Thin ctypes binding of include/ep.h (argument marshalling only).

Every computation runs in libep.so's CUDA kernels.  Importing this module
loads the library and raises if it is missing: there is no CPU fallback.
Functions keep the C names (ep_create, ep_solve_load_path, ...); `Context`
bundles them for numpy / torch callers.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libep.so")

# ep_status
EP_OK, EP_ERR_INVALID_ARG, EP_ERR_CUDA, EP_ERR_OOM, EP_ERR_BAD_ELEMENT, EP_ERR_RETURN_MAP, \
    EP_ERR_NEWTON_NO_CONVERGENCE, EP_ERR_KRYLOV, EP_ERR_NAN, EP_ERR_STATE = range(10)
# ep_elem
EP_P1, EP_P2, EP_Q1, EP_Q2 = range(4)
ELEM_IDS = {"P1": EP_P1, "P2": EP_P2, "Q1": EP_Q1, "Q2": EP_Q2}
# ep_model
EP_ELASTIC, EP_VM_KIN, EP_VM_ISO, EP_DP = range(4)
# ep_precision
EP_FP64, EP_MIXED = range(2)
# ep_field
(EP_U, EP_STRESS, EP_PLASTIC_STRAIN, EP_HARDENING, EP_PLASTIC_FLAG, EP_F_INT, EP_K_ROW_PTR, EP_K_COL_IDX,
 EP_K_VALUES, EP_K_ELASTIC, EP_WEIGHT, EP_DPHI, EP_SOLUTION, EP_K_VALUES_F32, EP_WS_X, EP_WS_T,
 EP_WS_START) = range(17)
# learned warm start
EP_WS_N_IN, EP_WS_WIDTH, EP_WS_N_OUT, EP_WS_N_PARAMS = 16, 128, 4, 19204

EXPORTED = [
    "ep_default_opts", "ep_create", "ep_create_batch", "ep_destroy", "ep_get_info", "ep_solve_load_path", "ep_get", "ep_set",
    "ep_reset",
    "ep_assemble", "ep_assemble_prec", "ep_commit", "ep_linear_solve", "ep_constitutive", "ep_status_str", "ep_last_error",
    "ep_linear_solve_noalloc", "ep_mlp_create", "ep_mlp_destroy", "ep_mlp_get_params", "ep_mlp_forward", "ep_mlp_grad",
    "ep_mlp_train_step", "ep_ws_record", "ep_ws_samples", "ep_ws_attach",
]
EP_NOALLOC_MAX_DOF = 32768
EP_NOALLOC_MAX_ITERATIONS = 10000


class ep_mesh(C.Structure):
    _fields_ = [("dim", C.c_int32), ("elem", C.c_int32), ("n_nodes", C.c_int64), ("n_elem", C.c_int64),
                ("coords", C.POINTER(C.c_double)), ("elem_nodes", C.POINTER(C.c_int32))]


class ep_material(C.Structure):
    _fields_ = [("model", C.c_int32), ("E", C.c_double), ("nu", C.c_double), ("Y", C.c_double),
                ("H", C.c_double), ("c0", C.c_double), ("phi", C.c_double), ("psi", C.c_double),
                ("Hc", C.c_double)]


class ep_bc(C.Structure):
    _fields_ = [("dirichlet_mask", C.POINTER(C.c_uint8)), ("u_D_unit", C.POINTER(C.c_double)),
                ("f_ext_unit", C.POINTER(C.c_double))]


class ep_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("newton_rtol", C.c_double), ("newton_maxit", C.c_int32),
                ("krylov", C.c_int32), ("krylov_rtol", C.c_double), ("krylov_maxit", C.c_int32),
                ("precond", C.c_int32), ("split_elastic_cache", C.c_int32), ("warm_start", C.c_int32),
                ("profile", C.c_int32), ("deterministic", C.c_int32), ("asm_tile", C.c_int32),
                ("krylov_graphs", C.c_int32), ("direct_fallback", C.c_int32)]


class ep_step_report(C.Structure):
    _fields_ = [("newton_its", C.c_int32), ("krylov_its", C.c_int32), ("n_plastic", C.c_int64),
                ("rel_resid", C.c_double), ("t_assemble_ms", C.c_double), ("t_solve_ms", C.c_double),
                ("t_step_ms", C.c_double), ("status", C.c_int32), ("launches", C.c_int32),
                ("n_assemble", C.c_int32), ("n_spmv", C.c_int32), ("t_assemble_kernel_ms", C.c_double),
                ("t_spmv_kernel_ms", C.c_double), ("n_plastic_assembled", C.c_int64),
                ("newton_its_fp32", C.c_int32), ("start", C.c_int32), ("n_learned", C.c_int32),
                ("n_smooth0", C.c_int32), ("t_smooth0_kernel_ms", C.c_double),
                ("n_plastic_elem_assembled", C.c_int64), ("precise", C.c_int32), ("direct", C.c_int32),
                ("n_direct_factor", C.c_int32), ("n_direct_solve", C.c_int32), ("t_direct_factor_ms", C.c_double),
                ("t_direct_solve_ms", C.c_double), ("direct_factor_flop", C.c_double),
                ("direct_solve_bytes", C.c_double)]


class ep_info(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_elem", C.c_int64), ("n_int", C.c_int64), ("nnz_blocks", C.c_int64),
                ("dim", C.c_int32), ("n_p", C.c_int32), ("n_q", C.c_int32), ("n_comp", C.c_int32)]


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"libep.so not found at {path}; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
    lib = C.CDLL(path)
    vp, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
    dp = C.POINTER(C.c_double)
    lib.ep_default_opts.argtypes = [C.POINTER(ep_opts)]
    lib.ep_default_opts.restype = None
    lib.ep_create.argtypes = [C.POINTER(vp), C.POINTER(ep_mesh), C.POINTER(ep_material), C.POINTER(ep_bc), i32, vp]
    lib.ep_create_batch.argtypes = [C.POINTER(vp), i32, C.POINTER(ep_mesh), C.POINTER(ep_material), C.POINTER(ep_bc),
                                    i32, vp]
    lib.ep_destroy.argtypes = [vp]
    lib.ep_get_info.argtypes = [vp, C.POINTER(ep_info)]
    lib.ep_solve_load_path.argtypes = [vp, i32, dp, C.POINTER(ep_opts), C.POINTER(ep_step_report)]
    lib.ep_get.argtypes = [vp, i32, vp, sz, i32]
    lib.ep_set.argtypes = [vp, i32, vp, sz, i32]
    lib.ep_reset.argtypes = [vp]
    lib.ep_assemble.argtypes = [vp, vp, i32, i32, C.POINTER(i64)]
    lib.ep_assemble_prec.argtypes = [vp, vp, i32, i32, i32, C.POINTER(i64)]
    lib.ep_commit.argtypes = [vp, vp, i32]
    lib.ep_linear_solve.argtypes = [vp, vp, i32, C.POINTER(ep_opts), C.POINTER(i32), dp]
    lib.ep_constitutive.argtypes = [C.POINTER(ep_material), i32, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.ep_linear_solve_noalloc.argtypes = [i32, i64, vp, vp, vp, vp, vp, vp, vp, i32, i32, C.c_double, i32,
                                            C.POINTER(i32), dp, vp]
    lib.ep_linear_solve_noalloc.restype = i32
    fp = C.POINTER(C.c_float)
    lib.ep_mlp_create.argtypes = [C.POINTER(vp), fp, i32, vp]
    lib.ep_mlp_destroy.argtypes = [vp]
    lib.ep_mlp_get_params.argtypes = [vp, fp]
    lib.ep_mlp_forward.argtypes = [vp, vp, i64, vp]
    lib.ep_mlp_grad.argtypes = [vp, vp, vp, i64, dp, fp]
    lib.ep_mlp_train_step.argtypes = [vp, vp, vp, i64, C.c_float, dp]
    lib.ep_ws_record.argtypes = [vp, i64]
    lib.ep_ws_samples.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(i64)]
    lib.ep_ws_attach.argtypes = [vp, vp]
    lib.ep_status_str.argtypes = [i32]
    lib.ep_status_str.restype = C.c_char_p
    lib.ep_last_error.argtypes = [vp]
    lib.ep_last_error.restype = C.c_char_p
    for name in ("ep_create", "ep_create_batch", "ep_destroy", "ep_get_info", "ep_solve_load_path", "ep_get", "ep_set", "ep_assemble",
                 "ep_assemble_prec", "ep_commit", "ep_linear_solve", "ep_constitutive", "ep_mlp_create", "ep_mlp_destroy",
                 "ep_mlp_get_params", "ep_mlp_forward", "ep_mlp_grad", "ep_mlp_train_step", "ep_ws_record",
                 "ep_ws_samples", "ep_ws_attach"):
        getattr(lib, name).restype = i32
    return lib


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


class EPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{lib().ep_status_str(status).decode()} ({status}): {msg}")
        self.status = status


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def default_opts(**kw) -> ep_opts:
    o = ep_opts()
    lib().ep_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def make_material(m) -> ep_material:
    """From any object with model, E, nu, Y, H, c0, phi, psi, Hc attributes."""
    return ep_material(int(m.model), float(m.E), float(m.nu), float(getattr(m, "Y", 0.0)), float(getattr(m, "H", 0.0)),
                       float(getattr(m, "c0", 0.0)), float(getattr(m, "phi", 0.0)), float(getattr(m, "psi", 0.0)),
                       float(getattr(m, "Hc", 0.0)))


def _stream_ptr(stream) -> int:
    if stream is None:
        try:
            import torch
            return int(torch.cuda.current_stream().cuda_stream)
        except Exception:
            return 0
    return int(getattr(stream, "cuda_stream", stream))


class Context:
    """One ep_create context.  Arrays are numpy (host) or torch CUDA tensors (device)."""

    def __init__(self, coords, elem, elem_type: str, material, dirichlet, u_D_unit=None, f_ext_unit=None,
                 device: int = 0, stream=None):
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        elem = np.ascontiguousarray(elem, dtype=np.int32)
        dim = coords.shape[1]
        self._keep = []
        mesh = ep_mesh(dim, ELEM_IDS[elem_type], coords.shape[0], elem.shape[0], _ptr(coords, C.c_double),
                       _ptr(elem, C.c_int32))
        mask = np.ascontiguousarray(dirichlet, dtype=np.uint8)
        uD = None if u_D_unit is None else np.ascontiguousarray(u_D_unit, dtype=np.float64)
        fe = None if f_ext_unit is None else np.ascontiguousarray(f_ext_unit, dtype=np.float64)
        bc = ep_bc(_ptr(mask, C.c_uint8), None if uD is None else _ptr(uD, C.c_double),
                   None if fe is None else _ptr(fe, C.c_double))
        self.material = make_material(material)
        h = C.c_void_p()
        st = lib().ep_create(C.byref(h), C.byref(mesh), C.byref(self.material), C.byref(bc), int(device),
                             C.c_void_p(_stream_ptr(stream)))
        if st != EP_OK:
            raise EPError(st, lib().ep_last_error(None).decode())
        self.h = h
        info = ep_info()
        lib().ep_get_info(h, C.byref(info))
        self.info = info
        self.dim = info.dim
        self.n_dof = info.n_nodes * info.dim

    @classmethod
    def from_problem(cls, problem, **kw):
        m = problem.mesh
        return cls(m.coords, m.elem, m.elem_type, problem.material, problem.dirichlet, problem.u_D_unit,
                   problem.f_unit, **kw)

    @classmethod
    def from_batch(cls, problems, device: int = 0, stream=None):
        """ep_create_batch over problems of one element type; fields are concatenated in order."""
        n = len(problems)
        meshes, mats, bcs = (ep_mesh * n)(), (ep_material * n)(), (ep_bc * n)()
        keep = []
        for i, pb in enumerate(problems):
            m = pb.mesh
            co = np.ascontiguousarray(m.coords, dtype=np.float64)
            el = np.ascontiguousarray(m.elem, dtype=np.int32)
            mk = np.ascontiguousarray(pb.dirichlet, dtype=np.uint8)
            ud = np.ascontiguousarray(pb.u_D_unit, dtype=np.float64)
            fe = np.ascontiguousarray(pb.f_unit, dtype=np.float64)
            keep += [co, el, mk, ud, fe]
            meshes[i] = ep_mesh(co.shape[1], ELEM_IDS[m.elem_type], co.shape[0], el.shape[0], _ptr(co, C.c_double),
                                _ptr(el, C.c_int32))
            mats[i] = make_material(pb.material)
            bcs[i] = ep_bc(_ptr(mk, C.c_uint8), _ptr(ud, C.c_double), _ptr(fe, C.c_double))
        h = C.c_void_p()
        st = lib().ep_create_batch(C.byref(h), n, meshes, mats, bcs, int(device), C.c_void_p(_stream_ptr(stream)))
        if st != EP_OK:
            raise EPError(st, lib().ep_last_error(None).decode())
        self = cls.__new__(cls)
        self._keep = []
        self.h = h
        self.material = mats[0]
        info = ep_info()
        lib().ep_get_info(h, C.byref(info))
        self.info = info
        self.dim = info.dim
        self.n_dof = info.n_nodes * info.dim
        self.node_off = np.cumsum([0] + [pb.mesh.n_nodes for pb in problems])
        self.ip_off = np.cumsum([0] + [pb.mesh.n_elem for pb in problems]) * info.n_q
        return self

    def split(self, field, arr):
        """Per-problem views of a concatenated batch field (EP_U, EP_F_INT, or a [n_comp][n_int] field)."""
        if field in (EP_U, EP_F_INT, EP_SOLUTION):
            o = self.node_off * self.dim
            return [arr[o[i]:o[i + 1]] for i in range(len(o) - 1)]
        o = self.ip_off
        return [arr[..., o[i]:o[i + 1]] for i in range(len(o) - 1)]

    def close(self):
        if getattr(self, "h", None):
            lib().ep_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != EP_OK:
            raise EPError(st, lib().ep_last_error(self.h).decode())

    # -- sizes -----------------------------------------------------------------
    def field_shape(self, field):
        i = self.info
        nc = i.n_comp
        hard_vec = self.material.model == EP_VM_KIN
        return {
            EP_U: ((self.n_dof,), np.float64), EP_STRESS: ((nc, i.n_int), np.float64),
            EP_PLASTIC_STRAIN: ((nc, i.n_int), np.float64),
            EP_HARDENING: (((nc, i.n_int) if hard_vec else (i.n_int,)), np.float64),
            EP_PLASTIC_FLAG: ((i.n_int,), np.uint8), EP_F_INT: ((self.n_dof,), np.float64),
            EP_K_ROW_PTR: ((i.n_nodes + 1,), np.int32), EP_K_COL_IDX: ((i.nnz_blocks,), np.int32),
            EP_K_VALUES: ((i.nnz_blocks, i.dim, i.dim), np.float64),
            EP_K_ELASTIC: ((i.nnz_blocks, i.dim, i.dim), np.float64), EP_WEIGHT: ((i.n_int,), np.float64),
            EP_DPHI: ((i.n_int, i.n_p, i.dim), np.float64), EP_SOLUTION: ((self.n_dof,), np.float64),
            EP_K_VALUES_F32: ((i.nnz_blocks, i.dim, i.dim), np.float32),
            EP_WS_X: ((self.ws_rows(), EP_WS_N_IN), np.float32), EP_WS_T: ((self.ws_rows(), EP_WS_N_OUT), np.float32),
            EP_WS_START: ((self.n_dof,), np.float64),
        }[field]

    # -- C calls -------------------------------------------------------------------
    def get(self, field, out=None):
        shape, dt = self.field_shape(field)
        if out is None:
            out = np.empty(shape, dtype=dt)
        if isinstance(out, np.ndarray):
            self._check(lib().ep_get(self.h, field, out.ctypes.data, out.nbytes, 0))
        else:   # torch CUDA tensor
            self._check(lib().ep_get(self.h, field, out.data_ptr(), out.numel() * out.element_size(), 1))
        return out

    def set(self, field, src):
        if isinstance(src, np.ndarray):
            _, dt = self.field_shape(field)
            a = np.ascontiguousarray(src, dtype=dt)
            self._check(lib().ep_set(self.h, field, a.ctypes.data, a.nbytes, 0))
        else:
            self._check(lib().ep_set(self.h, field, src.data_ptr(), src.numel() * src.element_size(), 1))

    def reset(self):
        """ep_reset: back to the virgin state (device memsets on the context's stream)."""
        self._check(lib().ep_reset(self.h))

    def _vec_arg(self, v):
        if isinstance(v, np.ndarray):
            a = np.ascontiguousarray(v, dtype=np.float64)
            self._keep = [a]
            return a.ctypes.data, 0
        return v.data_ptr(), 1

    def assemble(self, u, split=True, precision=EP_FP64) -> int:
        p, dev = self._vec_arg(u)
        npl = C.c_int64(0)
        if precision == EP_FP64:
            self._check(lib().ep_assemble(self.h, C.c_void_p(p), dev, int(bool(split)), C.byref(npl)))
        else:
            self._check(lib().ep_assemble_prec(self.h, C.c_void_p(p), dev, int(bool(split)), int(precision),
                                               C.byref(npl)))
        return npl.value

    def commit(self, u):
        p, dev = self._vec_arg(u)
        self._check(lib().ep_commit(self.h, C.c_void_p(p), dev))

    def linear_solve(self, b, opts=None):
        opts = opts or default_opts(krylov_rtol=1e-12)
        p, dev = self._vec_arg(b)
        its = C.c_int32(0)
        rel = C.c_double(0.0)
        self._check(lib().ep_linear_solve(self.h, C.c_void_p(p), dev, C.byref(opts), C.byref(its), C.byref(rel)))
        return self.get(EP_SOLUTION), its.value, rel.value

    def solve_load_path(self, zeta, opts=None, raise_on_error=True):
        z = np.ascontiguousarray(zeta, dtype=np.float64)
        reps = (ep_step_report * max(1, len(z)))()
        st = lib().ep_solve_load_path(self.h, len(z), _ptr(z, C.c_double), C.byref(opts or default_opts()), reps)
        out = [reps[i] for i in range(len(z))]
        if raise_on_error:
            self._check(st)
        return out if raise_on_error else (st, out)

    # -- learned warm start --------------------------------------------------------
    def ws_record(self, max_rows: int):
        """Record up to max_rows (inputs, targets) rows during later load paths (0 stops and frees)."""
        self._check(lib().ep_ws_record(self.h, int(max_rows)))

    def ws_samples_ptr(self):
        """(device address of X [n][16], of T [n][4], n) of the recorded rows."""
        x, t, n = C.c_void_p(), C.c_void_p(), C.c_int64(0)
        self._check(lib().ep_ws_samples(self.h, C.byref(x), C.byref(t), C.byref(n)))
        return x.value or 0, t.value or 0, n.value

    def ws_rows(self) -> int:
        return self.ws_samples_ptr()[2]

    def ws_attach(self, mlp):
        """Use `mlp` (an MLP) for warm_start = 2; None detaches."""
        self._mlp = mlp
        self._check(lib().ep_ws_attach(self.h, None if mlp is None else mlp.h))

    def K_csr(self, elastic=False, f32=False):
        """K as scipy CSR (DOF level) from the block-CSR arrays (f32: the FP32 tangent, as float64)."""
        import scipy.sparse as sp
        rp = self.get(EP_K_ROW_PTR)
        ci = self.get(EP_K_COL_IDX)
        field = EP_K_ELASTIC if elastic else (EP_K_VALUES_F32 if f32 else EP_K_VALUES)
        vals = self.get(field).astype(np.float64)
        return sp.bsr_matrix((vals, ci, rp), shape=(self.n_dof, self.n_dof)).tocsr()


class MLP:
    """ep_mlp_* handle: the warm-start network (16 -> 128 -> 128 -> 4) on one device.  X, T, Y are
    torch CUDA float32 tensors (or device addresses as int)."""

    def __init__(self, params, device: int = 0, stream=None):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.shape != (EP_WS_N_PARAMS,):
            raise ValueError(f"params must have {EP_WS_N_PARAMS} entries")
        h = C.c_void_p()
        st = lib().ep_mlp_create(C.byref(h), _ptr(p, C.c_float), int(device), C.c_void_p(_stream_ptr(stream)))
        if st != EP_OK:
            raise EPError(st, lib().ep_last_error(None).decode())
        self.h = h

    @staticmethod
    def _addr(a):
        return a if isinstance(a, int) else a.data_ptr()

    def _check(self, st, what):
        if st != EP_OK:
            raise EPError(st, what)

    def params(self) -> np.ndarray:
        out = np.empty(EP_WS_N_PARAMS, dtype=np.float32)
        self._check(lib().ep_mlp_get_params(self.h, _ptr(out, C.c_float)), "ep_mlp_get_params")
        return out

    def forward(self, X, Y, n_rows: int | None = None):
        n = X.shape[0] if n_rows is None else n_rows
        self._check(lib().ep_mlp_forward(self.h, C.c_void_p(self._addr(X)), int(n), C.c_void_p(self._addr(Y))),
                    "ep_mlp_forward")

    def grad(self, X, T, n_rows: int | None = None):
        n = X.shape[0] if n_rows is None else n_rows
        loss = C.c_double(0.0)
        g = np.empty(EP_WS_N_PARAMS, dtype=np.float32)
        self._check(lib().ep_mlp_grad(self.h, C.c_void_p(self._addr(X)), C.c_void_p(self._addr(T)), int(n),
                                      C.byref(loss), _ptr(g, C.c_float)), "ep_mlp_grad")
        return loss.value, g

    def train_step(self, X, T, lr: float, n_rows: int | None = None, want_loss: bool = True):
        n = X.shape[0] if n_rows is None else n_rows
        loss = C.c_double(float("nan"))
        self._check(lib().ep_mlp_train_step(self.h, C.c_void_p(self._addr(X)), C.c_void_p(self._addr(T)), int(n),
                                            float(lr), C.byref(loss) if want_loss else None), "ep_mlp_train_step")
        return loss.value

    def close(self):
        if getattr(self, "h", None):
            lib().ep_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def linear_solve_noalloc(dim: int, row_ptr, col_idx, diag_slot, vals, free_dof, b, x, method: int = 1,
                         precond: int = 1, rtol: float = 1e-12, maxit: int = 10000, stream=None):
    """ep_linear_solve_noalloc on torch CUDA tensors (the library allocates nothing for this call).

    row_ptr/col_idx/diag_slot int32, vals float64 [nnzb][dim][dim], free_dof uint8, b and x float64.
    Returns (status, iterations, relative residual); x is filled in place.
    """
    its = C.c_int32(0)
    rel = C.c_double(0.0)
    n_nodes = row_ptr.numel() - 1
    st = lib().ep_linear_solve_noalloc(dim, n_nodes, row_ptr.data_ptr(), col_idx.data_ptr(), diag_slot.data_ptr(),
                                       vals.data_ptr(), free_dof.data_ptr(), b.data_ptr(), x.data_ptr(), method,
                                       precond, rtol, maxit, C.byref(its), C.byref(rel),
                                       C.c_void_p(_stream_ptr(stream)))
    return st, its.value, rel.value


def constitutive(material, dim: int, E, ep_prev, hard_prev, stream=None):
    """Run ep_constitutive on torch CUDA tensors; returns (S, DS, flag, ep_new, hard_new) tensors."""
    import torch
    n = E.shape[1]
    nc = 4 if dim == 2 else 6
    ns = 3 if dim == 2 else 6
    dev = E.device
    S = torch.empty((nc, n), dtype=torch.float64, device=dev)
    DS = torch.empty((ns, ns, n), dtype=torch.float64, device=dev)
    flag = torch.empty((n,), dtype=torch.uint8, device=dev)
    ep_new = torch.empty_like(ep_prev)
    hard_new = torch.empty_like(hard_prev)
    mat = make_material(material)
    st = lib().ep_constitutive(C.byref(mat), dim, n, E.data_ptr(), ep_prev.data_ptr(), hard_prev.data_ptr(),
                               S.data_ptr(), DS.data_ptr(), flag.data_ptr(), ep_new.data_ptr(), hard_new.data_ptr(),
                               C.c_void_p(_stream_ptr(stream)))
    if st != EP_OK:
        raise EPError(st, "ep_constitutive")
    return S, DS, flag, ep_new, hard_new
