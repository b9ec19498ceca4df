"""Thin ctypes binding of the C-ABI in include/vms.h (argument marshalling only).

Every computation runs in the CUDA library libvms_gb300.so; if the library is missing this module
raises on load. Arrays may be numpy arrays (host) or torch tensors (host or CUDA); they are
passed as raw pointers after a dtype and contiguity check.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_int, c_int32, c_int64, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvms_gb300.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_CUDA = -2
ERR_OUT_OF_MEMORY = -3
ERR_NEG_JACOBIAN = -4
ERR_SINGULAR_KFF = -5
ERR_NAN = -6
ERR_KRYLOV_MAXIT = -7
ERR_NEWTON_DIVERGED = -8
ERR_STATE = -9
ERR_UNSUPPORTED = -10
ERR_TOO_LARGE = -11
ERR_ZERO_PIVOT = -12
ERR_TIMEOUT = -13
NOALLOC_MAX_ENTRIES = 2097152

PREC_FP64 = 0
PREC_MIXED = 1
PREC_MIXED_TC_BF16 = 2
PREC_MIXED_TC_TF32 = 3
SCATTER_ATOMIC = 0
SCATTER_COLOUR = 1
PRECOND_ILU0 = 0
PRECOND_BLOCK_JACOBI = 1
PRECOND_ILU0_FALLBACK = 2

# every symbol include/vms.h declares
EXPORTS = [
    "vms_create", "vms_destroy", "vms_set_stream", "vms_mesh_upload", "vms_set_params",
    "vms_state_upload", "vms_state_download", "vms_assemble_newton_schur", "vms_get_csr",
    "vms_residual", "vms_element_matrices", "vms_apply", "vms_solve", "vms_newton_step",
    "vms_newton_solve", "vms_last_error", "vms_version", "vms_profile_enable", "vms_profile_read",
    "vms_residual_norm_noalloc", "vms_set_preconditioner", "vms_solver_stats",
    "vms_set_element_viscosity", "vms_set_instances", "vms_solve_instance", "vms_set_graph",
    "vms_set_tuning", "vms_get_tuning", "vms_autotune",
    "vms_mlp_create", "vms_mlp_destroy", "vms_mlp_last_error", "vms_mlp_set_stream",
    "vms_mlp_set_params", "vms_mlp_get_params", "vms_mlp_forward", "vms_mlp_grad", "vms_mlp_adam",
    "vms_mlp_column_rms", "vms_mlp_scale_columns",
    "vms_node_features", "vms_node_increment", "vms_apply_increment", "vms_shift_time",
    "vms_newton_solve_to", "vms_state_download_prev", "vms_mesh_upload_tet", "vms_tet_rule",
    "vms_set_wait_limit", "vms_csr_download", "vms_fma_throughput", "vms_csr_download_async",
    "vms_csr_download_wait",
]
MLP_IN, MLP_WIDTH, MLP_OUT, MLP_PARAMS = 12, 128, 4, 18692
K_NAMES = ["residual", "tangent", "fill", "dirichlet", "reduce", "spmv", "krylov", "precond", "fused"]
SCHEDULE_FUSED = 0
SCHEDULE_TWO_STREAMS = 1


class VmsParams(ctypes.Structure):
    _fields_ = [("nu", c_double), ("visc_factor", c_double), ("dt", c_double),
                ("f", c_double * 3), ("bubble_scale", c_double), ("quad_order", c_int32),
                ("scatter_mode", c_int32)]


class VmsTuning(ctypes.Structure):
    _fields_ = [("tangent_warps", c_int32), ("residual_threads", c_int32),
                ("scatter_mode", c_int32), ("schedule", c_int32), ("ms", c_double)]

    def as_dict(self):
        return {"tangent_warps": self.tangent_warps, "residual_threads": self.residual_threads,
                "scatter_mode": self.scatter_mode, "schedule": self.schedule, "ms": self.ms}


class CsrView(ctypes.Structure):
    _fields_ = [("n_rows", c_int64), ("nnz", c_int64), ("rowptr", c_void_p), ("colidx", c_void_p),
                ("values", c_void_p), ("rhs", c_void_p), ("values_dtype", c_int32),
                ("n_colours", c_int32)]


class VmsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"vms error {code}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libvms_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_0809_4802_gb300.build`")
    lib = ctypes.CDLL(path)
    p = c_void_p
    sig = {
        "vms_create": (c_int, [POINTER(c_void_p), c_int, c_int]),
        "vms_destroy": (c_int, [p]),
        "vms_set_stream": (c_int, [p, p]),
        "vms_mesh_upload": (c_int, [p, c_int64, p, c_int64, p, c_int64, p, p]),
        "vms_set_params": (c_int, [p, POINTER(VmsParams)]),
        "vms_state_upload": (c_int, [p, p, p, p]),
        "vms_state_download": (c_int, [p, p, p]),
        "vms_assemble_newton_schur": (c_int, [p, POINTER(CsrView)]),
        "vms_get_csr": (c_int, [p, POINTER(CsrView)]),
        "vms_residual": (c_int, [p, POINTER(c_double), p]),
        "vms_element_matrices": (c_int, [p, c_int64, c_int64] + [p] * 8),
        "vms_apply": (c_int, [p, p, p]),
        "vms_solve": (c_int, [p, c_double, c_int, c_int, c_int, POINTER(c_int), POINTER(c_double)]),
        "vms_newton_step": (c_int, [p, POINTER(c_double)]),
        "vms_newton_solve": (c_int, [p, c_double, c_int, POINTER(c_int), p]),
        "vms_last_error": (c_char_p, [p]),
        "vms_version": (c_char_p, []),
        "vms_profile_enable": (c_int, [p, c_int]),
        "vms_profile_read": (c_int, [p, c_int, p, p]),
        "vms_set_preconditioner": (c_int, [p, c_int]),
        "vms_set_element_viscosity": (c_int, [p, p]),
        "vms_set_instances": (c_int, [p, c_int64, p, p]),
        "vms_solve_instance": (c_int, [p, c_int64, c_double, c_int, c_int, c_int, POINTER(c_int),
                                       POINTER(c_double)]),
        "vms_set_graph": (c_int, [p, c_int]),
        "vms_set_tuning": (c_int, [p, POINTER(VmsTuning)]),
        "vms_get_tuning": (c_int, [p, POINTER(VmsTuning)]),
        "vms_autotune": (c_int, [p, c_int, POINTER(VmsTuning)]),
        "vms_mlp_create": (c_int, [POINTER(c_void_p), c_int]),
        "vms_mlp_destroy": (c_int, [p]),
        "vms_mlp_last_error": (c_char_p, [p]),
        "vms_mlp_set_stream": (c_int, [p, p]),
        "vms_mlp_set_params": (c_int, [p, p]),
        "vms_mlp_get_params": (c_int, [p, p, c_int]),
        "vms_mlp_forward": (c_int, [p, c_int64, p, p]),
        "vms_mlp_grad": (c_int, [p, c_int64, p, p, p, POINTER(c_double), p]),
        "vms_mlp_adam": (c_int, [p, ctypes.c_float]),
        "vms_mlp_column_rms": (c_int, [p, c_int64, c_int, p, p]),
        "vms_mlp_scale_columns": (c_int, [p, c_int64, c_int, p, p, p]),
        "vms_node_features": (c_int, [p, p, p]),
        "vms_node_increment": (c_int, [p, p, p]),
        "vms_apply_increment": (c_int, [p, p, p]),
        "vms_shift_time": (c_int, [p]),
        "vms_newton_solve_to": (c_int, [p, c_double, c_int, POINTER(c_int), p]),
        "vms_state_download_prev": (c_int, [p, p]),
        "vms_mesh_upload_tet": (c_int, [p, c_int64, p, c_int64, p, c_int64, p, p]),
        "vms_tet_rule": (c_int, [c_int, p, p]),
        "vms_solver_stats": (c_int, [p, c_int, POINTER(c_int64), POINTER(c_int64)]),
        "vms_residual_norm_noalloc": (c_int, [c_int64, p, c_int64, p, c_int64, p, p, p, p,
                                              POINTER(VmsParams), p, p, p]),
        "vms_set_wait_limit": (c_int, [p, c_int64]),
        "vms_csr_download": (c_int, [p, p, p, p, p]),
        "vms_csr_download_async": (c_int, [p, p, p, p, p]),
        "vms_csr_download_wait": (c_int, [p]),
        "vms_fma_throughput": (c_int, [c_int, c_int, POINTER(c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a, dtype, n=None, writable=False):
    """Raw pointer of a numpy array or torch tensor with the expected dtype (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a C-contiguous {np.dtype(dtype)} array")
        if writable and not a.flags["WRITEABLE"]:
            raise TypeError("array is read-only")
        if n is not None and a.size != n:
            raise ValueError(f"expected {n} entries, got {a.size}")
        return a.ctypes.data
    import torch  # noqa: PLC0415
    if isinstance(a, torch.Tensor):
        tmap = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64,
                np.float32: torch.float32}
        if a.dtype != tmap[np.dtype(dtype).type] or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {np.dtype(dtype)} tensor")
        if n is not None and a.numel() != n:
            raise ValueError(f"expected {n} entries, got {a.numel()}")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


class DeviceArray:
    """A borrowed device buffer exposed through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr, shape, typestr, owner):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}
        self._owner = owner


class Context:
    """One library context (one GPU, one precision mode)."""

    def __init__(self, device: int = 0, precision: int = PREC_FP64):
        self.lib = load_library()
        h = c_void_p()
        rc = self.lib.vms_create(byref(h), device, precision)
        if rc != OK:
            raise VmsError(rc, "vms_create failed")
        self.h = h
        self.precision = precision
        self.n_nodes = self.n_elems = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.vms_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            raise VmsError(rc, self.lib.vms_last_error(self.h).decode())
        return rc

    # -- setup -------------------------------------------------------------------------------
    def set_stream(self, stream_handle: int):
        self._check(self.lib.vms_set_stream(self.h, c_void_p(stream_handle)))

    def set_preconditioner(self, kind: int):
        self._check(self.lib.vms_set_preconditioner(self.h, int(kind)))

    def set_params(self, nu, visc_factor=2.0, dt=0.0, f=(0.0, 0.0, 0.0), bubble_scale=1.0,
                   quad_order=3, scatter_mode=SCATTER_ATOMIC):
        p = VmsParams(nu, visc_factor, dt, (c_double * 3)(*f), bubble_scale, quad_order,
                      scatter_mode)
        self._check(self.lib.vms_set_params(self.h, byref(p)))

    def mesh_upload(self, xyz, conn, dir_dofs, dir_vals):
        """Upload a mesh: conn (n_elems, 8) hexahedra or (n_elems, 4) tetrahedra."""
        n_nodes = int(xyz.shape[0])
        n_elems = int(conn.shape[0])
        npe = int(conn.shape[1])
        if npe not in (4, 8):
            raise ValueError("elements must have 4 or 8 nodes")
        n_dir = int(dir_dofs.shape[0]) if dir_dofs is not None else 0
        fn = self.lib.vms_mesh_upload if npe == 8 else self.lib.vms_mesh_upload_tet
        self._check(fn(
            self.h, n_nodes, _ptr(xyz, np.float64, 3 * n_nodes), n_elems,
            _ptr(conn, np.int32, npe * n_elems), n_dir,
            _ptr(dir_dofs, np.int64, n_dir) if n_dir else None,
            _ptr(dir_vals, np.float64, n_dir) if n_dir else None))
        self.n_nodes, self.n_elems, self.npe = n_nodes, n_elems, npe

    def state_upload(self, u, beta=None, u_prev=None):
        self._check(self.lib.vms_state_upload(
            self.h, _ptr(u, np.float64, 4 * self.n_nodes),
            _ptr(beta, np.float64, 3 * self.n_elems), _ptr(u_prev, np.float64, 4 * self.n_nodes)))

    def state_download(self):
        u = np.empty((self.n_nodes, 4))
        beta = np.empty((self.n_elems, 3))
        self._check(self.lib.vms_state_download(self.h, u.ctypes.data, beta.ctypes.data))
        return u, beta

    def state_download_prev(self):
        up = np.empty((self.n_nodes, 4))
        self._check(self.lib.vms_state_download_prev(self.h, up.ctypes.data))
        return up

    # -- the hot path ---------------------------------------------------------------------
    def assemble(self) -> CsrView:
        v = CsrView()
        self._check(self.lib.vms_assemble_newton_schur(self.h, byref(v)))
        return v

    def csr(self) -> CsrView:
        v = CsrView()
        self._check(self.lib.vms_get_csr(self.h, byref(v)))
        return v

    def csr_device(self, view: CsrView | None = None):
        """(rowptr, colidx, values, rhs) as zero-copy torch CUDA tensors of the last assembly."""
        import torch  # noqa: PLC0415
        v = view or self.csr()
        vt = "<f4" if v.values_dtype == 1 else "<f8"
        mk = lambda ptr, n, t: torch.as_tensor(DeviceArray(ptr, (n,), t, self), device="cuda")  # noqa: E731
        return (mk(v.rowptr, v.n_rows + 1, "<i4"), mk(v.colidx, v.nnz, "<i4"),
                mk(v.values, v.nnz, vt), mk(v.rhs, v.n_rows, "<f8"))

    def csr_host(self):
        rowptr, colidx, vals, rhs = self.csr_device()
        return (rowptr.cpu().numpy(), colidx.cpu().numpy(), vals.cpu().numpy(), rhs.cpu().numpy())

    def csr_download(self, rowptr=None, colidx=None, values=None, rhs=None):
        """Copy the last assembled system into caller buffers (numpy arrays or torch tensors, host
        or device; values FP32 in mixed precision, FP64 otherwise)."""
        vdt = np.float32 if self.precision != PREC_FP64 else np.float64
        self._check(self.lib.vms_csr_download(self.h, _ptr(rowptr, np.int32), _ptr(colidx, np.int32),
                                              _ptr(values, vdt), _ptr(rhs, np.float64)))

    def csr_download_async(self, rowptr=None, colidx=None, values=None, rhs=None):
        """Start copying the last assembled system into caller buffers (page-locked host buffers
        overlap with the next assembly); csr_download_wait() blocks until it has landed."""
        vdt = np.float32 if self.precision != PREC_FP64 else np.float64
        self._check(self.lib.vms_csr_download_async(self.h, _ptr(rowptr, np.int32), _ptr(colidx, np.int32),
                                                    _ptr(values, vdt), _ptr(rhs, np.float64)))

    def csr_download_wait(self):
        self._check(self.lib.vms_csr_download_wait(self.h))

    def set_wait_limit(self, polls: int):
        """Polls of one device-side wait of the ILU(0) kernels before the solve gives up
        (VMS_ERR_TIMEOUT); 0 restores the default."""
        self._check(self.lib.vms_set_wait_limit(self.h, int(polls)))

    def residual(self, want_vector=False):
        norm = c_double()
        R = np.empty(4 * self.n_nodes + 3 * self.n_elems) if want_vector else None
        self._check(self.lib.vms_residual(self.h, byref(norm), _ptr(R, np.float64)))
        return (norm.value, R) if want_vector else norm.value

    def element_matrices(self, first, count, blocks=True):
        nc = 4 * getattr(self, "npe", 8)
        out = {"S": np.empty((count, nc, nc)), "r": np.empty((count, nc))}
        if blocks:
            out.update(Kcc=np.empty((count, nc, nc)), Kcf=np.empty((count, nc, 3)),
                       Kfc=np.empty((count, 3, nc)), Kff=np.empty((count, 3, 3)),
                       Rcp=np.empty((count, nc)), Rf=np.empty((count, 3)))
        g = lambda k: out[k].ctypes.data if k in out else None  # noqa: E731
        self._check(self.lib.vms_element_matrices(self.h, first, count, g("S"), g("r"), g("Kcc"),
                                                  g("Kcf"), g("Kfc"), g("Kff"), g("Rcp"), g("Rf")))
        return out

    def apply(self, x, y):
        self._check(self.lib.vms_apply(self.h, _ptr(x, np.float64), _ptr(y, np.float64)))

    def set_element_viscosity(self, nu_e):
        self._check(self.lib.vms_set_element_viscosity(
            self.h, _ptr(nu_e, np.float64, self.n_elems) if nu_e is not None else None))

    def set_instances(self, node_offsets, elem_offsets):
        no = np.ascontiguousarray(node_offsets, dtype=np.int64)
        eo = np.ascontiguousarray(elem_offsets, dtype=np.int64)
        if no.shape != eo.shape or no.ndim != 1 or no.size < 2:
            raise ValueError("offsets: two 1-D arrays of count + 1 entries")
        self._check(self.lib.vms_set_instances(self.h, no.size - 1, no.ctypes.data, eo.ctypes.data))

    def solve_instance(self, instance, rtol=1e-12, maxit=50, restart=50, update=True):
        it = c_int()
        rel = c_double()
        self._check(self.lib.vms_solve_instance(self.h, int(instance), rtol, maxit, restart,
                                                int(update), byref(it), byref(rel)))
        return it.value, rel.value

    def set_tuning(self, tangent_warps=0, residual_threads=0, scatter_mode=-1, schedule=SCHEDULE_FUSED):
        t = VmsTuning(tangent_warps, residual_threads, scatter_mode, schedule, 0.0)
        self._check(self.lib.vms_set_tuning(self.h, byref(t)))

    def get_tuning(self):
        t = VmsTuning()
        self._check(self.lib.vms_get_tuning(self.h, byref(t)))
        return t.as_dict()

    def autotune(self, repeats=3):
        t = VmsTuning()
        self._check(self.lib.vms_autotune(self.h, int(repeats), byref(t)))
        return t.as_dict()

    def set_graph(self, enable: bool = True):
        self._check(self.lib.vms_set_graph(self.h, int(enable)))

    def solve(self, rtol=1e-12, maxit=50, restart=50, update=True):
        it = c_int()
        rel = c_double()
        self._check(self.lib.vms_solve(self.h, rtol, maxit, restart, int(update), byref(it),
                                       byref(rel)))
        return it.value, rel.value

    def newton_step(self):
        r = c_double()
        self._check(self.lib.vms_newton_step(self.h, byref(r)))
        return r.value

    def newton_solve(self, rtol=1e-8, maxit=20):
        it = c_int()
        hist = np.zeros(maxit + 1)
        self._check(self.lib.vms_newton_solve(self.h, rtol, maxit, byref(it), hist.ctypes.data))
        return it.value, hist[: it.value + 1]

    def solver_stats(self, reset: bool = True):
        """(linear solves, Krylov iterations) since the last reset."""
        a, b = c_int64(), c_int64()
        self._check(self.lib.vms_solver_stats(self.h, int(reset), byref(a), byref(b)))
        return a.value, b.value

    # -- transient driver -------------------------------------------------------------------
    def node_features(self, X, scale_in=None):
        """X: device float32 tensor (n_nodes, 12) receiving [u, d, 1-ring mean of d] / scale with
        d = u - u_prev."""
        sc = None if scale_in is None else np.ascontiguousarray(scale_in, dtype=np.float32)
        self._check(self.lib.vms_node_features(self.h, None if sc is None else sc.ctypes.data,
                                               _ptr(X, np.float32, self.n_nodes * MLP_IN)))

    def node_increment(self, D, scale_out=None):
        sc = None if scale_out is None else np.ascontiguousarray(scale_out, dtype=np.float32)
        self._check(self.lib.vms_node_increment(self.h, None if sc is None else sc.ctypes.data,
                                                _ptr(D, np.float32, self.n_nodes * MLP_OUT)))

    def apply_increment(self, D, scale_out=None):
        sc = None if scale_out is None else np.ascontiguousarray(scale_out, dtype=np.float32)
        self._check(self.lib.vms_apply_increment(self.h, None if sc is None else sc.ctypes.data,
                                                 _ptr(D, np.float32, self.n_nodes * MLP_OUT)))

    def shift_time(self):
        self._check(self.lib.vms_shift_time(self.h))

    def newton_solve_to(self, target, maxit=20):
        it = c_int()
        hist = np.zeros(maxit + 1)
        self._check(self.lib.vms_newton_solve_to(self.h, target, maxit, byref(it), hist.ctypes.data))
        return it.value, hist[: it.value + 1]

    # -- kernel accounting ----------------------------------------------------------------
    def profile_enable(self, timing: bool = True):
        self._check(self.lib.vms_profile_enable(self.h, int(timing)))

    def profile_read(self, reset: bool = True):
        """{kind: (milliseconds, launches)} accumulated since the last reset."""
        ms = np.zeros(len(K_NAMES))
        n = np.zeros(len(K_NAMES), np.int64)
        self._check(self.lib.vms_profile_read(self.h, int(reset), ms.ctypes.data, n.ctypes.data))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(K_NAMES)}


class Mlp:
    """The warm-start network (VMS_MLP_*): BF16 weights, FP32 activations, own kernels."""

    def __init__(self, device: int = 0):
        self.lib = load_library()
        h = c_void_p()
        rc = self.lib.vms_mlp_create(byref(h), device)
        if rc != OK:
            raise VmsError(rc, "vms_mlp_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.vms_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            raise VmsError(rc, self.lib.vms_mlp_last_error(self.h).decode())
        return rc

    def set_stream(self, stream_handle: int):
        self._check(self.lib.vms_mlp_set_stream(self.h, c_void_p(stream_handle)))

    def set_params(self, params):
        a = np.ascontiguousarray(params, dtype=np.float32)
        if a.size != MLP_PARAMS:
            raise ValueError(f"expected {MLP_PARAMS} parameters")
        self._check(self.lib.vms_mlp_set_params(self.h, a.ctypes.data))

    def get_params(self, stored: bool = True):
        out = np.empty(MLP_PARAMS, np.float32)
        self._check(self.lib.vms_mlp_get_params(self.h, out.ctypes.data, int(stored)))
        return out

    def forward(self, X, Y):
        n = int(X.shape[0])
        self._check(self.lib.vms_mlp_forward(self.h, n, _ptr(X, np.float32, n * MLP_IN),
                                             _ptr(Y, np.float32, n * MLP_OUT)))

    def grad(self, X, T, rows=None, n=None, want=True):
        """Loss and gradient over the rows (device int32 tensor) or the first n rows of X, T."""
        n = int(rows.shape[0]) if rows is not None else int(n if n is not None else X.shape[0])
        loss = c_double()
        g = np.empty(MLP_PARAMS, np.float32) if want else None
        self._check(self.lib.vms_mlp_grad(self.h, n, _ptr(rows, np.int32), _ptr(X, np.float32),
                                          _ptr(T, np.float32), byref(loss) if want else None,
                                          g.ctypes.data if want else None))
        return (loss.value, g) if want else None

    def adam(self, lr: float):
        self._check(self.lib.vms_mlp_adam(self.h, ctypes.c_float(lr)))

    def column_rms(self, X):
        """Per-column RMS of a device FP32 (n, cols) tensor (FP64 sums), as a numpy array."""
        n, cols = int(X.shape[0]), int(X.shape[1])
        out = np.empty(cols, np.float64)
        self._check(self.lib.vms_mlp_column_rms(self.h, n, cols, _ptr(X, np.float32, n * cols),
                                                out.ctypes.data))
        return out

    def scale_columns(self, X, mul, out):
        """out = X * mul column-wise (device FP32 (n, cols); out may be X)."""
        n, cols = int(X.shape[0]), int(X.shape[1])
        m = np.ascontiguousarray(mul, dtype=np.float32)
        if m.size != cols:
            raise ValueError("one multiplier per column")
        self._check(self.lib.vms_mlp_scale_columns(self.h, n, cols, _ptr(X, np.float32, n * cols),
                                                   m.ctypes.data, _ptr(out, np.float32, n * cols)))


def tet_rule(n: int):
    """The library's tetrahedral quadrature rule (host code): points (n^3, 3), weights (n^3)."""
    pts = np.empty((n ** 3, 3))
    wts = np.empty(n ** 3)
    rc = load_library().vms_tet_rule(n, pts.ctypes.data, wts.ctypes.data)
    if rc != OK:
        raise VmsError(rc, "vms_tet_rule failed")
    return pts, wts


def fma_throughput(device: int, kind: int) -> float:
    """Measured TFLOP/s of the GPU's FMA pipe: kind 0 FP64, 1 FP32, 2 packed FP32."""
    t = c_double()
    rc = load_library().vms_fma_throughput(int(device), int(kind), byref(t))
    if rc != OK:
        raise VmsError(rc, "vms_fma_throughput failed")
    return t.value


def version() -> str:
    return load_library().vms_version().decode()
