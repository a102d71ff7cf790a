"""ctypes binding of libflexi_gb300.so (argument marshalling only).

The functions here carry the C names of include/flexi.h.  Device buffers are
passed as raw pointers of torch CUDA tensors; streams are torch CUDA streams.
There is no CPU fallback: loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libflexi_gb300.so")

FLEXI_OK, FLEXI_EINVAL, FLEXI_ENOMEM, FLEXI_ECUDA, FLEXI_EMESH, FLEXI_ENONPHYSICAL, FLEXI_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
NODES_GAUSS, NODES_LOBATTO = 0, 1
RIEMANN_ROE, RIEMANN_HLLC, RIEMANN_ROE_SMOOTH, RIEMANN_RUSANOV, RIEMANN_EC = 0, 1, 2, 3, 4
FP64, FP32, FP32_TF32, FP32_BF16 = 0, 1, 2, 3
EXACT_TGV, EXACT_FREESTREAM, EXACT_MANUFACTURED = 0, 1, 2
SPLIT_STANDARD, SPLIT_KEP, SPLIT_EC = 0, 1, 2
CONN_MORTAR = -(1 << 30)
BC_EXACT, BC_OUTFLOW, BC_SLIP_WALL = 0, 1, 2
LIFTING_BR1, LIFTING_BR2 = 0, 1
Q_K, Q_N, Q_NSIDES, Q_NBCSIDES, Q_DOF, Q_BYTES_PER_STAGE, Q_FLOPS_PER_STAGE, Q_STATUS, Q_DEVICE_BYTES, Q_PRECISION = range(10)
KERNEL_CLASSES = ["lift_vol", "face", "surf_rk", "prolong", "bc", "adjoint", "reduce", "other"]

# every entry point declared in include/flexi.h
EXPORTS = ["flexi_mesh_init", "flexi_mesh_init_mortar", "flexi_set_bc", "flexi_rhs", "flexi_rk_step", "flexi_rk_run", "flexi_rk_step_stages", "flexi_adjoint_step",
           "flexi_rhs_adjoint", "flexi_rk_run_host", "flexi_reduce", "flexi_reduce_noalloc", "flexi_query",
           "flexi_profile", "flexi_kernel_times", "flexi_strerror", "flexi_destroy"]
NOALLOC_MAX_ELEMENTS = 65536


class flexi_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("Ngeo", ctypes.c_int), ("node_type", ctypes.c_int), ("riemann", ctypes.c_int),
                ("precision", ctypes.c_int), ("bc_exact", ctypes.c_int), ("source", ctypes.c_int),
                ("split_form", ctypes.c_int), ("gamma", ctypes.c_double), ("Pr", ctypes.c_double),
                ("mu", ctypes.c_double), ("Ma", ctypes.c_double), ("adjoint", ctypes.c_int),
                ("lifting", ctypes.c_int), ("eta_br2", ctypes.c_double)]


class FlexiError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


_lib = None


def lib() -> ctypes.CDLL:
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1910_02858_gb300.build.build() "
                               "(the CUDA path has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, d, i, i64p = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)
        L.flexi_mesh_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(flexi_params), i, vp, vp, vp]
        L.flexi_mesh_init_mortar.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(flexi_params), i, vp, vp, i, vp, vp]
        L.flexi_set_bc.argtypes = [vp, i, i]
        L.flexi_rhs.argtypes = [vp, vp, vp, d, vp]
        L.flexi_rk_step.argtypes = [vp, vp, vp, d, d, vp]
        L.flexi_rk_run.argtypes = [vp, vp, vp, i, d, d, vp]
        L.flexi_rk_step_stages.argtypes = [vp, vp, vp, d, d, vp, vp]
        L.flexi_adjoint_step.argtypes = [vp, vp, vp, vp, d, d, vp]
        L.flexi_rhs_adjoint.argtypes = [vp, vp, vp, vp, d, vp]
        L.flexi_rk_run_host.argtypes = [vp, vp, i, d, d, vp]
        L.flexi_reduce.argtypes = [vp, vp, vp, d, ctypes.POINTER(ctypes.c_double), vp]
        L.flexi_reduce_noalloc.argtypes = [vp, vp, vp, d, ctypes.POINTER(ctypes.c_double), vp]
        L.flexi_query.argtypes = [vp, i, i64p]
        L.flexi_profile.argtypes = [vp, i]
        L.flexi_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), i64p, i]
        L.flexi_strerror.argtypes = [i]
        L.flexi_strerror.restype = ctypes.c_char_p
        L.flexi_destroy.argtypes = [vp]
        L.flexi_destroy.restype = None
        for name in EXPORTS:
            if name not in ("flexi_strerror", "flexi_destroy"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().flexi_strerror(code).decode()


def check(code: int, where: str) -> int:
    if code != FLEXI_OK:
        raise FlexiError(code, where)
    return code


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if stream is None else stream.cuda_stream)


def flexi_mesh_init(params: flexi_params, coords: np.ndarray, conn: np.ndarray, stream=None) -> ctypes.c_void_p:
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    ctx = ctypes.c_void_p()
    check(lib().flexi_mesh_init(ctypes.byref(ctx), ctypes.byref(params), int(coords.shape[0]),
                                coords.ctypes.data_as(ctypes.c_void_p), conn.ctypes.data_as(ctypes.c_void_p),
                                _stream(stream)), "flexi_mesh_init")
    return ctx


def flexi_mesh_init_mortar(params: flexi_params, coords: np.ndarray, conn: np.ndarray, mortars: np.ndarray,
                           stream=None) -> ctypes.c_void_p:
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    mortars = np.ascontiguousarray(mortars, dtype=np.int32).reshape(-1, 15)
    ctx = ctypes.c_void_p()
    check(lib().flexi_mesh_init_mortar(ctypes.byref(ctx), ctypes.byref(params), int(coords.shape[0]),
                                       coords.ctypes.data_as(ctypes.c_void_p), conn.ctypes.data_as(ctypes.c_void_p),
                                       int(mortars.shape[0]), mortars.ctypes.data_as(ctypes.c_void_p),
                                       _stream(stream)), "flexi_mesh_init_mortar")
    return ctx


def flexi_set_bc(ctx, bc_id: int, kind: int):
    return check(lib().flexi_set_bc(ctx, int(bc_id), int(kind)), "flexi_set_bc")


def flexi_rhs(ctx, U, Ut, t, stream=None):
    return check(lib().flexi_rhs(ctx, _ptr(U), _ptr(Ut), float(t), _stream(stream)), "flexi_rhs")


def flexi_rk_step(ctx, U, dU, t, dt, stream=None):
    return check(lib().flexi_rk_step(ctx, _ptr(U), _ptr(dU), float(t), float(dt), _stream(stream)), "flexi_rk_step")


def flexi_rk_run(ctx, U, dU, nsteps, t0, dt, stream=None):
    return check(lib().flexi_rk_run(ctx, _ptr(U), _ptr(dU), int(nsteps), float(t0), float(dt), _stream(stream)),
                 "flexi_rk_run")


def flexi_rk_step_stages(ctx, U, dU, t, dt, U_stages, stream=None):
    return check(lib().flexi_rk_step_stages(ctx, _ptr(U), _ptr(dU), float(t), float(dt), _ptr(U_stages),
                                            _stream(stream)), "flexi_rk_step_stages")


def flexi_adjoint_step(ctx, U_stages, lamU, lam_dU, t, dt, stream=None):
    return check(lib().flexi_adjoint_step(ctx, _ptr(U_stages), _ptr(lamU), _ptr(lam_dU), float(t), float(dt),
                                          _stream(stream)), "flexi_adjoint_step")


def flexi_rhs_adjoint(ctx, U, lam, out, t, stream=None):
    return check(lib().flexi_rhs_adjoint(ctx, _ptr(U), _ptr(lam), _ptr(out), float(t), _stream(stream)),
                 "flexi_rhs_adjoint")


def flexi_rk_run_host(ctx, U_host, nsteps, t0, dt, stream=None):
    """U_host: contiguous CPU torch tensor or numpy array, updated in place."""
    p = ctypes.c_void_p(U_host.data_ptr()) if hasattr(U_host, "data_ptr") else U_host.ctypes.data_as(ctypes.c_void_p)
    return check(lib().flexi_rk_run_host(ctx, p, int(nsteps), float(t0), float(dt), _stream(stream)),
                 "flexi_rk_run_host")


def flexi_reduce(ctx, U, Ut=None, cfl=0.9, stream=None, allow_nonphysical=False):
    out = (ctypes.c_double * 8)()
    code = lib().flexi_reduce(ctx, _ptr(U), _ptr(Ut), float(cfl), out, _stream(stream))
    if not (allow_nonphysical and code == FLEXI_ENONPHYSICAL):
        check(code, "flexi_reduce")
    return list(out), code


def flexi_reduce_noalloc(ctx, U, Ut=None, cfl=0.9, stream=None):
    """Same outputs as flexi_reduce, without any device allocation (returns the
    8 values and the status code, which is not raised)."""
    out = (ctypes.c_double * 8)()
    code = lib().flexi_reduce_noalloc(ctx, _ptr(U), _ptr(Ut), float(cfl), out, _stream(stream))
    return list(out), code


def flexi_query(ctx, what: int) -> int:
    v = ctypes.c_int64()
    check(lib().flexi_query(ctx, int(what), ctypes.byref(v)), "flexi_query")
    return v.value


def flexi_profile(ctx, enable: bool):
    return check(lib().flexi_profile(ctx, int(bool(enable))), "flexi_profile")


def flexi_kernel_times(ctx, reset: bool = True):
    ms = (ctypes.c_double * 8)()
    cnt = (ctypes.c_int64 * 8)()
    check(lib().flexi_kernel_times(ctx, ms, cnt, int(bool(reset))), "flexi_kernel_times")
    return {KERNEL_CLASSES[k]: (ms[k], cnt[k]) for k in range(8)}


def flexi_destroy(ctx):
    if ctx:
        lib().flexi_destroy(ctx)
