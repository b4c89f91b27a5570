"""Thin ctypes binding of libidugks (include/idugks.h): same names, argument
marshalling only.  Every step of the scheme runs in the CUDA library; there is
no Python or CPU fallback.  Importing this module fails loudly when the library
has not been built (run paper_1709_01819_gb300.build.build()).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB

IDG_OK, IDG_ERR_ARG, IDG_ERR_STATE, IDG_ERR_CUDA, IDG_ERR_OOM = 0, 1, 2, 3, 4
IDG_ERR_NONFINITE, IDG_ERR_TIMEOUT, IDG_ERR_NOT_CONVERGED = 5, 6, 7
IDG_FP64, IDG_MIXED = 0, 1
IDG_BC_PERIODIC, IDG_BC_WALL, IDG_BC_FARFIELD = 0, 1, 2
IDG_NC_TRAP, IDG_NC_SIMPSON, IDG_GAUSS_HERMITE = 0, 1, 2
IDG_IMIN, IDG_IMAX, IDG_JMIN, IDG_JMAX = 0, 1, 2, 3
IDG_BGK, IDG_SHAKHOV = 0, 1
IDG_TUNE_SWEEP_TV, IDG_TUNE_SWEEP_STAGES, IDG_TUNE_MACRO_STAGES, IDG_TUNE_GRAPH, IDG_TUNE_SWEEP_VPT = 1, 2, 3, 4, 5
IDG_TUNE_MACRO_KIND = 6
IDG_OBJ_FORCE_X, IDG_OBJ_FORCE_Y = 0, 1
IDG_PAR_KN, IDG_PAR_WALL_T, IDG_PAR_WALL_U, IDG_PAR_WALL_V = 0, 1, 2, 3
IDG_NUM_EXPLICIT = 1


def IDG_PARAM(kind: int, side_mask: int = 0) -> int:
    """Parameter id of idg_adjoint: a kind and, for wall parameters, a mask of sides."""
    return kind | (side_mask << 8)


_STATUS = {0: "IDG_OK", 1: "IDG_ERR_ARG", 2: "IDG_ERR_STATE", 3: "IDG_ERR_CUDA", 4: "IDG_ERR_OOM",
           5: "IDG_ERR_NONFINITE", 6: "IDG_ERR_TIMEOUT", 7: "IDG_ERR_NOT_CONVERGED"}

# (name, restype, argtypes)
_d, _i, _vp, _sz = C.c_double, C.c_int, C.c_void_p, C.c_size_t
_P = C.POINTER
SIGNATURES = [
    ("idg_create", _i, [_P(_vp), _i, _i]),
    ("idg_destroy", None, [_vp]),
    ("idg_last_error", C.c_char_p, [_vp]),
    ("idg_set_mesh_structured", _i, [_vp, _i, _i, _P(_d), _P(_d)]),
    ("idg_set_velocity_grid", _i, [_vp, _i, _i, _i, _d, _d, _d, _d]),
    ("idg_set_gas", _i, [_vp, _i, _d, _d, _d, _d, _i]),
    ("idg_set_boundary", _i, [_vp, _i, _i, _d, _d, _d, _d]),
    ("idg_set_numerics", _i, [_vp, _d, _d, _i, _d, _i]),
    ("idg_set_predictor", _i, [_vp, _i]),
    ("idg_set_implicit_wall", _i, [_vp, _i]),
    ("idg_save", _i, [_vp, C.c_char_p, _vp]),
    ("idg_load", _i, [_vp, C.c_char_p, _vp]),
    ("idg_set_mesh_unstructured", _i, [_vp, _i, _P(_d), _P(_d), _i, _P(_i), _P(_i)]),
    ("idg_workspace_size", _i, [_vp, _P(_sz)]),
    ("idg_bind_workspace", _i, [_vp, _vp, _sz]),
    ("idg_init_uniform", _i, [_vp, _d, _d, _d, _d, _vp]),
    ("idg_set_state", _i, [_vp, _P(_d), _P(_d), _P(_d), _vp]),
    ("idg_get_state", _i, [_vp, _P(_d), _P(_d), _P(_d), _vp]),
    ("idg_iterate", _i, [_vp, _i, _d, _vp, _P(_i), _P(_d)]),
    ("idg_iterate_profiled", _i, [_vp, _vp, _P(_d)]),
    ("idg_set_tuning", _i, [_vp, _i, _i]),
    ("idg_get_tuning", _i, [_vp, _i, _P(_i)]),
    ("idg_get_moments", _i, [_vp, _P(_d), _vp]),
    ("idg_get_moments_noalloc", _i, [_vp, _vp, _vp]),
    ("idg_get_residual_history", _i, [_vp, _P(_d), _i, _P(_i)]),
    ("idg_get_face_flux_moments", _i, [_vp, _P(_d), _vp]),
    ("idg_get_sizes", _i, [_vp, _P(_i), _P(_i), _P(_i)]),
    ("idg_get_dt", _i, [_vp, _P(_d)]),
    ("idg_velocity_grid", _i, [_vp, _P(_d), _P(_d), _P(_d)]),
    ("idg_batch_create", _i, [_P(_vp), _P(_vp), _i]),
    ("idg_batch_destroy", None, [_vp]),
    ("idg_batch_last_error", C.c_char_p, [_vp]),
    ("idg_batch_workspace_size", _i, [_vp, _P(_sz)]),
    ("idg_batch_bind_workspace", _i, [_vp, _vp, _sz]),
    ("idg_batch_iterate", _i, [_vp, _i, _d, _vp, _P(_i), _P(_d), _P(_i)]),
    ("idg_get_wall_force", _i, [_vp, _i, _P(_d), _vp]),
    ("idg_get_wall", _i, [_vp, _i, _P(_d), _i, _P(_i), _vp]),
    ("idg_adjoint_workspace_size", _i, [_vp, _P(_sz)]),
    ("idg_set_adjoint_solver", _i, [_vp, _i, _i]),
    ("idg_set_adjoint_limiter", _i, [_vp, _i]),
    ("idg_set_limiter_smoothing", _i, [_vp, _d]),
    ("idg_adjoint_state", _i, [_vp, _vp, _i, _P(_d), _P(_d), _P(_d), _vp]),
    ("idg_adjoint", _i, [_vp, _i, _i, _P(_i), _i, _vp, _sz, _i, _d, _vp, _P(_d), _P(_d), _P(_i), _P(_d)]),
]

_lib = None


def lib():
    """Load libidugks.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(f"libidugks.so not built at {LIB}; call paper_1709_01819_gb300.build.build()")
        L = C.CDLL(LIB)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class IdgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def check(ctx, status: int, allow=()):
    if status != IDG_OK and status not in allow:
        msg = lib().idg_last_error(ctx)
        raise IdgError(status, msg.decode() if msg else "")
    return status


# ---- one Python function per C entry point (argument marshalling only) ----

def idg_create(precision: int, device: int):
    h = C.c_void_p()
    check(None, lib().idg_create(C.byref(h), precision, device))
    return h


def idg_destroy(ctx):
    lib().idg_destroy(ctx)


def idg_last_error(ctx) -> str:
    m = lib().idg_last_error(ctx)
    return m.decode() if m else ""


def idg_set_mesh_structured(ctx, nodes_x: np.ndarray, nodes_y: np.ndarray):
    X = np.ascontiguousarray(nodes_x, dtype=np.float64)
    Y = np.ascontiguousarray(nodes_y, dtype=np.float64)
    nj, ni = X.shape[0] - 1, X.shape[1] - 1
    return check(ctx, lib().idg_set_mesh_structured(ctx, ni, nj, dptr(X), dptr(Y)))


def idg_set_velocity_grid(ctx, rule, nx, ny, xmin, xmax, ymin, ymax):
    return check(ctx, lib().idg_set_velocity_grid(ctx, rule, nx, ny, xmin, xmax, ymin, ymax))


def idg_set_gas(ctx, K, Pr, omega, Kn, RT_ref, model):
    return check(ctx, lib().idg_set_gas(ctx, K, Pr, omega, Kn, RT_ref, model))


def idg_set_boundary(ctx, side, kind, rho, u, v, T):
    return check(ctx, lib().idg_set_boundary(ctx, side, kind, rho, u, v, T))


def idg_set_numerics(ctx, cfl_imp, cfl_phys, limiter, lusgs_omega, flags=0):
    return check(ctx, lib().idg_set_numerics(ctx, cfl_imp, cfl_phys, limiter, lusgs_omega, flags))


def idg_set_predictor(ctx, relax_sweeps):
    return check(ctx, lib().idg_set_predictor(ctx, relax_sweeps))


def idg_set_implicit_wall(ctx, on):
    return check(ctx, lib().idg_set_implicit_wall(ctx, on))


def idg_save(ctx, path, stream=None):
    return check(ctx, lib().idg_save(ctx, str(path).encode(), stream))


def idg_load(ctx, path, stream=None):
    return check(ctx, lib().idg_load(ctx, str(path).encode(), stream))


def idg_set_mesh_unstructured(ctx, x, y, cell_nodes, edge_side):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    cn = np.ascontiguousarray(cell_nodes, dtype=np.int32)
    es = np.ascontiguousarray(edge_side, dtype=np.int32)
    return check(ctx, lib().idg_set_mesh_unstructured(
        ctx, len(x), x.ctypes.data_as(C.POINTER(C.c_double)), y.ctypes.data_as(C.POINTER(C.c_double)),
        len(cn), cn.ctypes.data_as(C.POINTER(C.c_int)), es.ctypes.data_as(C.POINTER(C.c_int))))


def idg_workspace_size(ctx) -> int:
    n = C.c_size_t()
    check(ctx, lib().idg_workspace_size(ctx, C.byref(n)))
    return n.value


def idg_bind_workspace(ctx, dev_ptr: int, nbytes: int):
    return check(ctx, lib().idg_bind_workspace(ctx, C.c_void_p(dev_ptr), nbytes))


def idg_init_uniform(ctx, rho, u, v, T, stream=None):
    return check(ctx, lib().idg_init_uniform(ctx, rho, u, v, T, stream))


def idg_set_state(ctx, G, H, W, stream=None):
    G = np.ascontiguousarray(G, dtype=np.float64)
    H = np.ascontiguousarray(H, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    return check(ctx, lib().idg_set_state(ctx, dptr(G), dptr(H), dptr(W), stream))


def idg_get_state(ctx, N, Nv, stream=None):
    G = np.zeros((N, Nv))
    H = np.zeros((N, Nv))
    W = np.zeros((N, 4))
    check(ctx, lib().idg_get_state(ctx, dptr(G), dptr(H), dptr(W), stream))
    return G, H, W


def idg_iterate(ctx, max_iter, tol, stream=None):
    n = C.c_int()
    r = C.c_double()
    st = check(ctx, lib().idg_iterate(ctx, max_iter, tol, stream, C.byref(n), C.byref(r)),
               allow=(IDG_ERR_NOT_CONVERGED,))
    return st, n.value, r.value


def idg_iterate_profiled(ctx, stream=None):
    ms = np.zeros(6)
    check(ctx, lib().idg_iterate_profiled(ctx, stream, dptr(ms)))
    return ms


def idg_set_tuning(ctx, key, value):
    return check(ctx, lib().idg_set_tuning(ctx, key, value))


def idg_get_tuning(ctx, key):
    v = C.c_int()
    check(ctx, lib().idg_get_tuning(ctx, key, C.byref(v)))
    return v.value


def idg_get_moments(ctx, N, stream=None):
    out = np.zeros((N, 6))
    check(ctx, lib().idg_get_moments(ctx, dptr(out), stream))
    return out


def idg_get_moments_noalloc(ctx, out6_dev_ptr: int, stream=None):
    return check(ctx, lib().idg_get_moments_noalloc(ctx, C.c_void_p(out6_dev_ptr), stream))


def idg_get_residual_history(ctx, cap):
    out = np.zeros(max(cap, 1))
    n = C.c_int()
    check(ctx, lib().idg_get_residual_history(ctx, dptr(out), cap, C.byref(n)))
    return out[: n.value]


def idg_get_face_flux_moments(ctx, nf, stream=None):
    out = np.zeros((nf, 4))
    check(ctx, lib().idg_get_face_flux_moments(ctx, dptr(out), stream))
    return out


def idg_get_wall_force(ctx, side_mask, stream=None):
    out = np.zeros(2)
    check(ctx, lib().idg_get_wall_force(ctx, side_mask, dptr(out), stream))
    return out


def idg_get_wall(ctx, side, stream=None):
    """Per face of wall side `side`: x, y (midpoint), p, tau_w, q_n ([nface][5])."""
    n = C.c_int()
    check(ctx, lib().idg_get_wall(ctx, side, None, 0, C.byref(n), stream))
    out = np.zeros((max(n.value, 1), 5))
    check(ctx, lib().idg_get_wall(ctx, side, dptr(out), n.value, C.byref(n), stream))
    return out[: n.value]


IDG_ADJ_FIXED_POINT, IDG_ADJ_GMRES = 0, 1


def idg_set_adjoint_solver(ctx, method, restart=20):
    return check(ctx, lib().idg_set_adjoint_solver(ctx, method, restart))


def idg_set_limiter_smoothing(ctx, K):
    return check(ctx, lib().idg_set_limiter_smoothing(ctx, float(K)))


IDG_ADJ_LIMITER_EXACT, IDG_ADJ_LIMITER_FROZEN = 0, 1


def idg_set_adjoint_limiter(ctx, mode):
    return check(ctx, lib().idg_set_adjoint_limiter(ctx, mode))


def idg_adjoint_workspace_size(ctx) -> int:
    n = C.c_size_t()
    check(ctx, lib().idg_adjoint_workspace_size(ctx, C.byref(n)))
    return n.value


def idg_adjoint(ctx, objective, side_mask, params, ws_ptr: int, ws_bytes: int, max_iter, tol, stream=None):
    """Returns (status, J, grad[len(params)], iterations, relative update)."""
    p = np.ascontiguousarray(params, dtype=np.int32)
    g = np.zeros(max(len(p), 1))
    J, r, n = C.c_double(), C.c_double(), C.c_int()
    st = check(ctx, lib().idg_adjoint(ctx, objective, side_mask, p.ctypes.data_as(_P(_i)), len(p),
                                      C.c_void_p(ws_ptr), ws_bytes, max_iter, tol, stream, C.byref(J),
                                      dptr(g), C.byref(n), C.byref(r)),
               allow=(IDG_ERR_NOT_CONVERGED,))
    return st, J.value, g[: len(p)], n.value, r.value


def idg_adjoint_state(ctx, ws_ptr: int, which, N, Nv, stream=None):
    G = np.zeros((N, Nv))
    H = np.zeros((N, Nv))
    W = np.zeros((N, 4))
    check(ctx, lib().idg_adjoint_state(ctx, C.c_void_p(ws_ptr), which, dptr(G), dptr(H), dptr(W), stream))
    return G, H, W


def idg_get_sizes(ctx):
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    check(ctx, lib().idg_get_sizes(ctx, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def idg_get_dt(ctx) -> float:
    d = C.c_double()
    check(ctx, lib().idg_get_dt(ctx, C.byref(d)))
    return d.value


def idg_velocity_grid(ctx, Nv):
    ux, uy, w = np.zeros(Nv), np.zeros(Nv), np.zeros(Nv)
    check(ctx, lib().idg_velocity_grid(ctx, dptr(ux), dptr(uy), dptr(w)))
    return ux, uy, w


# ---- batches ----

def _bcheck(b, status: int, allow=()):
    if status != IDG_OK and status not in allow:
        msg = lib().idg_batch_last_error(b)
        raise IdgError(status, msg.decode() if msg else "")
    return status


def idg_batch_create(ctxs):
    arr = (C.c_void_p * len(ctxs))(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    h = C.c_void_p()
    _bcheck(None, lib().idg_batch_create(C.byref(h), arr, len(ctxs)))
    return h


def idg_batch_destroy(b):
    lib().idg_batch_destroy(b)


def idg_batch_last_error(b) -> str:
    m = lib().idg_batch_last_error(b)
    return m.decode() if m else ""


def idg_batch_workspace_size(b) -> int:
    n = C.c_size_t()
    _bcheck(b, lib().idg_batch_workspace_size(b, C.byref(n)))
    return n.value


def idg_batch_bind_workspace(b, dev_ptr: int, nbytes: int):
    return _bcheck(b, lib().idg_batch_bind_workspace(b, C.c_void_p(dev_ptr), nbytes))


def idg_batch_iterate(b, n_inst, max_iter, tol, stream=None):
    it = C.c_int()
    r = C.c_double()
    conv = (C.c_int * n_inst)()
    st = _bcheck(b, lib().idg_batch_iterate(b, max_iter, tol, stream, C.byref(it), C.byref(r), conv),
                 allow=(IDG_ERR_NOT_CONVERGED,))
    return st, it.value, r.value, [bool(x) for x in conv]
