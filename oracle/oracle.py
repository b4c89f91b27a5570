"""ctypes wrapper of the FP64 CPU oracle (idugks_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the CPU baseline leg of bench.py.  The product path never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "idugks_oracle.c")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP; no architecture-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "idugks_oracle.h"))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [
        ("ni", C.c_int), ("nj", C.c_int),
        ("nodes_x", C.POINTER(C.c_double)), ("nodes_y", C.POINTER(C.c_double)),
        ("bc_kind", C.c_int * 4),
        ("bc_rho", C.c_double * 4), ("bc_u", C.c_double * 4), ("bc_v", C.c_double * 4),
        ("bc_T", C.c_double * 4),
        ("vrule", C.c_int), ("nvx", C.c_int), ("nvy", C.c_int),
        ("vxmin", C.c_double), ("vxmax", C.c_double), ("vymin", C.c_double), ("vymax", C.c_double),
        ("K", C.c_int),
        ("Pr", C.c_double), ("omega", C.c_double), ("Kn", C.c_double), ("RT_ref", C.c_double),
        ("shakhov", C.c_int),
        ("cfl_imp", C.c_double), ("cfl_phys", C.c_double),
        ("limiter", C.c_int), ("flags", C.c_int),
        ("lusgs_omega", C.c_double),
        ("relax_sweeps", C.c_int),
        ("n_ucells", C.c_int), ("n_unodes", C.c_int),
        ("ucell_nodes", C.POINTER(C.c_int)), ("uedge_side", C.POINTER(C.c_int)),
        ("implicit_wall", C.c_int),
        ("venkat_k", C.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i, vp = C.c_double, C.c_int, C.c_void_p
        P = C.POINTER
        _lib.orc_create.restype = vp
        _lib.orc_create.argtypes = [P(_Problem)]
        _lib.orc_destroy.argtypes = [vp]
        for n in ("orc_num_cells", "orc_num_vel", "orc_num_faces"):
            getattr(_lib, n).restype = i
            getattr(_lib, n).argtypes = [vp]
        _lib.orc_dt.restype = d
        _lib.orc_dt.argtypes = [vp]
        _lib.orc_init_uniform.argtypes = [vp, d, d, d, d]
        _lib.orc_set_state.argtypes = [vp, P(d), P(d), P(d)]
        _lib.orc_get_state.argtypes = [vp, P(d), P(d), P(d)]
        _lib.orc_iterate.argtypes = [vp, i, P(d)]
        _lib.orc_explicit_step.argtypes = [vp, i]
        _lib.orc_get_moments.argtypes = [vp, P(d)]
        _lib.orc_get_face_phi.argtypes = [vp, P(d)]
        _lib.orc_get_rw.argtypes = [vp, P(d)]
        _lib.orc_get_faces.argtypes = [vp, P(i), P(i), P(i), P(i), P(d), P(d), P(d)]
        _lib.orc_get_geometry.argtypes = [vp, P(d), P(d), P(d)]
        _lib.orc_quadrature.restype = i
        _lib.orc_quadrature.argtypes = [i, i, d, d, P(d), P(d)]
        _lib.orc_velocity_grid.argtypes = [vp, P(d), P(d), P(d)]
        _lib.orc_equilibrium.argtypes = [vp, d, d, d, d, d, d, P(d), P(d)]
        _lib.orc_ls_gradient.argtypes = [vp, P(d), P(d)]
        _lib.orc_limiter.argtypes = [vp, P(d), P(d)]
        _lib.orc_venkat_theta.restype = d
        _lib.orc_venkat_theta.argtypes = [d]
        _lib.orc_debug_cell_prep.argtypes = [vp, P(d), P(d), P(d), P(d)]
        _lib.orc_debug_predictor.argtypes = [vp, P(d), P(d)]
        _lib.orc_debug_micro_residual.argtypes = [vp, P(d), P(d)]
        _lib.orc_debug_micro_sweeps.argtypes = [vp, P(d), P(d), P(d), P(d), P(d)]
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def quadrature(rule: int, n: int, a: float, b: float):
    x = np.zeros(n)
    w = np.zeros(n)
    rc = lib().orc_quadrature(rule, n, a, b, _dp(x), _dp(w))
    if rc != 0:
        raise ValueError(f"oracle quadrature rule {rule} n={n} failed ({rc})")
    return x, w


def venkat_theta(x: float) -> float:
    return lib().orc_venkat_theta(float(x))


class Oracle:
    """One problem instance in the FP64 oracle."""

    def __init__(self, prob):
        L = lib()
        self.prob = prob
        self._nx = np.ascontiguousarray(prob.nodes_x, dtype=np.float64)
        self._ny = np.ascontiguousarray(prob.nodes_y, dtype=np.float64)
        p = _Problem()
        p.ni, p.nj = prob.ni, prob.nj
        p.nodes_x, p.nodes_y = _dp(self._nx), _dp(self._ny)
        for s in range(4):
            kind, rho, u, v, T = prob.bc[s]
            p.bc_kind[s] = kind
            p.bc_rho[s], p.bc_u[s], p.bc_v[s], p.bc_T[s] = rho, u, v, T
        p.vrule, p.nvx, p.nvy = prob.vrule, prob.nvx, prob.nvy
        p.vxmin, p.vxmax, p.vymin, p.vymax = prob.vrange
        p.K, p.Pr, p.omega, p.Kn, p.RT_ref = prob.K, prob.Pr, prob.omega, prob.Kn, prob.RT_ref
        p.shakhov = prob.shakhov
        p.cfl_imp, p.cfl_phys = prob.cfl_imp, prob.cfl_phys
        p.limiter, p.flags, p.lusgs_omega = prob.limiter, prob.flags, prob.lusgs_omega
        p.relax_sweeps = prob.relax_sweeps
        p.implicit_wall = int(getattr(prob, "implicit_wall", 0))
        p.venkat_k = float(getattr(prob, "venkat_k", 0.0))
        if getattr(prob, "cell_nodes", None) is not None:
            self._cn = np.ascontiguousarray(prob.cell_nodes, dtype=np.int32)
            self._es = np.ascontiguousarray(prob.edge_side, dtype=np.int32)
            p.n_ucells, p.n_unodes = len(self._cn), len(self._nx)
            p.ucell_nodes, p.uedge_side = _ip(self._cn), _ip(self._es)
        self._p = p
        self._h = L.orc_create(C.byref(p))
        if not self._h:
            raise ValueError("oracle rejected the problem")
        self.N = L.orc_num_cells(self._h)
        self.Nv = L.orc_num_vel(self._h)
        self.nf = L.orc_num_faces(self._h)
        self.dt = L.orc_dt(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def init_uniform(self, rho=None, u=None, v=None, T=None):
        r0, u0, v0, T0 = self.prob.init
        lib().orc_init_uniform(self._h, r0 if rho is None else rho, u0 if u is None else u,
                               v0 if v is None else v, T0 if T is None else T)

    def set_state(self, G, H, W):
        G = np.ascontiguousarray(G, dtype=np.float64)
        H = np.ascontiguousarray(H, dtype=np.float64)
        W = np.ascontiguousarray(W, dtype=np.float64)
        assert G.size == self.N * self.Nv and W.size == 4 * self.N
        lib().orc_set_state(self._h, _dp(G), _dp(H), _dp(W))

    def get_state(self):
        G = np.zeros((self.N, self.Nv))
        H = np.zeros((self.N, self.Nv))
        W = np.zeros((self.N, 4))
        lib().orc_get_state(self._h, _dp(G), _dp(H), _dp(W))
        return G, H, W

    def iterate(self, n: int) -> np.ndarray:
        res = np.zeros(max(n, 1))
        lib().orc_iterate(self._h, n, _dp(res))
        return res[:n]

    def explicit(self, n: int):
        lib().orc_explicit_step(self._h, n)

    def predictor(self):
        """(R_W, dW) of the current state: the macroscopic residual and the
        predictor's increment (the state is not advanced)."""
        rw, dW = np.zeros((self.N, 4)), np.zeros((self.N, 4))
        lib().orc_debug_predictor(self._h, _dp(rw), _dp(dW))
        return rw, dW

    def micro_residual(self):
        """(R_G, R_H) [N][Nv]: the right-hand side of the micro sweeps of the
        current state (with the wall ghost term under implicit_wall); the
        state is not advanced."""
        RG, RH = np.zeros((self.N, self.Nv)), np.zeros((self.N, self.Nv))
        lib().orc_debug_micro_residual(self._h, _dp(RG), _dp(RH))
        return RG, RH

    def debug_micro_sweeps(self, RG: np.ndarray, RH: np.ndarray):
        """The micro LU-SGS sweeps of the current state's iteration applied to
        the right-hand side (RG, RH) [N][Nv]: (dG, dH, D); the state is not
        advanced."""
        RG = np.ascontiguousarray(RG, dtype=np.float64)
        RH = np.ascontiguousarray(RH, dtype=np.float64)
        dG, dH, D = (np.zeros((self.N, self.Nv)) for _ in range(3))
        lib().orc_debug_micro_sweeps(self._h, _dp(RG), _dp(RH), _dp(dG), _dp(dH), _dp(D))
        return dG, dH, D

    def moments(self) -> np.ndarray:
        out = np.zeros((self.N, 6))
        lib().orc_get_moments(self._h, _dp(out))
        return out

    def face_phi(self) -> np.ndarray:
        out = np.zeros((self.nf, 4))
        lib().orc_get_face_phi(self._h, _dp(out))
        return out

    def rw(self) -> np.ndarray:
        out = np.zeros((self.N, 4))
        lib().orc_get_rw(self._h, _dp(out))
        return out

    def faces(self):
        n = self.nf
        L, R, bc, side = (np.zeros(n, dtype=np.int32) for _ in range(4))
        nx, ny, S = (np.zeros(n) for _ in range(3))
        lib().orc_get_faces(self._h, _ip(L), _ip(R), _ip(bc), _ip(side), _dp(nx), _dp(ny), _dp(S))
        return dict(L=L, R=R, bc=bc, side=side, nx=nx, ny=ny, S=S)

    def geometry(self):
        cx, cy, a = np.zeros(self.N), np.zeros(self.N), np.zeros(self.N)
        lib().orc_get_geometry(self._h, _dp(cx), _dp(cy), _dp(a))
        return cx, cy, a

    def velocity_grid(self):
        ux, uy, w = np.zeros(self.Nv), np.zeros(self.Nv), np.zeros(self.Nv)
        lib().orc_velocity_grid(self._h, _dp(ux), _dp(uy), _dp(w))
        return ux, uy, w

    def equilibrium(self, rho, u, v, RT, qx=0.0, qy=0.0):
        G = np.zeros(self.Nv)
        H = np.zeros(self.Nv)
        lib().orc_equilibrium(self._h, rho, u, v, RT, qx, qy, _dp(G), _dp(H))
        return G, H

    def cell_prep(self):
        fbG = np.zeros((self.N, self.Nv))
        fbH = np.zeros((self.N, self.Nv))
        q = np.zeros((self.N, 2))
        tau = np.zeros(self.N)
        lib().orc_debug_cell_prep(self._h, _dp(fbG), _dp(fbH), _dp(q), _dp(tau))
        return fbG, fbH, q, tau

    def limiter(self, phi: np.ndarray) -> np.ndarray:
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        out = np.zeros(self.N)
        lib().orc_limiter(self._h, _dp(phi), _dp(out))
        return out

    def ls_gradient(self, phi: np.ndarray) -> np.ndarray:
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        out = np.zeros((self.N, 2))
        lib().orc_ls_gradient(self._h, _dp(phi), _dp(out))
        return out
