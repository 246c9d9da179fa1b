"""ctypes wrapper of the plain FP64 CPU oracle (``btdf_oracle.c``).

TEST INFRASTRUCTURE: imported only by the tests, the smoke check and the CPU
baseline leg of ``bench.py``.  The product path never imports this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "btdf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no GPU needed)."""
    src_m = os.path.getmtime(_SRC)
    hdr_m = os.path.getmtime(os.path.join(_HERE, "btdf_oracle.h"))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(src_m, hdr_m):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-fopenmp", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib: Optional[C.CDLL] = None


def lib() -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    L = C.CDLL(build())
    vp = C.c_void_p
    L.oracle_create.restype = vp
    L.oracle_create.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                                C.c_double, C.c_double, C.c_int, C.c_int]
    L.oracle_destroy.argtypes = [vp]
    L.oracle_init_fields.argtypes = [vp, _dp, _dp, _dp]
    L.oracle_get_pops.argtypes = [vp, _dp]
    L.oracle_set_pops.argtypes = [vp, _dp]
    L.oracle_apply_inlet.argtypes = [vp]
    L.oracle_set_boundary_velocity.argtypes = [vp, _dp, _dp]
    L.oracle_add_body.restype = C.c_int
    L.oracle_add_body.argtypes = [vp, C.c_int, _dp, _dp, _dp, _dp, C.c_double, C.c_double]
    L.oracle_set_marker_velocity.argtypes = [vp, C.c_int, _dp, _dp]
    L.oracle_step.argtypes = [vp, C.c_int64]
    L.oracle_step_count.restype = C.c_int64
    L.oracle_step_count.argtypes = [vp]
    L.oracle_moments.argtypes = [vp, _dp, _dp, _dp]
    L.oracle_force_field.argtypes = [vp, _dp, _dp]
    L.oracle_history.restype = C.c_int64
    L.oracle_history.argtypes = [vp, C.c_int, C.c_int64, C.c_int64, _dp, _dp]
    L.oracle_marker_diag.argtypes = [vp, C.c_int] + [vp] * 7
    L.oracle_body_drs.restype = C.c_double
    L.oracle_body_drs.argtypes = [vp, C.c_int]
    L.oracle_delta.restype = C.c_double
    L.oracle_delta.argtypes = [C.c_int, C.c_double]
    L.oracle_drs_paper.restype = C.c_double
    L.oracle_drs_paper.argtypes = [C.c_int]
    L.oracle_support_width.restype = C.c_int
    L.oracle_support_width.argtypes = [C.c_int]
    L.oracle_support.restype = C.c_int
    L.oracle_support.argtypes = [vp, C.c_double, C.c_double, _i64p, _dp]
    L.oracle_interp.argtypes = [vp, C.c_int, _dp, _dp, _dp, _dp]
    L.oracle_spread.argtypes = [vp, C.c_int, _dp, _dp, _dp, _dp]
    L.oracle_drs_local.restype = C.c_int
    L.oracle_drs_local.argtypes = [vp, C.c_int, _dp]
    L.oracle_feq.argtypes = [C.c_double, C.c_double, C.c_double, _dp]
    L.oracle_guo.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, _dp]
    L.oracle_set_threads.argtypes = [C.c_int]
    L.oracle_get_threads.restype = C.c_int
    _lib = L
    return L


def delta(kind: int, r: float) -> float:
    return lib().oracle_delta(kind, float(r))


def drs_paper(kind: int) -> float:
    return lib().oracle_drs_paper(kind)


def feq(rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.zeros(9)
    lib().oracle_feq(rho, ux, uy, out)
    return out


def guo(tau: float, ux: float, uy: float, fx: float, fy: float) -> np.ndarray:
    out = np.zeros(9)
    lib().oracle_guo(tau, ux, uy, fx, fy, out)
    return out


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return lib().oracle_get_threads()


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Sim:
    """One oracle lattice.  Fields are numpy arrays of shape (ny, nx)."""

    def __init__(self, nx, ny, tau, u_in=0.0, bc_x=0, bc_y=0, gx=0.0, gy=0.0,
                 delta=3, nf=1):
        self.nx, self.ny = int(nx), int(ny)
        self._p = lib().oracle_create(self.nx, self.ny, float(tau), float(u_in), int(bc_x),
                                      int(bc_y), float(gx), float(gy), int(delta), int(nf))
        if not self._p:
            raise ValueError("oracle_create rejected the configuration")
        self.nbodies = 0
        self._nmark = []

    @classmethod
    def from_case(cls, case, drs=None):
        s = cls(case.nx, case.ny, case.tau, case.u_in, case.bc_x, case.bc_y, case.gx, case.gy,
                case.delta, case.nf)
        rho, ux, uy = case.initial_fields()
        s.init_fields(rho, ux, uy)
        for b in case.bodies:
            s.add_body(b.X, b.Y, b.ds, b.Ubx, b.Uby, drs=case.drs if drs is None else drs)
        return s

    def __del__(self):
        p = getattr(self, "_p", None)
        if p:
            lib().oracle_destroy(p)
            self._p = None

    def init_fields(self, rho, ux, uy):
        lib().oracle_init_fields(self._p, _c(rho).ravel(), _c(ux).ravel(), _c(uy).ravel())

    def add_body(self, X, Y, ds, Ubx=None, Uby=None, drs=0.0):
        n = len(X)
        Ubx = np.zeros(n) if Ubx is None else Ubx
        Uby = np.zeros(n) if Uby is None else Uby
        b = lib().oracle_add_body(self._p, n, _c(X), _c(Y), _c(Ubx), _c(Uby), float(ds),
                                  float(drs or 0.0))
        self.nbodies += 1
        self._nmark.append(n)
        return b

    def set_marker_velocity(self, body, Ubx, Uby):
        lib().oracle_set_marker_velocity(self._p, body, _c(Ubx), _c(Uby))

    def step(self, n=1):
        lib().oracle_step(self._p, int(n))

    @property
    def steps(self):
        return lib().oracle_step_count(self._p)

    def moments(self):
        sh = (self.ny, self.nx)
        r, ux, uy = np.zeros(sh), np.zeros(sh), np.zeros(sh)
        lib().oracle_moments(self._p, r.ravel(), ux.ravel(), uy.ravel())
        return r, ux, uy

    def pops(self):
        out = np.zeros((self.ny, self.nx, 9))
        lib().oracle_get_pops(self._p, out.ravel())
        return out

    def set_pops(self, f):
        lib().oracle_set_pops(self._p, _c(f).ravel())

    def apply_inlet(self):
        lib().oracle_apply_inlet(self._p)

    def set_boundary_velocity(self, ubx, uby):
        lib().oracle_set_boundary_velocity(self._p, _c(ubx), _c(uby))

    def force_field(self):
        sh = (self.ny, self.nx)
        fx, fy = np.zeros(sh), np.zeros(sh)
        lib().oracle_force_field(self._p, fx.ravel(), fy.ravel())
        return fx, fy

    def history(self, body=0, first=0, n=None):
        n = self.steps - first if n is None else n
        Fx, Fy = np.zeros(n), np.zeros(n)
        c = lib().oracle_history(self._p, body, first, n, Fx, Fy)
        return Fx[:c], Fy[:c]

    def marker_diag(self, body=0):
        n = self._nmark[body]
        arrs = [np.zeros(n) for _ in range(7)]
        lib().oracle_marker_diag(self._p, body, *[a.ctypes.data for a in arrs])
        keys = ["Usx", "Usy", "Fbx", "Fby", "Ux", "Uy", "rho"]
        return dict(zip(keys, arrs))

    def body_drs(self, body=0):
        return lib().oracle_body_drs(self._p, body)

    def support(self, X, Y):
        nodes = np.zeros(16, dtype=np.int64)
        w = np.zeros(16)
        c = lib().oracle_support(self._p, float(X), float(Y), nodes, w)
        return nodes[:c], w[:c]

    def interp(self, body, fx, fy):
        n = self._nmark[body]
        Ux, Uy = np.zeros(n), np.zeros(n)
        lib().oracle_interp(self._p, body, _c(fx).ravel(), _c(fy).ravel(), Ux, Uy)
        return Ux, Uy

    def spread(self, body, Fx, Fy):
        fx = np.zeros(self.nx * self.ny)
        fy = np.zeros(self.nx * self.ny)
        lib().oracle_spread(self._p, body, _c(Fx), _c(Fy), fx, fy)
        return fx.reshape(self.ny, self.nx), fy.reshape(self.ny, self.nx)

    def drs_local(self, body=0):
        out = np.zeros(self._nmark[body])
        if lib().oracle_drs_local(self._p, body, out) != 0:
            raise ValueError("singular thickness matrix")
        return out
