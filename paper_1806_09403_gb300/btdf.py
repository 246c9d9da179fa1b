"""Thin ctypes binding of the C ABI in ``include/btdf.h``.

Argument marshalling only: every step of the method runs in the CUDA library
``_lib/libbtdf.so``.  There is no CPU fallback: if the library is missing or
cannot be loaded, importing the binding raises.

The raw entry points keep their C names (``btdf_create``, ``btdf_step``, ...);
``Lattice`` wraps one context for numpy / torch callers.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Tuple

import numpy as np

from . import _build

BTDF_OK, BTDF_EINVAL, BTDF_ENOMEM, BTDF_ECUDA, BTDF_EUNSTABLE, BTDF_ETIMEOUT, BTDF_ESTATE = \
    0, -1, -2, -3, -4, -5, -6
BTDF_F32, BTDF_F16DEV, BTDF_BF16DEV = 0, 1, 2
BTDF_BCX_PERIODIC, BTDF_BCX_INOUT, BTDF_BCX_CONVECTIVE, BTDF_BCX_BOX = 0, 1, 2, 3
BTDF_BCY_PERIODIC, BTDF_BCY_FREESLIP, BTDF_BCY_NOSLIP = 0, 1, 2
FIELD_RHO, FIELD_UX, FIELD_UY, FIELD_POPS, FIELD_FX, FIELD_FY = 0, 1, 2, 3, 4, 5
LAYOUT_PLANES, LAYOUT_ROWS = 0, 1

# Every symbol include/btdf.h declares.
EXPORTS = [
    "btdf_config_default", "btdf_create", "btdf_destroy", "btdf_init_fields",
    "btdf_add_markers", "btdf_set_marker_velocity", "btdf_step", "btdf_sync",
    "btdf_read_forces", "btdf_read_markers", "btdf_read_field", "btdf_step_count",
    "btdf_state_size", "btdf_save_state", "btdf_load_state", "btdf_profile_enable",
    "btdf_profile_read", "btdf_tune", "btdf_device_bytes", "btdf_last_error", "btdf_status_string",
    "btdf_version", "btdf_ib_forces_static",
    "btdf_batch_create", "btdf_batch_destroy", "btdf_batch_init_fields", "btdf_batch_add_markers",
    "btdf_batch_body_count", "btdf_batch_body_lattice", "btdf_batch_tune", "btdf_batch_step",
    "btdf_batch_sync", "btdf_batch_step_count", "btdf_batch_read_forces", "btdf_batch_read_field",
    "btdf_batch_last_error", "btdf_set_inflow", "btdf_move_markers", "btdf_adjoint_forward",
    "btdf_adjoint_backward", "btdf_adjoint_release", "btdf_autotune", "btdf_batch_autotune",
    "btdf_read_forces_async", "btdf_add_cylinder", "btdf_set_boundary_velocity",
    "btdf_set_wait_limit",
]
STATIC_MAX_MARKERS = 2048
VARIANT_COUNT = 14          # BTDF_VARIANT_COUNT: variants 0 (automatic) .. 13, see btdf_tune
STATE_HEADER_BYTES = 48


class btdf_config(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32),
        ("tau", C.c_double), ("u_in", C.c_double),
        ("delta", C.c_int32), ("nf", C.c_int32), ("storage", C.c_int32),
        ("bc_x", C.c_int32), ("bc_y", C.c_int32), ("history_len", C.c_int32),
        ("gx", C.c_double), ("gy", C.c_double),
        ("layout", C.c_int32), ("reserved", C.c_int32),
    ]


class BtdfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def library_path() -> str:
    return _build.LIB


_lib: Optional[C.CDLL] = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def lib() -> C.CDLL:
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"libbtdf.so is not built ({path}); run __graft_entry__.build()")
    L = C.CDLL(path)
    vp = C.c_void_p
    ctxp = C.c_void_p
    L.btdf_config_default.argtypes = [C.POINTER(btdf_config)]
    L.btdf_create.argtypes = [C.POINTER(btdf_config), vp, C.POINTER(ctxp)]
    L.btdf_destroy.argtypes = [ctxp]
    L.btdf_init_fields.argtypes = [ctxp, _dp, _dp, _dp]
    L.btdf_add_markers.argtypes = [ctxp, C.c_int32, _dp, _dp, vp, vp, C.c_double, C.c_double,
                                   C.POINTER(C.c_int32)]
    L.btdf_set_marker_velocity.argtypes = [ctxp, C.c_int32, _dp, _dp]
    L.btdf_step.argtypes = [ctxp, C.c_int64]
    L.btdf_sync.argtypes = [ctxp]
    L.btdf_read_forces.argtypes = [ctxp, C.c_int32, C.c_int64, C.c_int64, vp, vp]
    L.btdf_read_markers.argtypes = [ctxp, C.c_int32, vp, vp, vp, vp]
    L.btdf_read_forces_async.argtypes = [ctxp, C.c_int32, C.c_int64, C.c_int64, vp]
    L.btdf_set_boundary_velocity.argtypes = [ctxp, _dp, _dp]
    L.btdf_add_cylinder.argtypes = [ctxp, C.c_double, C.c_double, C.c_double, C.c_int32, C.c_double,
                                    C.POINTER(C.c_int32)]
    L.btdf_read_field.argtypes = [ctxp, C.c_int32, vp, C.c_int32]
    L.btdf_step_count.argtypes = [ctxp]
    L.btdf_step_count.restype = C.c_int64
    L.btdf_state_size.argtypes = [ctxp, C.POINTER(C.c_size_t)]
    L.btdf_save_state.argtypes = [ctxp, vp, C.c_size_t, C.POINTER(C.c_size_t)]
    L.btdf_load_state.argtypes = [ctxp, vp, C.c_size_t]
    L.btdf_profile_enable.argtypes = [ctxp, C.c_int32]
    L.btdf_profile_read.argtypes = [ctxp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.btdf_tune.argtypes = [ctxp, C.c_int32, C.c_int32]
    L.btdf_device_bytes.argtypes = [ctxp, C.POINTER(C.c_size_t)]
    L.btdf_last_error.argtypes = [ctxp]
    L.btdf_last_error.restype = C.c_char_p
    L.btdf_status_string.argtypes = [C.c_int]
    L.btdf_status_string.restype = C.c_char_p
    L.btdf_version.restype = C.c_int
    L.btdf_ib_forces_static.argtypes = [C.POINTER(btdf_config), vp, C.c_int32, C.c_double,
                                        C.c_int32, _dp, _dp, vp, vp, C.c_double, C.c_double, vp,
                                        _dp, vp]
    L.btdf_batch_create.argtypes = [C.POINTER(btdf_config), C.c_int32, vp, C.POINTER(vp)]
    L.btdf_batch_destroy.argtypes = [vp]
    L.btdf_batch_init_fields.argtypes = [vp, C.c_int32, _dp, _dp, _dp]
    L.btdf_batch_add_markers.argtypes = [vp, C.c_int32, C.c_int32, _dp, _dp, vp, vp, C.c_double,
                                         C.c_double, C.POINTER(C.c_int32)]
    L.btdf_batch_body_count.argtypes = [vp, C.POINTER(C.c_int32)]
    L.btdf_batch_body_lattice.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32)]
    L.btdf_batch_tune.argtypes = [vp, C.c_int32]
    L.btdf_batch_step.argtypes = [vp, C.c_int64]
    L.btdf_batch_sync.argtypes = [vp]
    L.btdf_batch_step_count.argtypes = [vp]
    L.btdf_batch_step_count.restype = C.c_int64
    L.btdf_batch_read_forces.argtypes = [vp, C.c_int32, C.c_int64, C.c_int64, vp, vp]
    L.btdf_batch_read_field.argtypes = [vp, C.c_int32, C.c_int32, vp, C.c_int32]
    L.btdf_set_inflow.argtypes = [ctxp, C.c_double]
    L.btdf_set_wait_limit.argtypes = [ctxp, C.c_int32]
    L.btdf_move_markers.argtypes = [ctxp, C.c_int32, _dp, _dp]
    L.btdf_adjoint_forward.argtypes = [ctxp, C.c_int64, C.c_int32, C.c_int32, C.c_double,
                                       C.POINTER(C.c_double)]
    L.btdf_adjoint_backward.argtypes = [ctxp, C.POINTER(C.c_double), vp, vp]
    L.btdf_adjoint_release.argtypes = [ctxp]
    L.btdf_autotune.argtypes = [ctxp, C.c_int32, C.c_int32, C.POINTER(C.c_int32), vp]
    L.btdf_batch_autotune.argtypes = [vp, C.c_int32, C.c_int32, C.POINTER(C.c_int32), vp]
    L.btdf_batch_last_error.argtypes = [vp]
    L.btdf_batch_last_error.restype = C.c_char_p
    _lib = L
    return L


# ---- raw entry points with the C names -----------------------------------------

def btdf_config_default() -> btdf_config:
    cfg = btdf_config()
    lib().btdf_config_default(C.byref(cfg))
    return cfg


def btdf_create(cfg: btdf_config, stream: int = 0) -> Tuple[int, Optional[int]]:
    out = C.c_void_p()
    rc = lib().btdf_create(C.byref(cfg), C.c_void_p(stream or None), C.byref(out))
    return rc, out.value


def btdf_status_string(rc: int) -> str:
    return lib().btdf_status_string(rc).decode()


def btdf_version() -> int:
    return lib().btdf_version()


def btdf_ib_forces_static(cfg: btdf_config, pops_ptr: int, pull: bool, X, Y, ds, Ubx=None,
                          Uby=None, drs=0.0, fb_ptr: int = 0, stream: int = 0, u_ref=None):
    """IB force stage of one body on a caller-owned device population buffer,
    without any device allocation (see include/btdf.h).  u_ref is the
    reference velocity of the stored deviations (default: cfg.u_in).  Returns
    (status, (Fx, Fy)); F_b per marker is written to the device pointer fb_ptr."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    ubx = None if Ubx is None else np.ascontiguousarray(Ubx, dtype=np.float64)
    uby = None if Uby is None else np.ascontiguousarray(Uby, dtype=np.float64)
    Fp = np.zeros(2)
    ur = float(cfg.u_in if u_ref is None else u_ref)
    rc = lib().btdf_ib_forces_static(C.byref(cfg), C.c_void_p(pops_ptr), 1 if pull else 0, ur,
                                     len(X), X, Y, None if ubx is None else ubx.ctypes.data,
                                     None if uby is None else uby.ctypes.data, float(ds),
                                     float(drs or 0.0), C.c_void_p(fb_ptr), Fp,
                                     C.c_void_p(stream or None))
    return rc, (float(Fp[0]), float(Fp[1]))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64).ravel()


class Lattice:
    """One BTDF-IB/LBM context.  Fields are (ny, nx) arrays, x fastest."""

    def __init__(self, nx, ny, tau, u_in=0.0, delta=3, nf=1, storage=BTDF_F32,
                 bc_x=BTDF_BCX_PERIODIC, bc_y=BTDF_BCY_PERIODIC, gx=0.0, gy=0.0,
                 history_len=4096, stream: int = 0, layout=None):
        cfg = btdf_config_default()
        if layout is not None:
            cfg.layout = int(layout)
        cfg.nx, cfg.ny, cfg.tau, cfg.u_in = int(nx), int(ny), float(tau), float(u_in)
        cfg.delta, cfg.nf, cfg.storage = int(delta), int(nf), int(storage)
        cfg.bc_x, cfg.bc_y, cfg.history_len = int(bc_x), int(bc_y), int(history_len)
        cfg.gx, cfg.gy = float(gx), float(gy)
        self.cfg = cfg
        self.nx, self.ny = int(nx), int(ny)
        rc, ctx = btdf_create(cfg, stream)
        if rc != BTDF_OK:
            raise BtdfError(rc, f"btdf_create: {btdf_status_string(rc)}")
        self._ctx = ctx
        self.body_markers = []

    @classmethod
    def from_case(cls, case, storage=BTDF_F32, stream: int = 0, history_len=4096, drs=None,
                  layout=None):
        lat = cls(case.nx, case.ny, case.tau, case.u_in, case.delta, case.nf, storage,
                  case.bc_x, case.bc_y, case.gx, case.gy, history_len, stream, layout)
        lat.init_fields(*case.initial_fields())
        for b in case.bodies:
            lat.add_markers(b.X, b.Y, b.ds, b.Ubx, b.Uby, drs=case.drs if drs is None else drs)
        return lat

    def _check(self, rc: int, what: str):
        if rc != BTDF_OK:
            msg = lib().btdf_last_error(self._ctx).decode()
            raise BtdfError(rc, f"{what}: {btdf_status_string(rc)}: {msg}")

    def close(self):
        if getattr(self, "_ctx", None):
            lib().btdf_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, rho, ux, uy):
        self._check(lib().btdf_init_fields(self._ctx, _f64(rho), _f64(ux), _f64(uy)),
                    "btdf_init_fields")

    def add_markers(self, X, Y, ds, Ubx=None, Uby=None, drs=0.0) -> int:
        X, Y = _f64(X), _f64(Y)
        n = len(X)
        ubx = None if Ubx is None else _f64(Ubx)
        uby = None if Uby is None else _f64(Uby)
        bid = C.c_int32(-1)
        rc = lib().btdf_add_markers(self._ctx, n, X, Y,
                                    None if ubx is None else ubx.ctypes.data,
                                    None if uby is None else uby.ctypes.data,
                                    float(ds), float(drs or 0.0), C.byref(bid))
        self._check(rc, "btdf_add_markers")
        self.body_markers.append(n)
        return bid.value

    def set_boundary_velocity(self, ubx, uby):
        """Outer-node velocities of a BTDF_BCX_BOX lattice, perimeter order
        (row 0, row ny-1, column 0 without corners, column nx-1 without corners)."""
        self._check(lib().btdf_set_boundary_velocity(self._ctx, _f64(ubx), _f64(uby)),
                    "btdf_set_boundary_velocity")

    def add_cylinder(self, cx, cy, D, n, drs=0.0) -> int:
        bid = C.c_int32(-1)
        self._check(lib().btdf_add_cylinder(self._ctx, float(cx), float(cy), float(D), int(n),
                                            float(drs or 0.0), C.byref(bid)), "btdf_add_cylinder")
        self.body_markers.append(int(n))
        return bid.value

    def set_marker_velocity(self, body, Ubx, Uby):
        """Prescribed velocities of one body's markers, or with body = -1 of
        every marker (in the order the bodies were added)."""
        self._check(lib().btdf_set_marker_velocity(self._ctx, body, _f64(Ubx), _f64(Uby)),
                    "btdf_set_marker_velocity")

    def step(self, n=1):
        self._check(lib().btdf_step(self._ctx, int(n)), "btdf_step")

    def sync(self):
        self._check(lib().btdf_sync(self._ctx), "btdf_sync")

    @property
    def steps(self) -> int:
        return lib().btdf_step_count(self._ctx)

    def forces(self, body=0, first=0, n=None, out=None):
        """Body force (Eq. 27) of steps first .. first+n-1: arrays of n, or,
        with body = -1, of shape (n, bodies) (every body per step)."""
        n = self.steps - first if n is None else n
        shape = (n, len(self.body_markers)) if body == -1 else (n,)
        if out is None:
            out = (np.zeros(shape), np.zeros(shape))
        Fx, Fy = out
        self._check(lib().btdf_read_forces(self._ctx, body, first, n, Fx.ctypes.data,
                                           Fy.ctypes.data), "btdf_read_forces")
        return Fx, Fy

    def forces_async(self, body, first, n, ptr: int):
        """Enqueues the copy of n steps' body force into host memory at ptr
        (n x 2 doubles, Fx Fy; page-locked for a true asynchronous copy);
        valid after sync()."""
        self._check(lib().btdf_read_forces_async(self._ctx, int(body), int(first), int(n), ptr),
                    "btdf_read_forces_async")

    def markers(self, body=0):
        n = self.body_markers[body]
        a = [np.zeros(n, dtype=np.float32) for _ in range(4)]
        self._check(lib().btdf_read_markers(self._ctx, body, *[x.ctypes.data for x in a]),
                    "btdf_read_markers")
        return dict(zip(["Usx", "Usy", "Fbx", "Fby"], a))

    def field(self, kind):
        shape = (9, self.ny, self.nx) if kind == FIELD_POPS else (self.ny, self.nx)
        out = np.zeros(shape, dtype=np.float32)
        self._check(lib().btdf_read_field(self._ctx, kind, out.ctypes.data, 0), "btdf_read_field")
        return out

    def field_to_device(self, kind, ptr: int):
        self._check(lib().btdf_read_field(self._ctx, kind, ptr, 1), "btdf_read_field")

    def moments(self):
        return self.field(FIELD_RHO), self.field(FIELD_UX), self.field(FIELD_UY)

    def save_state(self) -> bytes:
        n = C.c_size_t()
        self._check(lib().btdf_state_size(self._ctx, C.byref(n)), "btdf_state_size")
        buf = (C.c_char * n.value)()
        used = C.c_size_t()
        self._check(lib().btdf_save_state(self._ctx, buf, n.value, C.byref(used)),
                    "btdf_save_state")
        return bytes(buf)

    def load_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        self._check(lib().btdf_load_state(self._ctx, buf, len(blob)), "btdf_load_state")

    def profile(self, on: bool):
        self._check(lib().btdf_profile_enable(self._ctx, 1 if on else 0), "btdf_profile_enable")

    def profile_read(self):
        a, b = C.c_double(), C.c_double()
        la, lb = C.c_int64(), C.c_int64()
        self._check(lib().btdf_profile_read(self._ctx, C.byref(a), C.byref(b), C.byref(la),
                                            C.byref(lb)), "btdf_profile_read")
        return a.value, b.value, la.value, lb.value

    def tune(self, variant=0, grid_blocks=0):
        """Collide-stream kernel variant (btdf_tune: 0 automatic, 1 .. VARIANT_COUNT - 1)
        and an optional cap on its grid (0: the variant's default)."""
        self._check(lib().btdf_tune(self._ctx, int(variant), int(grid_blocks)), "btdf_tune")

    def device_bytes(self) -> int:
        n = C.c_size_t()
        self._check(lib().btdf_device_bytes(self._ctx, C.byref(n)), "btdf_device_bytes")
        return n.value

    def autotune(self, steps=20, flush_l2=True):
        """Times every collide-stream variant on this lattice (btdf_autotune),
        keeps the fastest; returns (chosen, {variant: interquartile mean ms per step})."""
        ch = C.c_int32()
        ms = np.zeros(VARIANT_COUNT, dtype=np.float32)
        self._check(lib().btdf_autotune(self._ctx, int(steps), 1 if flush_l2 else 0, C.byref(ch),
                                        ms.ctypes.data), "btdf_autotune")
        return ch.value, {v: float(ms[v]) for v in range(1, VARIANT_COUNT) if ms[v] >= 0}

    def set_wait_limit(self, polls):
        """Polls before a TMA stage wait gives up (< 0: the default bound)."""
        self._check(lib().btdf_set_wait_limit(self._ctx, int(polls)), "btdf_set_wait_limit")

    def set_inflow(self, u_in):
        self._check(lib().btdf_set_inflow(self._ctx, float(u_in)), "btdf_set_inflow")

    def move_markers(self, body, X, Y):
        self._check(lib().btdf_move_markers(self._ctx, int(body), _f64(X), _f64(Y)),
                    "btdf_move_markers")

    @property
    def marker_count(self) -> int:
        return int(sum(self.body_markers))

    def body_first_marker(self, body) -> int:
        return int(sum(self.body_markers[:body]))

    def adjoint_forward(self, nsteps, every=50, body=-1, dref=1.0) -> float:
        """Window-averaged drag coefficient over the next nsteps steps
        (btdf_adjoint_forward); keeps the tape for adjoint_backward."""
        J = C.c_double()
        self._check(lib().btdf_adjoint_forward(self._ctx, int(nsteps), int(every), int(body),
                                               float(dref), C.byref(J)), "btdf_adjoint_forward")
        return J.value

    def adjoint_backward(self):
        """(dJ/du_in, dJ/dX[markers], dJ/dY[markers]) of the last forward window."""
        n = self.marker_count
        dX, dY = np.zeros(n), np.zeros(n)
        dU = C.c_double()
        self._check(lib().btdf_adjoint_backward(self._ctx, C.byref(dU), dX.ctypes.data,
                                                dY.ctypes.data), "btdf_adjoint_backward")
        return dU.value, dX, dY

    def adjoint_release(self):
        self._check(lib().btdf_adjoint_release(self._ctx), "btdf_adjoint_release")


def _case_config(case, storage=BTDF_F32, history_len=4096, layout=None) -> btdf_config:
    cfg = btdf_config_default()
    cfg.nx, cfg.ny, cfg.tau, cfg.u_in = case.nx, case.ny, float(case.tau), float(case.u_in)
    cfg.delta, cfg.nf, cfg.storage = int(case.delta), int(case.nf), int(storage)
    cfg.bc_x, cfg.bc_y, cfg.history_len = int(case.bc_x), int(case.bc_y), int(history_len)
    cfg.gx, cfg.gy = float(case.gx), float(case.gy)
    if layout is not None:
        cfg.layout = int(layout)
    return cfg


class Batch:
    """Many independent lattices advanced together (btdf_batch_*)."""

    def __init__(self, cases, storage=BTDF_F32, history_len=4096, stream: int = 0, layout=None):
        n = len(cases)
        cfgs = (btdf_config * n)(*[_case_config(c, storage, history_len, layout) for c in cases])
        out = C.c_void_p()
        rc = lib().btdf_batch_create(cfgs, n, C.c_void_p(stream or None), C.byref(out))
        if rc != BTDF_OK:
            raise BtdfError(rc, f"btdf_batch_create: {btdf_status_string(rc)}")
        self._b = out.value
        self.cases = list(cases)
        self.storage = int(storage)
        self.bodies = []          # (lattice, markers) per batch-wide body id

    @classmethod
    def from_cases(cls, cases, storage=BTDF_F32, history_len=4096, stream: int = 0, layout=None):
        bt = cls(cases, storage, history_len, stream, layout)
        for i, c in enumerate(cases):
            bt.init_fields(i, *c.initial_fields())
        for i, c in enumerate(cases):
            for b in c.bodies:
                bt.add_markers(i, b.X, b.Y, b.ds, b.Ubx, b.Uby, drs=c.drs)
        return bt

    def _check(self, rc, what):
        if rc != BTDF_OK:
            msg = lib().btdf_batch_last_error(self._b).decode()
            raise BtdfError(rc, f"{what}: {btdf_status_string(rc)}: {msg}")

    def close(self):
        if getattr(self, "_b", None):
            lib().btdf_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, lattice, rho, ux, uy):
        self._check(lib().btdf_batch_init_fields(self._b, lattice, _f64(rho), _f64(ux), _f64(uy)),
                    "btdf_batch_init_fields")

    def add_markers(self, lattice, X, Y, ds, Ubx=None, Uby=None, drs=0.0) -> int:
        X, Y = _f64(X), _f64(Y)
        ubx = None if Ubx is None else _f64(Ubx)
        uby = None if Uby is None else _f64(Uby)
        bid = C.c_int32(-1)
        rc = lib().btdf_batch_add_markers(self._b, lattice, len(X), X, Y,
                                          None if ubx is None else ubx.ctypes.data,
                                          None if uby is None else uby.ctypes.data, float(ds),
                                          float(drs or 0.0), C.byref(bid))
        self._check(rc, "btdf_batch_add_markers")
        self.bodies.append((lattice, len(X)))
        return bid.value

    def tune(self, variant):
        self._check(lib().btdf_batch_tune(self._b, int(variant)), "btdf_batch_tune")

    def autotune(self, steps=10, flush_l2=False):
        """Times launch shapes 1..4 on the batch (btdf_batch_autotune)."""
        ch = C.c_int32()
        ms = np.zeros(5, dtype=np.float32)
        self._check(lib().btdf_batch_autotune(self._b, int(steps), 1 if flush_l2 else 0,
                                              C.byref(ch), ms.ctypes.data), "btdf_batch_autotune")
        return ch.value, {v: float(ms[v]) for v in (1, 2, 3, 4)}

    def step(self, n=1):
        self._check(lib().btdf_batch_step(self._b, int(n)), "btdf_batch_step")

    def sync(self):
        self._check(lib().btdf_batch_sync(self._b), "btdf_batch_sync")

    @property
    def steps(self):
        return lib().btdf_batch_step_count(self._b)

    def forces(self, body, first=0, n=None):
        n = self.steps - first if n is None else n
        Fx, Fy = np.zeros(n), np.zeros(n)
        self._check(lib().btdf_batch_read_forces(self._b, body, first, n, Fx.ctypes.data,
                                                 Fy.ctypes.data), "btdf_batch_read_forces")
        return Fx, Fy

    def field(self, lattice, kind):
        c = self.cases[lattice]
        shape = (9, c.ny, c.nx) if kind == FIELD_POPS else (c.ny, c.nx)
        out = np.zeros(shape, dtype=np.float32)
        self._check(lib().btdf_batch_read_field(self._b, lattice, kind, out.ctypes.data, 0),
                    "btdf_batch_read_field")
        return out
