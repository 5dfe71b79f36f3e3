"""Thin ctypes binding of libdugks.so (declared in include/dugks.h).

Argument marshalling only: every step of the method runs in the CUDA kernels of
the library. There is no CPU fallback: if the library cannot be loaded, or no
CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

DUGKS_OK, DUGKS_EINVAL, DUGKS_ENOMEM, DUGKS_ECUDA, DUGKS_ETIMEOUT, DUGKS_ENONFINITE, DUGKS_ESTATE, DUGKS_EAGAIN = range(8)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENONFINITE", 6: "ESTATE",
                7: "EAGAIN"}
DUGKS_FP64, DUGKS_FP32, DUGKS_FP16F = 0, 1, 2
DUGKS_UPWIND, DUGKS_CENTRAL = 0, 1
DUGKS_VEL_UNIFORM, DUGKS_VEL_ROTATION, DUGKS_VEL_VORTEX, DUGKS_VEL_FIELD, DUGKS_VEL_DEFORM = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": DUGKS_FP64, "fp32": DUGKS_FP32, "fp16f": DUGKS_FP16F}
VEL_KINDS = {"uniform": 0, "rotation": 1, "vortex": 2, "field": 3, "deformation": 4}


class dugks_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("W", ctypes.c_double), ("M", ctypes.c_double), ("cfl", ctypes.c_double),
        ("order", ctypes.c_int32), ("flux", ctypes.c_int32), ("stages", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("dtphiu", ctypes.c_int32),
        ("phiA", ctypes.c_double), ("phiB", ctypes.c_double),
    ]


class DugksError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        super().__init__(f"dugks error {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None

# (name, restype, argtypes) of every entry point declared in include/dugks.h
_VP, _DP, _I64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64
SIGNATURES = [
    ("dugks_create", ctypes.c_int, [ctypes.POINTER(dugks_params), _DP, _VP, ctypes.POINTER(_VP)]),
    ("dugks_set_velocity", ctypes.c_int, [_VP, ctypes.c_int, _DP, _DP, _DP]),
    ("dugks_step", ctypes.c_int, [_VP, _I64]),
    ("dugks_read_phi", ctypes.c_int, [_VP, _DP]),
    ("dugks_read_phi_device", ctypes.c_int, [_VP, _VP]),
    ("dugks_debug_faces", ctypes.c_int, [_VP, _DP, _DP, _DP, _DP]),
    ("dugks_mass", ctypes.c_int, [_VP, _DP]),
    ("dugks_mass_device", ctypes.c_int, [_VP, _VP]),
    ("dugks_status", ctypes.c_int, [_VP]),
    ("dugks_selftest_wait_timeout", ctypes.c_int, [_VP, ctypes.c_uint32]),
    ("dugks_selftest_fail_allocs", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32]),
    ("dugks_last_error", ctypes.c_char_p, [_VP]),
    ("dugks_step_index", _I64, [_VP]),
    ("dugks_set_variant", ctypes.c_int, [_VP, ctypes.c_int]),
    ("dugks_get_variant", ctypes.c_int, [_VP]),
    ("dugks_state_bytes", ctypes.c_size_t, [_VP]),
    ("dugks_save_state", ctypes.c_int, [_VP, _VP, ctypes.c_size_t, ctypes.POINTER(_I64)]),
    ("dugks_load_state", ctypes.c_int, [_VP, _VP, ctypes.c_size_t, _I64]),
    ("dugks_destroy", None, [_VP]),
    ("dugks_field_mass_noalloc", ctypes.c_int,
     [_VP, ctypes.c_int, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP, _VP]),
    ("dugks_batch_create", ctypes.c_int, [ctypes.POINTER(dugks_params), _VP, ctypes.POINTER(_VP)]),
    ("dugks_batch_grid_bytes", ctypes.c_size_t, [ctypes.POINTER(dugks_params), ctypes.c_int32, ctypes.c_int32]),
    ("dugks_batch_add", ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, _DP, ctypes.c_int, _DP, _I64,
                                       ctypes.POINTER(ctypes.c_int32)]),
    ("dugks_batch_remove", ctypes.c_int, [_VP, ctypes.c_int32]),
    ("dugks_batch_retire", ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64)]),
    ("dugks_batch_collect", ctypes.c_int, [_VP, ctypes.c_int32, _DP, ctypes.c_int]),
    ("dugks_batch_fence", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint64)]),
    ("dugks_batch_reached", ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32)]),
    ("dugks_batch_set_ctas", ctypes.c_int, [_VP, ctypes.c_int32]),
    ("dugks_batch_step", ctypes.c_int, [_VP, _I64]),
    ("dugks_batch_step_index", _I64, [_VP, ctypes.c_int32]),
    ("dugks_batch_read_phi", ctypes.c_int, [_VP, ctypes.c_int32, _DP]),
    ("dugks_batch_mass", ctypes.c_int, [_VP, ctypes.c_int32, _DP]),
    ("dugks_batch_set_variant", ctypes.c_int, [_VP, ctypes.c_int]),
    ("dugks_batch_active_cells", _I64, [_VP]),
    ("dugks_batch_status", ctypes.c_int, [_VP]),
    ("dugks_batch_last_error", ctypes.c_char_p, [_VP]),
    ("dugks_batch_destroy", None, [_VP]),
]
DUGKS_NOALLOC_MAX_TILES = 65536


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libdugks.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(ctx, code: int):
    if code != DUGKS_OK:
        msg = lib().dugks_last_error(ctx).decode() if ctx else ""
        raise DugksError(code, msg)


# ---- the C entry points under the same names --------------------------------

def dugks_create(params: dugks_params, phi0: np.ndarray, stream: int | None = None):
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
    if phi0.shape != (params.ny, params.nx):
        raise ValueError("phi0 must be (ny, nx)")
    out = ctypes.c_void_p()
    code = lib().dugks_create(ctypes.byref(params), _dptr(phi0), ctypes.c_void_p(stream or 0), ctypes.byref(out))
    _check(None, code)
    return out.value


def dugks_set_velocity(ctx, kind: int, params=None, u: np.ndarray | None = None, v: np.ndarray | None = None):
    p = np.ascontiguousarray(list(params or []) + [0.0] * 4, dtype=np.float64)
    up = vp = None
    if u is not None:
        u = np.ascontiguousarray(u, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        up, vp = _dptr(u), _dptr(v)
    _check(ctx, lib().dugks_set_velocity(ctx, kind, _dptr(p), up, vp))


def dugks_step(ctx, nsteps: int):
    _check(ctx, lib().dugks_step(ctx, int(nsteps)))


def dugks_read_phi(ctx, out: np.ndarray):
    _check(ctx, lib().dugks_read_phi(ctx, _dptr(out)))
    return out


def dugks_read_phi_device(ctx, dev_ptr: int):
    _check(ctx, lib().dugks_read_phi_device(ctx, ctypes.c_void_p(dev_ptr)))


def dugks_debug_faces(ctx, fbar_E: np.ndarray, fbar_N: np.ndarray, f_E: np.ndarray, f_N: np.ndarray):
    _check(ctx, lib().dugks_debug_faces(ctx, _dptr(fbar_E), _dptr(fbar_N), _dptr(f_E), _dptr(f_N)))


def dugks_mass(ctx) -> float:
    m = ctypes.c_double()
    _check(ctx, lib().dugks_mass(ctx, ctypes.byref(m)))
    return m.value


def dugks_mass_device(ctx, dev_ptr: int):
    _check(ctx, lib().dugks_mass_device(ctx, ctypes.c_void_p(dev_ptr)))


def dugks_status(ctx) -> int:
    return lib().dugks_status(ctx)


def dugks_selftest_wait_timeout(ctx, max_polls: int) -> int:
    """Enqueues the bounded-wait self-test (see include/dugks.h); returns the code."""
    return lib().dugks_selftest_wait_timeout(ctx, int(max_polls))


def dugks_selftest_fail_allocs(skip: int, count: int) -> int:
    """Arms the host-side allocation-failure hook (see include/dugks.h); returns the code."""
    return lib().dugks_selftest_fail_allocs(int(skip), int(count))


def dugks_last_error(ctx) -> str:
    return lib().dugks_last_error(ctx).decode()


def dugks_step_index(ctx) -> int:
    return lib().dugks_step_index(ctx)


def dugks_set_variant(ctx, variant: int):
    _check(ctx, lib().dugks_set_variant(ctx, int(variant)))


def dugks_get_variant(ctx) -> int:
    return lib().dugks_get_variant(ctx)


def dugks_state_bytes(ctx) -> int:
    return lib().dugks_state_bytes(ctx)


def dugks_save_state(ctx, buf) -> int:
    """buf: a writable buffer (numpy uint8 array, or an address with .nbytes)."""
    idx = ctypes.c_int64()
    addr, n = _buf(buf)
    _check(ctx, lib().dugks_save_state(ctx, ctypes.c_void_p(addr), n, ctypes.byref(idx)))
    return idx.value


def dugks_load_state(ctx, buf, step_index: int):
    addr, n = _buf(buf)
    _check(ctx, lib().dugks_load_state(ctx, ctypes.c_void_p(addr), n, int(step_index)))


def dugks_destroy(ctx):
    if ctx:
        lib().dugks_destroy(ctx)


def _buf(buf):
    if isinstance(buf, np.ndarray):
        assert buf.flags["C_CONTIGUOUS"]
        return buf.ctypes.data, buf.nbytes
    # torch tensor (e.g. pinned host memory)
    return buf.data_ptr(), buf.numel() * buf.element_size()


def dugks_field_mass_noalloc(field_ptr: int, dtype: int, nx: int, ny: int, pitch: int, out_ptr: int,
                             stream: int | None = None) -> int:
    """FP64 sum of a device field (double: dtype 0, float: dtype 1) into the
    device double at out_ptr, without allocating device memory. Returns the
    status code (enqueues only; does not wait)."""
    return lib().dugks_field_mass_noalloc(ctypes.c_void_p(field_ptr), int(dtype), int(nx), int(ny), int(pitch),
                                          ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream or 0))


def make_params(nx, ny, W=4.0, M=0.01, cfl=0.8, order=2, flux=0, stages=2, precision="fp64",
                dtphiu=1, phiA=1.0, phiB=0.0) -> dugks_params:
    p = dugks_params()
    p.nx, p.ny, p.W, p.M, p.cfl = nx, ny, W, M, cfl
    p.order, p.flux, p.stages = order, flux, stages
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else precision
    p.dtphiu, p.phiA, p.phiB = dtphiu, phiA, phiB
    return p


# ---- batches of grids ----------------------------------------------------------

def _bcheck(b, code: int):
    if code != DUGKS_OK:
        msg = lib().dugks_batch_last_error(b).decode() if b else ""
        raise DugksError(code, msg)


def dugks_batch_create(params: dugks_params, stream: int | None = None):
    out = ctypes.c_void_p()
    _bcheck(None, lib().dugks_batch_create(ctypes.byref(params), ctypes.c_void_p(stream or 0), ctypes.byref(out)))
    return out.value


def dugks_batch_grid_bytes(params: dugks_params, nx: int, ny: int) -> int:
    return lib().dugks_batch_grid_bytes(ctypes.byref(params), int(nx), int(ny))


def dugks_batch_add(b, nx: int, ny: int, phi0: np.ndarray, vel_kind: int, vel, target_steps: int = -1) -> int:
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
    if phi0.shape != (ny, nx):
        raise ValueError("phi0 must be (ny, nx)")
    v = np.ascontiguousarray(list(vel) + [0.0] * 4, dtype=np.float64)
    gid = ctypes.c_int32()
    _bcheck(b, lib().dugks_batch_add(b, int(nx), int(ny), _dptr(phi0), int(vel_kind), _dptr(v), int(target_steps),
                                     ctypes.byref(gid)))
    return gid.value


def dugks_batch_remove(b, gid: int):
    _bcheck(b, lib().dugks_batch_remove(b, int(gid)))


def dugks_batch_retire(b, gid: int) -> int:
    t = ctypes.c_uint64()
    _bcheck(b, lib().dugks_batch_retire(b, int(gid), ctypes.byref(t)))
    return t.value


def dugks_batch_collect(b, gid: int, out: np.ndarray, wait: bool = False) -> bool:
    """True with phi in `out` (freed grid); False if the read-out is still in flight."""
    r = lib().dugks_batch_collect(b, int(gid), _dptr(out), 1 if wait else 0)
    if r == DUGKS_EAGAIN:
        return False
    _bcheck(b, r)
    return True


def dugks_batch_fence(b) -> int:
    t = ctypes.c_uint64()
    _bcheck(b, lib().dugks_batch_fence(b, ctypes.byref(t)))
    return t.value


def dugks_batch_reached(b, ticket: int) -> bool:
    done = ctypes.c_int32()
    _bcheck(b, lib().dugks_batch_reached(b, ctypes.c_uint64(int(ticket)), ctypes.byref(done)))
    return bool(done.value)


def dugks_batch_set_ctas(b, ctas: int):
    _bcheck(b, lib().dugks_batch_set_ctas(b, int(ctas)))


def dugks_batch_step(b, nsteps: int):
    _bcheck(b, lib().dugks_batch_step(b, int(nsteps)))


def dugks_batch_step_index(b, gid: int) -> int:
    return lib().dugks_batch_step_index(b, int(gid))


def dugks_batch_read_phi(b, gid: int, out: np.ndarray):
    _bcheck(b, lib().dugks_batch_read_phi(b, int(gid), _dptr(out)))
    return out


def dugks_batch_mass(b, gid: int) -> float:
    m = ctypes.c_double()
    _bcheck(b, lib().dugks_batch_mass(b, int(gid), ctypes.byref(m)))
    return m.value


def dugks_batch_set_variant(b, variant: int):
    _bcheck(b, lib().dugks_batch_set_variant(b, int(variant)))


def dugks_batch_active_cells(b) -> int:
    return lib().dugks_batch_active_cells(b)


def dugks_batch_status(b) -> int:
    return lib().dugks_batch_status(b)


def dugks_batch_last_error(b) -> str:
    return lib().dugks_batch_last_error(b).decode()


def dugks_batch_destroy(b):
    if b:
        lib().dugks_batch_destroy(b)


class Batch:
    """Owning wrapper of a batch of independent grids sharing W, M, cfl, order, flux, precision."""

    def __init__(self, *, stream: int | None = None, **kw):
        self.params = make_params(8, 8, **kw)
        self.b = dugks_batch_create(self.params, stream)
        self.shapes = {}
        self.tickets = {}   # grid id -> fence ticket of its pending read-out

    def grid_bytes(self, nx: int, ny: int) -> int:
        return dugks_batch_grid_bytes(self.params, nx, ny)

    def add(self, phi0: np.ndarray, vel_kind="uniform", vel=(0.0, 0.0), target_steps: int = -1) -> int:
        ny, nx = phi0.shape
        gid = dugks_batch_add(self.b, nx, ny, phi0, VEL_KINDS[vel_kind], vel, target_steps)
        self.shapes[gid] = (ny, nx)
        return gid

    def add_problem(self, prob, target_steps: int | None = None) -> int:
        return self.add(prob.phi0, prob.vel_kind, prob.vel, prob.steps if target_steps is None else target_steps)

    def remove(self, gid: int):
        dugks_batch_remove(self.b, gid)
        self.shapes.pop(gid, None)
        self.tickets.pop(gid, None)

    def step(self, n: int = 1):
        dugks_batch_step(self.b, n)
        return self

    def step_index(self, gid: int) -> int:
        return dugks_batch_step_index(self.b, gid)

    def retire(self, gid: int) -> int:
        """Freezes the grid and queues its read-out; returns the fence ticket."""
        t = dugks_batch_retire(self.b, gid)
        self.tickets[gid] = t
        return t

    def collect(self, gid: int, wait: bool = False):
        """phi of a retired grid (the grid is freed), or None while the copy is in flight."""
        t = self.tickets.get(gid)
        if not wait and t is not None and not dugks_batch_reached(self.b, t):
            return None   # (no output buffer made while the copy is in flight)
        out = np.empty(self.shapes[gid])
        if not dugks_batch_collect(self.b, gid, out, wait):
            return None
        self.shapes.pop(gid, None)
        self.tickets.pop(gid, None)
        return out

    def fence(self) -> int:
        return dugks_batch_fence(self.b)

    def reached(self, ticket: int) -> bool:
        return dugks_batch_reached(self.b, ticket)

    def set_ctas(self, ctas: int):
        dugks_batch_set_ctas(self.b, ctas)

    def phi(self, gid: int) -> np.ndarray:
        out = np.empty(self.shapes[gid])
        return dugks_batch_read_phi(self.b, gid, out)

    def mass(self, gid: int) -> float:
        return dugks_batch_mass(self.b, gid)

    def set_variant(self, v: int):
        dugks_batch_set_variant(self.b, v)

    def active_cells(self) -> int:
        return dugks_batch_active_cells(self.b)

    def status(self) -> int:
        return dugks_batch_status(self.b)

    def close(self):
        if getattr(self, "b", None):
            dugks_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Solver:
    """Owning wrapper of one context: create, set velocity, step, read."""

    def __init__(self, nx, ny, phi0, *, vel_kind="uniform", vel=(0.0, 0.0), u=None, v=None,
                 stream: int | None = None, **kw):
        self.params = make_params(nx, ny, **kw)
        self.ctx = dugks_create(self.params, phi0, stream)
        try:
            dugks_set_velocity(self.ctx, VEL_KINDS[vel_kind], vel, u, v)
        except Exception:
            self.close()
            raise

    @classmethod
    def from_problem(cls, prob, precision="fp64", stream=None):
        return cls(prob.nx, prob.ny, prob.phi0, vel_kind=prob.vel_kind, vel=prob.vel, W=prob.W, M=prob.M,
                   cfl=prob.cfl, order=prob.order, flux=prob.flux, stages=prob.stages,
                   precision=precision, dtphiu=prob.dtphiu, stream=stream)

    def step(self, n=1):
        dugks_step(self.ctx, n)
        return self

    def phi(self) -> np.ndarray:
        out = np.empty((self.params.ny, self.params.nx))
        return dugks_read_phi(self.ctx, out)

    def mass(self) -> float:
        return dugks_mass(self.ctx)

    def debug_faces(self):
        """(bar f at east faces, at north faces, f at east faces, at north faces) of the
        current state's step, each (9, ny, nx); the state does not advance."""
        shape = (9, self.params.ny, self.params.nx)
        out = [np.empty(shape) for _ in range(4)]
        dugks_debug_faces(self.ctx, *out)
        return tuple(out)

    @property
    def step_index(self) -> int:
        return dugks_step_index(self.ctx)

    def set_variant(self, v: int):
        dugks_set_variant(self.ctx, v)

    def status(self) -> int:
        return dugks_status(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            dugks_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
