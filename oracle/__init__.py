"""Python handle on the FP64 CPU oracle (``oracle/dugks_oracle.c``).

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module. It shares no code with the
CUDA library and never imports it.

All arrays are float64 numpy arrays, row-major with x fastest; a "9-plane"
array has shape (9, ny, nx) in the D2Q9 velocity order
(0,0),(1,0),(1,1),(0,1),(-1,1),(-1,0),(-1,-1),(0,-1),(1,-1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dugks_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, OpenMP if present)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "dugks_oracle.h"))
    ):
        return _LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]
    tmp = _LIB + f".{os.getpid()}.tmp"
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("W", ctypes.c_double), ("M", ctypes.c_double), ("cfl", ctypes.c_double),
        ("order", ctypes.c_int), ("flux", ctypes.c_int), ("stages", ctypes.c_int),
        ("dtphiu", ctypes.c_int),
        ("phiA", ctypes.c_double), ("phiB", ctypes.c_double),
        ("vel_kind", ctypes.c_int), ("vel", ctypes.c_double * 4),
        ("u_field", ctypes.POINTER(ctypes.c_double)), ("v_field", ctypes.POINTER(ctypes.c_double)),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(_Params)
        D = ctypes.POINTER(ctypes.c_double)
        L.orc_run_lbm.argtypes = [P, D, D, ctypes.c_long, ctypes.c_long]
        L.orc_stencil.argtypes = [ctypes.c_int, ctypes.c_int, D]
        L.orc_derivative.argtypes = [ctypes.c_int, ctypes.c_int, D, ctypes.c_int, ctypes.c_int, D]
        L.orc_velocity.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double, D]
        L.orc_cell_quantities.argtypes = [P, D, D, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, D, D]
        L.orc_reconstruct.argtypes = [P, D, ctypes.c_double, D, D]
        L.orc_face_f.argtypes = [P, D, D, D, ctypes.c_double, ctypes.c_double, D, D]
        L.orc_flux.argtypes = [P, D, D, D]
        L.orc_phi.argtypes = [P, D, D]
        L.orc_init.argtypes = [P, D, D, D]
        L.orc_run.argtypes = [P, D, D, ctypes.c_long, ctypes.c_long]
        L.orc_mass.argtypes = [P, D]
        L.orc_mass.restype = ctypes.c_double
        L.orc_check.argtypes = [P]
        L.orc_coefficients.argtypes = [P, D]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


VEL_KINDS = {"uniform": 0, "rotation": 1, "vortex": 2, "field": 3, "reversing": 4, "deformation": 5}


@dataclass
class Params:
    """Problem statement of Sec. II-III: W, M, C, stencil order, flux, stages."""
    nx: int
    ny: int
    W: float = 4.0
    M: float = 0.01
    cfl: float = 0.8
    order: int = 2
    flux: int = 0            # 0 upwind, 1 central
    stages: int = 2
    dtphiu: int = 1
    phiA: float = 1.0
    phiB: float = 0.0
    vel_kind: str = "uniform"
    vel: tuple = (0.0, 0.0, 0.0, 0.0)
    u_field: np.ndarray | None = None
    v_field: np.ndarray | None = None
    _keep: list = field(default_factory=list, repr=False)

    def c(self) -> _Params:
        p = _Params()
        p.nx, p.ny, p.W, p.M, p.cfl = self.nx, self.ny, self.W, self.M, self.cfl
        p.order, p.flux, p.stages, p.dtphiu = self.order, self.flux, self.stages, self.dtphiu
        p.phiA, p.phiB = self.phiA, self.phiB
        p.vel_kind = VEL_KINDS[self.vel_kind]
        v = list(self.vel) + [0.0] * (4 - len(self.vel))
        for i in range(4):
            p.vel[i] = float(v[i])
        if self.vel_kind == "field":
            u = np.ascontiguousarray(self.u_field, dtype=np.float64)
            w = np.ascontiguousarray(self.v_field, dtype=np.float64)
            self._keep[:] = [u, w]
            p.u_field, p.v_field = _ptr(u), _ptr(w)
        return p

    @property
    def tau(self) -> float:
        return 3.0 * self.M

    @property
    def dt(self) -> float:
        return self.cfl


def stencil(order: int, which: int) -> np.ndarray:
    """5x5 table c[dy + 2, dx + 2] of derivative ``which`` (see dugks_oracle.h)."""
    c = np.zeros(25)
    if lib().orc_stencil(order, which, _ptr(c)):
        raise ValueError("unsupported stencil")
    return c.reshape(5, 5)


def derivative(order: int, which: int, F: np.ndarray) -> np.ndarray:
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.empty_like(F)
    if lib().orc_derivative(order, which, _ptr(F), F.shape[1], F.shape[0], _ptr(out)):
        raise ValueError("unsupported stencil")
    return out


def velocity(p: Params, x: float, y: float, t: float):
    uv = np.zeros(2)
    pc = p.c()
    lib().orc_velocity(ctypes.byref(pc), x, y, t, _ptr(uv))
    return uv


def cell_quantities(p: Params, phi, phi_old, t, t_old, dtD, use_D):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    phi_old = np.ascontiguousarray(phi_old, dtype=np.float64)
    V = np.empty((2, p.ny, p.nx))
    g = np.empty((9, p.ny, p.nx))
    pc = p.c()
    lib().orc_cell_quantities(ctypes.byref(pc), _ptr(phi), _ptr(phi_old), t, t_old, dtD,
                              int(use_D), _ptr(V), _ptr(g))
    return V, g


def reconstruct(p: Params, fbp, h):
    fbp = np.ascontiguousarray(fbp, dtype=np.float64)
    E = np.empty((9, p.ny, p.nx))
    N = np.empty((9, p.ny, p.nx))
    pc = p.c()
    lib().orc_reconstruct(ctypes.byref(pc), _ptr(fbp), h, _ptr(E), _ptr(N))
    return E, N


def face_f(p: Params, fbarE, fbarN, V, h, t_face):
    fbarE = np.ascontiguousarray(fbarE, dtype=np.float64)
    fbarN = np.ascontiguousarray(fbarN, dtype=np.float64)
    V = np.ascontiguousarray(V, dtype=np.float64)
    E = np.empty((9, p.ny, p.nx))
    N = np.empty((9, p.ny, p.nx))
    pc = p.c()
    lib().orc_face_f(ctypes.byref(pc), _ptr(fbarE), _ptr(fbarN), _ptr(V), h, t_face, _ptr(E), _ptr(N))
    return E, N


def flux(p: Params, fE, fN):
    fE = np.ascontiguousarray(fE, dtype=np.float64)
    fN = np.ascontiguousarray(fN, dtype=np.float64)
    L = np.empty((9, p.ny, p.nx))
    pc = p.c()
    lib().orc_flux(ctypes.byref(pc), _ptr(fE), _ptr(fN), _ptr(L))
    return L


def phi_of(p: Params, X):
    X = np.ascontiguousarray(X, dtype=np.float64)
    out = np.empty((p.ny, p.nx))
    pc = p.c()
    lib().orc_phi(ctypes.byref(pc), _ptr(X), _ptr(out))
    return out


def coefficients(p: Params) -> np.ndarray:
    c = np.zeros(8)
    pc = p.c()
    lib().orc_coefficients(ctypes.byref(pc), _ptr(c))
    return c


def check(p: Params) -> bool:
    pc = p.c()
    return lib().orc_check(ctypes.byref(pc)) == 0


class State:
    """Oracle simulation state: 9 planes plus the previous phi and the step index."""

    def __init__(self, p: Params, phi0: np.ndarray):
        self.p = p
        phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
        assert phi0.shape == (p.ny, p.nx)
        self.f = np.empty((9, p.ny, p.nx))
        self.phi_prev = np.empty((p.ny, p.nx))
        self._pc = p.c()
        if lib().orc_init(ctypes.byref(self._pc), _ptr(phi0), _ptr(self.f), _ptr(self.phi_prev)):
            raise ValueError("invalid parameters")
        self.step_index = 0

    def run(self, nsteps: int) -> "State":
        if lib().orc_run(ctypes.byref(self._pc), _ptr(self.f), _ptr(self.phi_prev),
                         self.step_index, int(nsteps)):
            raise ValueError("invalid parameters")
        self.step_index += int(nsteps)
        return self

    def run_lbm(self, nsteps: int) -> "State":
        """The lattice Boltzmann method (stages = 1, cfl = 1): plain streaming."""
        if lib().orc_run_lbm(ctypes.byref(self._pc), _ptr(self.f), _ptr(self.phi_prev),
                             self.step_index, int(nsteps)):
            raise ValueError("invalid parameters")
        self.step_index += int(nsteps)
        return self

    def phi(self) -> np.ndarray:
        return phi_of(self.p, self.f)

    def mass(self) -> float:
        return lib().orc_mass(ctypes.byref(self._pc), _ptr(self.f))


def num_threads() -> int:
    return lib().orc_num_threads()
