"""FP64 CPU oracle for the D2Q9I lattice-BGK update (PortLBM, Sec. 3.1-3.3).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline / reference leg may import this package; the product path
(``paper_2607_20650_gb300``) never does. The arithmetic lives in
``lbm_oracle.c`` (plain C, FP64, two-lattice pull, canonical layout
h[i*N + n]); this module only compiles it and marshals numpy arrays.

Every function here is pinned by ``tests/test_oracle_pins.py`` against closed
forms, invariants or exact-rational brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_SRC3 = os.path.join(_HERE, "lbm3_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liblbm_oracle.so")

# Edge conditions (same numbering as the C source).
PERIODIC, WALL, FREESLIP, INLET_ZOUHE, INLET_EQ, OUTFLOW_ZG, INLET_EQ_NEUMANN, OUTLET_PRESSURE = range(8)

CX = np.array([-1, 0, 1, -1, 0, 1, -1, 0, 1])
CY = np.array([-1, -1, -1, 0, 0, 0, 1, 1, 1])


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("tau", ctypes.c_double), ("fx", ctypes.c_double), ("fy", ctypes.c_double),
        ("ux_in", ctypes.c_double), ("uy_in", ctypes.c_double),
        ("bc_w", ctypes.c_int32), ("bc_e", ctypes.c_int32),
        ("bc_s", ctypes.c_int32), ("bc_n", ctypes.c_int32),
        ("rho_out", ctypes.c_double),
    ]


class _Params3(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("tau", ctypes.c_double), ("fx", ctypes.c_double), ("fy", ctypes.c_double),
        ("fz", ctypes.c_double),
        ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32), ("bc_z", ctypes.c_int32),
        ("bc_xe", ctypes.c_int32),
        ("ux_in", ctypes.c_double), ("uy_in", ctypes.c_double), ("uz_in", ctypes.c_double),
        ("rho_out", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c with gcc (OpenMP, no FP contraction) if stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC3))):
        return _LIB
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-std=c11", _SRC, _SRC3, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, u8 = P(ctypes.c_double), P(ctypes.c_uint8)
        lib.oracle_equilibrium.argtypes = [ctypes.c_double] * 3 + [d]
        lib.oracle_effective_solid.argtypes = [P(_Params), u8, u8]
        lib.oracle_init.argtypes = [P(_Params), u8, d, d, d, d]
        lib.oracle_step.argtypes = [P(_Params), u8, d, d, d, d, d]
        lib.oracle_run.argtypes = [P(_Params), u8, d, ctypes.c_int64, d, d, d]
        lib.oracle_run.restype = ctypes.c_int
        lib.oracle_mass.argtypes = [P(_Params), u8, d]
        lib.oracle_mass.restype = ctypes.c_double
        lib.oracle_force.argtypes = [P(_Params), u8, u8, d, d]
        lib.oracle_omp_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        P3 = P(_Params3)
        lib.oracle3_directions.argtypes = [P(ctypes.c_int32), d]
        lib.oracle3_equilibrium.argtypes = [ctypes.c_double] * 4 + [d]
        lib.oracle3_effective_solid.argtypes = [P3, u8, u8]
        lib.oracle3_init.argtypes = [P3, u8, d, d, d, d, d]
        lib.oracle3_run.argtypes = [P3, u8, d, ctypes.c_int64, d, d, d, d]
        lib.oracle3_run.restype = ctypes.c_int
        lib.oracle3_mass.argtypes = [P3, u8, d]
        lib.oracle3_mass.restype = ctypes.c_double
        lib.oracle3_force.argtypes = [P3, u8, u8, d, d]
        _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


@dataclass
class Case:
    """One lattice: size, relaxation time, force, inlet velocity, edges."""
    nx: int
    ny: int
    tau: float
    fx: float = 0.0
    fy: float = 0.0
    ux_in: float = 0.0
    uy_in: float = 0.0
    bc_w: int = PERIODIC
    bc_e: int = PERIODIC
    bc_s: int = PERIODIC
    bc_n: int = PERIODIC
    rho_out: float = 1.0

    def _c(self):
        return _Params(self.nx, self.ny, self.tau, self.fx, self.fy, self.ux_in,
                       self.uy_in, self.bc_w, self.bc_e, self.bc_s, self.bc_n, self.rho_out)


def omp_threads() -> int:
    return int(_load().oracle_omp_threads())


def set_threads(n: int) -> None:
    """OpenMP threads of the oracle's parallel loops from now on."""
    _load().oracle_set_threads(int(n))


def equilibrium(drho: float, ux: float, uy: float) -> np.ndarray:
    """h_i^eq = f_i^eq - w_i of Eq. (2) for rho = 1 + drho, velocity (ux, uy)."""
    out = np.zeros(9)
    _load().oracle_equilibrium(drho, ux, uy, _dp(out))
    return out


def effective_solid(case: Case, mask: np.ndarray) -> np.ndarray:
    mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    out = np.zeros_like(mask)
    _load().oracle_effective_solid(ctypes.byref(case._c()), _u8(mask), _u8(out))
    return out


class Lattice:
    """Oracle state: canonical h[i, n] (shape 9 x N, FP64) + effective solid mask."""

    def __init__(self, case: Case, mask: np.ndarray | None = None,
                 rho=None, ux=None, uy=None):
        self.case = case
        N = case.nx * case.ny
        if mask is None:
            mask = np.zeros(N, np.uint8)
        self.solid = effective_solid(case, mask)
        self.h = np.zeros((9, N))
        arr = [None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
               for a in (rho, ux, uy)]
        _load().oracle_init(ctypes.byref(case._c()), _u8(self.solid),
                            *[_dp(a) for a in arr], _dp(self.h))
        self.rho = np.where(self.solid > 0, 1.0, 1.0 if arr[0] is None else arr[0])
        self.ux = np.where(self.solid > 0, 0.0, 0.0 if arr[1] is None else arr[1])
        self.uy = np.where(self.solid > 0, 0.0, 0.0 if arr[2] is None else arr[2])
        self.steps = 0

    def set_h(self, h: np.ndarray):
        self.h = np.ascontiguousarray(h, dtype=np.float64).reshape(9, -1).copy()

    def run(self, nsteps: int):
        """nsteps updates; rho/ux/uy hold the moments of the last one."""
        if nsteps <= 0:
            return self
        N = self.case.nx * self.case.ny
        self.rho = np.empty(N)
        self.ux = np.empty(N)
        self.uy = np.empty(N)
        rc = _load().oracle_run(ctypes.byref(self.case._c()), _u8(self.solid), _dp(self.h),
                                int(nsteps), _dp(self.rho), _dp(self.ux), _dp(self.uy))
        if rc != 0:
            raise MemoryError("oracle_run: out of host memory")
        self.steps += nsteps
        return self

    def mass(self) -> float:
        return float(_load().oracle_mass(ctypes.byref(self.case._c()), _u8(self.solid),
                                         _dp(self.h)))

    def force(self, body: np.ndarray) -> np.ndarray:
        body = np.ascontiguousarray(body, dtype=np.uint8).reshape(-1)
        out = np.zeros(2)
        _load().oracle_force(ctypes.byref(self.case._c()), _u8(self.solid), _u8(body),
                             _dp(self.h), _dp(out))
        return out

    def field(self, a: np.ndarray) -> np.ndarray:
        return a.reshape(self.case.ny, self.case.nx)


# ------------------------------------------------------------ D3Q19

@dataclass
class Case3:
    """A D3Q19 lattice: size, tau, force, per-axis faces (PERIODIC or WALL);
    on x the west face may be INLET_EQ or INLET_ZOUHE (velocity u_in) and the
    east face (bc_xe, default: as bc_x) OUTFLOW_ZG or OUTLET_PRESSURE
    (density rho_out)."""
    nx: int
    ny: int
    nz: int
    tau: float
    fx: float = 0.0
    fy: float = 0.0
    fz: float = 0.0
    bc_x: int = PERIODIC
    bc_y: int = PERIODIC
    bc_z: int = PERIODIC
    bc_xe: int = -1
    u_in: tuple = (0.0, 0.0, 0.0)
    rho_out: float = 1.0

    def _c(self):
        east = self.bc_x if self.bc_xe < 0 else self.bc_xe
        return _Params3(self.nx, self.ny, self.nz, self.tau, self.fx, self.fy, self.fz,
                        self.bc_x, self.bc_y, self.bc_z, east, *[float(u) for u in self.u_in],
                        float(self.rho_out))


def directions3():
    """(19 x 3) integer velocities and 19 weights of the D3Q19 set."""
    c = np.zeros(57, dtype=np.int32)
    w = np.zeros(19)
    _load().oracle3_directions(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(w))
    return c.reshape(19, 3), w


def equilibrium3(drho, ux, uy, uz) -> np.ndarray:
    out = np.zeros(19)
    _load().oracle3_equilibrium(drho, ux, uy, uz, _dp(out))
    return out


class Lattice3:
    """D3Q19 oracle state: canonical h[i, n], n = (z*ny + y)*nx + x."""

    def __init__(self, case: Case3, mask=None, rho=None, ux=None, uy=None, uz=None):
        self.case = case
        N = case.nx * case.ny * case.nz
        if mask is None:
            mask = np.zeros(N, np.uint8)
        mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        self.solid = np.zeros_like(mask)
        _load().oracle3_effective_solid(ctypes.byref(case._c()), _u8(mask), _u8(self.solid))
        self.h = np.zeros((19, N))
        arr = [None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
               for a in (rho, ux, uy, uz)]
        _load().oracle3_init(ctypes.byref(case._c()), _u8(self.solid), *[_dp(a) for a in arr],
                             _dp(self.h))
        self.steps = 0

    def set_h(self, h):
        self.h = np.ascontiguousarray(h, dtype=np.float64).reshape(19, -1).copy()

    def run(self, nsteps: int):
        N = self.h.shape[1]
        self.rho, self.ux, self.uy, self.uz = (np.empty(N) for _ in range(4))
        rc = _load().oracle3_run(ctypes.byref(self.case._c()), _u8(self.solid), _dp(self.h),
                                 int(nsteps), _dp(self.rho), _dp(self.ux), _dp(self.uy), _dp(self.uz))
        if rc != 0:
            raise MemoryError("oracle3_run: out of host memory")
        self.steps += nsteps
        return self

    def mass(self) -> float:
        return float(_load().oracle3_mass(ctypes.byref(self.case._c()), _u8(self.solid), _dp(self.h)))

    def force(self, body: np.ndarray) -> np.ndarray:
        """Momentum-exchange force on the body (3 components)."""
        body = np.ascontiguousarray(body, dtype=np.uint8).reshape(-1)
        out = np.zeros(3)
        _load().oracle3_force(ctypes.byref(self.case._c()), _u8(self.solid), _u8(body), _dp(self.h),
                              _dp(out))
        return out
