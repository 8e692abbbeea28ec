"""ctypes binding of liblbm.so (C ABI in include/lbm.h).

Functions carry the C names and only marshal arguments: every step of the
update runs in the library's CUDA kernels. PyTorch supplies device memory
(the workspace) and streams. There is no CPU fallback: if the library is not
built, the first call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EDIVERGED, LBM_ETIMEOUT, LBM_EUNSUPPORTED = range(7)
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EDIVERGED", 5: "ETIMEOUT", 6: "EUNSUPPORTED"}
LAYOUTS = {"stream": 0, "bundle": 1, "collision": 2}
ALGOS = {"lptl": 0, "nptl": 1, "npol": 2, "nsol": 3, "aa": 4}
STORAGES = {"f64": 0, "f32": 1, "f16s": 2, "bf16s": 3}
ROUNDINGS = {"rne": 0, "sr": 1}
PERIODIC, WALL, FREESLIP, INLET_ZOUHE, INLET_EQ, OUTFLOW_ZG, INLET_EQ_NEUMANN, OUTLET_PRESSURE = range(8)
LBM_FLAG_NO_GRAPH = 1
LBM_FLAG_TWO_NODES_PER_THREAD = 2
LBM_FLAG_NO_STAGING = 4
LBM_FLAG_WIDE_OFFSETS = 8
LBM_FLAG_NO_PREFETCH = 16
LBM_FLAG_NO_PAIRS = 32
LBM_FLAG_NO_TMA = 64
LBM_AUTO = -1


class LbmError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("tau", ctypes.c_double),
        ("force", ctypes.c_double * 2),
        ("u_in", ctypes.c_double * 2),
        ("bc_west", ctypes.c_int32), ("bc_east", ctypes.c_int32),
        ("bc_south", ctypes.c_int32), ("bc_north", ctypes.c_int32),
        ("layout", ctypes.c_int32), ("algo", ctypes.c_int32),
        ("storage", ctypes.c_int32), ("rounding", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
        ("rho_out", ctypes.c_double),
    ]


class lbm_info(ctypes.Structure):
    _fields_ = [
        ("cells", ctypes.c_int64), ("fluid_cells", ctypes.c_int64), ("steps", ctypes.c_int64),
        ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32), ("aux", ctypes.c_int32),
        ("bytes_per_update", ctypes.c_double), ("workspace_bytes", ctypes.c_size_t),
    ]


class lbm_tuning(ctypes.Structure):
    _fields_ = [
        ("ns_per_cell", (ctypes.c_double * 4) * 3),
        ("ns_per_tile", ctypes.c_double),
        ("valid", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class lbm3_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("tau", ctypes.c_double),
        ("force", ctypes.c_double * 3),
        ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32), ("bc_z", ctypes.c_int32),
        ("layout", ctypes.c_int32), ("algo", ctypes.c_int32),
        ("storage", ctypes.c_int32), ("rounding", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32), ("tile_z", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
        ("bc_x_east", ctypes.c_int32),
        ("u_in", ctypes.c_double * 3),
        ("rho_out", ctypes.c_double),
    ]


# Every symbol include/lbm.h declares, with (restype, argtypes).
_P = ctypes.POINTER
_vp, _i32, _i64, _u32, _u64, _dbl, _sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                          ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                                          ctypes.c_size_t)
SIGNATURES = {
    "lbm_workspace_bytes": (_i32, [_P(lbm_params), _P(_sz)]),
    "lbm_create": (_i32, [_P(lbm_params), _vp, _vp, _sz, _vp, _P(_vp)]),
    "lbm_init": (_i32, [_vp, _vp, _vp, _vp]),
    "lbm_step": (_i32, [_vp, _i64, _u32]),
    "lbm_sync": (_i32, [_vp]),
    "lbm_wait": (_i32, [_vp, _dbl]),
    "lbm_read_moments": (_i32, [_vp, _vp, _vp, _vp]),
    "lbm_moments_device": (_i32, [_vp, _vp, _vp, _vp]),
    "lbm_mass": (_i32, [_vp, _P(_dbl)]),
    "lbm_force": (_i32, [_vp, _vp, _P(_dbl)]),
    "lbm_read_populations": (_i32, [_vp, _vp, _i32]),
    "lbm_write_populations": (_i32, [_vp, _vp, _i32]),
    "lbm_face_pack": (_i32, [_vp, _i32, _i32, _vp]),
    "lbm_face_unpack": (_i32, [_vp, _i32, _i32, _vp]),
    "lbm_face_exchange": (_i32, [_i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "lbm_get_info": (_i32, [_vp, _P(lbm_info)]),
    "lbm_destroy": (None, [_vp]),
    "lbm_last_error": (ctypes.c_char_p, []),
    "lbm_layout_index": (_i64, [_i32, _i64, _i64, _i32]),
    "lbm_quantize": (_i32, [_i32, _i32, _u64, _i64, _vp, _vp, _vp, _i64, _vp]),
    "lbm_mass_f32_noalloc": (_i32, [_vp, _vp, _i64, _P(_dbl), _vp]),
    "lbm_mask_channel_walls": (_i32, [_i32, _i32, _vp]),
    "lbm_mask_disc": (_i32, [_i32, _i32, _dbl, _dbl, _dbl, _i32, _vp]),
    "lbm_mask_porous_discs": (_i32, [_i32, _i32, _u64, _dbl, _dbl, _dbl, _vp]),
    "lbm_mask_naca4": (_i32, [_i32, _i32, _dbl, _dbl, _dbl, _dbl, _dbl, _i32, _vp]),
    "lbm3_mask_porous_spheres": (_i32, [_i32, _i32, _i32, _u64, _dbl, _dbl, _dbl, _vp]),
    "lbm_tune": (_i32, [_P(lbm_params), _vp, _vp, _sz, _vp, _P(lbm_tuning)]),
    "lbm_tune_workspace_bytes": (_i32, [_P(lbm_params), _P(_sz)]),
    "lbm_batch_plan": (_i32, [_i32, _P(lbm_params), _P(lbm_tuning)]),
    "lbm_batch_workspace_bytes": (_i32, [_i32, _P(lbm_params), _P(_sz)]),
    "lbm_batch_create": (_i32, [_i32, _P(lbm_params), _P(_vp), _vp, _sz, _vp, _P(_vp)]),
    "lbm_batch_init": (_i32, [_vp, _i32, _vp, _vp, _vp]),
    "lbm_batch_step": (_i32, [_vp, _i64, _u32]),
    "lbm_batch_sync": (_i32, [_vp]),
    "lbm_batch_read_moments": (_i32, [_vp, _i32, _vp, _vp, _vp]),
    "lbm_batch_read_populations": (_i32, [_vp, _i32, _vp, _i32]),
    "lbm_batch_get_info": (_i32, [_vp, _P(_i64), _P(_i32), _P(_i64)]),
    "lbm_batch_destroy": (None, [_vp]),
    "lbm3_workspace_bytes": (_i32, [_P(lbm3_params), _P(_sz)]),
    "lbm3_create": (_i32, [_P(lbm3_params), _vp, _vp, _sz, _vp, _P(_vp)]),
    "lbm3_init": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "lbm3_step": (_i32, [_vp, _i64, _u32]),
    "lbm3_sync": (_i32, [_vp]),
    "lbm3_read_moments": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "lbm3_read_populations": (_i32, [_vp, _vp, _i32]),
    "lbm3_write_populations": (_i32, [_vp, _vp, _i32]),
    "lbm3_mass": (_i32, [_vp, _P(_dbl)]),
    "lbm3_force": (_i32, [_vp, _vp, _P(_dbl)]),
    "lbm3_get_info": (_i32, [_vp, _P(lbm_info)]),
    "lbm3_destroy": (None, [_vp]),
    "lbm3_layout_index": (_i64, [_i32, _i64, _i64, _i32]),
    "lbm3_face_pack": (_i32, [_vp, _i32, _i32, _vp]),
    "lbm3_face_unpack": (_i32, [_vp, _i32, _i32, _vp]),
    "lbm3_face_exchange": (_i32, [_i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "lbm3_batch_workspace_bytes": (_i32, [_i32, _P(lbm3_params), _P(_sz)]),
    "lbm3_batch_create": (_i32, [_i32, _P(lbm3_params), _P(_vp), _vp, _sz, _vp, _P(_vp)]),
    "lbm3_batch_init": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp]),
    "lbm3_batch_step": (_i32, [_vp, _i64, _u32]),
    "lbm3_batch_sync": (_i32, [_vp]),
    "lbm3_batch_read_moments": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp]),
    "lbm3_batch_read_populations": (_i32, [_vp, _i32, _vp, _i32]),
    "lbm3_batch_mass": (_i32, [_vp, _i32, _P(_dbl)]),
    "lbm3_batch_get_info": (_i32, [_vp, _P(_i64), _P(_i64), _P(_i64), _P(_dbl)]),
    "lbm3_batch_destroy": (None, [_vp]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load liblbm.so; raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            if not build_if_missing:
                raise RuntimeError(f"liblbm.so not built ({_build.LIB}); run "
                                   "paper_2607_20650_gb300.build.build()")
            _build.build()
        lib = ctypes.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(status: int, where: str):
    if status != LBM_OK:
        raise LbmError(status, where, load().lbm_last_error().decode())


def _ptr(a) -> int | None:
    """Device or host address of a torch tensor / numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)


def make_params(nx, ny, tau, *, force=(0.0, 0.0), u_in=(0.0, 0.0), bc=(PERIODIC,) * 4,
                layout="stream", algo="nptl", storage="f32", rounding="rne", seed=0,
                tile=(0, 0), flags=0, rho_out=1.0) -> lbm_params:
    """bc = (west, east, south, north)."""
    p = lbm_params()
    p.nx, p.ny, p.tau = int(nx), int(ny), float(tau)
    p.force[0], p.force[1] = force
    p.u_in[0], p.u_in[1] = u_in
    p.bc_west, p.bc_east, p.bc_south, p.bc_north = bc
    p.layout = LAYOUTS[layout] if isinstance(layout, str) else int(layout)
    p.algo = ALGOS[algo] if isinstance(algo, str) else int(algo)
    p.storage = STORAGES[storage] if isinstance(storage, str) else int(storage)
    p.rounding = ROUNDINGS[rounding] if isinstance(rounding, str) else int(rounding)
    p.seed = int(seed)
    p.tile_x, p.tile_y = tile
    p.flags = int(flags)
    p.rho_out = float(rho_out)
    return p


# ------------------------------------------------------------ C names

def lbm_workspace_bytes(p: lbm_params) -> int:
    b = ctypes.c_size_t()
    _check(load().lbm_workspace_bytes(ctypes.byref(p), ctypes.byref(b)), "lbm_workspace_bytes")
    return b.value


def lbm_create(p: lbm_params, mask: np.ndarray, workspace, nbytes: int, stream: int):
    m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    h = ctypes.c_void_p()
    _check(load().lbm_create(ctypes.byref(p), m.ctypes.data, _ptr(workspace), nbytes, stream,
                             ctypes.byref(h)), "lbm_create")
    return h


def lbm_init(h, rho=None, ux=None, uy=None):
    arrs = [_f64(a) for a in (rho, ux, uy)]
    _check(load().lbm_init(h, *[_ptr(a) for a in arrs]), "lbm_init")


def lbm_step(h, nsteps: int, want_moments: bool = False):
    _check(load().lbm_step(h, int(nsteps), 1 if want_moments else 0), "lbm_step")


def lbm_sync(h):
    _check(load().lbm_sync(h), "lbm_sync")


def lbm_wait(h, timeout_s: float) -> int:
    """Returns the status (LBM_OK or LBM_ETIMEOUT); raises on other errors."""
    s = load().lbm_wait(h, float(timeout_s))
    if s not in (LBM_OK, LBM_ETIMEOUT):
        _check(s, "lbm_wait")
    return s


def lbm_read_moments(h, N: int, out=None):
    """(rho, ux, uy) as FP64 host arrays; ``out`` gives the three arrays
    (N contiguous doubles each, e.g. views of page-locked torch tensors)."""
    if out is None:
        out = [np.empty(N) for _ in range(3)]
    for a in out:
        if a.dtype != np.float64 or a.size != N or not a.flags.c_contiguous:
            raise ValueError("moments output arrays must be N contiguous float64 values each")
    _check(load().lbm_read_moments(h, *[a.ctypes.data for a in out]), "lbm_read_moments")
    return out


def lbm_moments_device(h, rho, ux, uy):
    _check(load().lbm_moments_device(h, _ptr(rho), _ptr(ux), _ptr(uy)), "lbm_moments_device")


def lbm_mass(h) -> float:
    out = ctypes.c_double()
    _check(load().lbm_mass(h, ctypes.byref(out)), "lbm_mass")
    return out.value


def lbm_force(h, body=None) -> np.ndarray:
    out = (ctypes.c_double * 2)()
    _check(load().lbm_force(h, _ptr(body), out), "lbm_force")
    return np.array([out[0], out[1]])


def lbm_read_populations(h, N: int, as_: str = "f64") -> np.ndarray:
    out = np.empty((9, N), dtype=np.float64 if as_ == "f64" else np.float32)
    _check(load().lbm_read_populations(h, out.ctypes.data, STORAGES[as_]), "lbm_read_populations")
    return out


def lbm_write_populations(h, pops: np.ndarray):
    a = np.ascontiguousarray(pops)
    as_ = "f64" if a.dtype == np.float64 else "f32"
    a = a.astype(np.float64 if as_ == "f64" else np.float32, copy=False)
    _check(load().lbm_write_populations(h, a.ctypes.data, STORAGES[as_]), "lbm_write_populations")


def lbm_face_pack(h, x: int, sense: int, d_buf):
    """Three populations crossing the face x -> x + sense of column x into
    d_buf (device, 3 * ny stored values)."""
    _check(load().lbm_face_pack(h, int(x), int(sense), _ptr(d_buf)), "lbm_face_pack")


def lbm_face_unpack(h, x: int, sense: int, d_buf):
    _check(load().lbm_face_unpack(h, int(x), int(sense), _ptr(d_buf)), "lbm_face_unpack")


def _face_exchange(fn: str, src: list, xs: list, dst: list, xd: list, sense: list, stream: int):
    n = len(src)
    hs = (ctypes.c_void_p * max(n, 1))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in src])
    hd = (ctypes.c_void_p * max(n, 1))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in dst])
    a, b, c = [(ctypes.c_int32 * max(n, 1))(*map(int, v)) for v in (xs, xd, sense)]
    _check(getattr(load(), fn)(n, hs, a, hd, b, c, stream), fn)


def lbm_face_exchange(src: list, xs: list, dst: list, xd: list, sense: list, stream: int):
    """One launch for every message between lattices of this process:
    column xs[k] of src[k] -> column xd[k] of dst[k] (handles)."""
    _face_exchange("lbm_face_exchange", src, xs, dst, xd, sense, stream)


def lbm3_face_pack(h, x: int, sense: int, d_buf):
    _check(load().lbm3_face_pack(h, int(x), int(sense), _ptr(d_buf)), "lbm3_face_pack")


def lbm3_face_unpack(h, x: int, sense: int, d_buf):
    _check(load().lbm3_face_unpack(h, int(x), int(sense), _ptr(d_buf)), "lbm3_face_unpack")


def lbm3_face_exchange(src: list, xs: list, dst: list, xd: list, sense: list, stream: int):
    _face_exchange("lbm3_face_exchange", src, xs, dst, xd, sense, stream)


def lbm_get_info(h) -> dict:
    i = lbm_info()
    _check(load().lbm_get_info(h, ctypes.byref(i)), "lbm_get_info")
    out = {f: getattr(i, f) for f, _ in lbm_info._fields_ if f != "aux"}
    out["aux"] = int(i.aux)   # NSOL: 1 = tiles staged by tensor copies; else the prefetch distance
    out["prefetch_distance"] = int(i.aux)
    return out


def lbm_destroy(h):
    load().lbm_destroy(h)


def lbm_layout_index(layout, N: int, n: int, i: int) -> int:
    lay = LAYOUTS[layout] if isinstance(layout, str) else int(layout)
    return int(load().lbm_layout_index(lay, int(N), int(n), int(i)))


def lbm_quantize(storage, rounding, seed, t, d_in, d_out, d_back, count, stream):
    _check(load().lbm_quantize(STORAGES[storage] if isinstance(storage, str) else storage,
                               ROUNDINGS[rounding] if isinstance(rounding, str) else rounding,
                               int(seed), int(t), _ptr(d_in), _ptr(d_out), _ptr(d_back),
                               int(count), stream), "lbm_quantize")


def lbm_mask_channel_walls(nx: int, ny: int) -> np.ndarray:
    m = np.empty((ny, nx), np.uint8)
    _check(load().lbm_mask_channel_walls(nx, ny, m.ctypes.data), "lbm_mask_channel_walls")
    return m


def lbm_mask_disc(nx: int, ny: int, xc: float, yc: float, r: float, periodic: bool = False,
                  out: np.ndarray | None = None) -> np.ndarray:
    m = np.zeros((ny, nx), np.uint8) if out is None else out
    _check(load().lbm_mask_disc(nx, ny, xc, yc, r, int(periodic), m.ctypes.data), "lbm_mask_disc")
    return m


def lbm_mask_porous_discs(nx: int, ny: int, seed: int, rmin: float = 8.0, rmax: float = 32.0,
                          solid_fraction: float = 0.4) -> np.ndarray:
    m = np.empty((ny, nx), np.uint8)
    _check(load().lbm_mask_porous_discs(nx, ny, seed, rmin, rmax, solid_fraction, m.ctypes.data),
           "lbm_mask_porous_discs")
    return m


def lbm_mask_naca4(nx: int, ny: int, chord: float, m: float = 0.02, p: float = 0.4, t: float = 0.12,
                   aoa_deg: float = 8.0, n_points: int = 2048) -> np.ndarray:
    out = np.empty((ny, nx), np.uint8)
    _check(load().lbm_mask_naca4(nx, ny, chord, m, p, t, aoa_deg, n_points, out.ctypes.data), "lbm_mask_naca4")
    return out


def lbm3_mask_porous_spheres(nx: int, ny: int, nz: int, seed: int, rmin: float = 4.0, rmax: float = 12.0,
                             solid_fraction: float = 0.3) -> np.ndarray:
    m = np.empty((nz, ny, nx), np.uint8)
    _check(load().lbm3_mask_porous_spheres(nx, ny, nz, seed, rmin, rmax, solid_fraction, m.ctypes.data),
           "lbm3_mask_porous_spheres")
    return m


def lbm_mass_f32_noalloc(d_h, d_solid, N: int, stream: int) -> float:
    """Mass of a canonical FP32 state on the device without any workspace."""
    out = ctypes.c_double()
    _check(load().lbm_mass_f32_noalloc(_ptr(d_h), _ptr(d_solid), int(N), ctypes.byref(out), stream),
           "lbm_mass_f32_noalloc")
    return out.value


def lbm_tune_workspace_bytes(probe: lbm_params) -> int:
    b = ctypes.c_size_t()
    _check(load().lbm_tune_workspace_bytes(ctypes.byref(probe), ctypes.byref(b)), "lbm_tune_workspace_bytes")
    return b.value


def lbm_tune(probe: lbm_params, mask, workspace, nbytes: int, stream: int) -> lbm_tuning:
    t = lbm_tuning()
    m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    _check(load().lbm_tune(ctypes.byref(probe), m.ctypes.data, _ptr(workspace), nbytes, stream,
                           ctypes.byref(t)), "lbm_tune")
    return t


def _param_array(params):
    arr = (lbm_params * len(params))()
    for k, p in enumerate(params):
        arr[k] = p
    return arr


def lbm_batch_plan(params: list, tuning: lbm_tuning | None = None) -> list:
    """Resolve LBM_AUTO layout/algo and (0, 0) tiles; returns updated params."""
    arr = _param_array(params)
    _check(load().lbm_batch_plan(len(params), arr, ctypes.byref(tuning) if tuning else None),
           "lbm_batch_plan")
    return [arr[k] for k in range(len(params))]


def lbm_batch_workspace_bytes(params: list) -> int:
    b = ctypes.c_size_t()
    _check(load().lbm_batch_workspace_bytes(len(params), _param_array(params), ctypes.byref(b)),
           "lbm_batch_workspace_bytes")
    return b.value


def lbm_batch_create(params: list, masks: list, workspace, nbytes: int, stream: int):
    arr = _param_array(params)
    ms = [np.ascontiguousarray(m, dtype=np.uint8).reshape(-1) for m in masks]
    ptrs = (ctypes.c_void_p * len(ms))(*[m.ctypes.data for m in ms])
    h = ctypes.c_void_p()
    _check(load().lbm_batch_create(len(params), arr, ptrs, _ptr(workspace), nbytes, stream,
                                   ctypes.byref(h)), "lbm_batch_create")
    return h, ms


def lbm_batch_init(h, c: int, rho=None, ux=None, uy=None):
    arrs = [_f64(a) for a in (rho, ux, uy)]
    _check(load().lbm_batch_init(h, int(c), *[_ptr(a) for a in arrs]), "lbm_batch_init")


def lbm_batch_step(h, nsteps: int, want_moments: bool = False):
    _check(load().lbm_batch_step(h, int(nsteps), 1 if want_moments else 0), "lbm_batch_step")


def lbm_batch_sync(h):
    _check(load().lbm_batch_sync(h), "lbm_batch_sync")


def lbm_batch_read_moments(h, c: int, N: int):
    out = [np.empty(N) for _ in range(3)]
    _check(load().lbm_batch_read_moments(h, int(c), *[a.ctypes.data for a in out]),
           "lbm_batch_read_moments")
    return out


def lbm_batch_read_populations(h, c: int, N: int, as_: str = "f64") -> np.ndarray:
    out = np.empty((9, N), dtype=np.float64 if as_ == "f64" else np.float32)
    _check(load().lbm_batch_read_populations(h, int(c), out.ctypes.data, STORAGES[as_]),
           "lbm_batch_read_populations")
    return out


def lbm_batch_get_info(h) -> dict:
    t, g, c = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
    _check(load().lbm_batch_get_info(h, ctypes.byref(t), ctypes.byref(g), ctypes.byref(c)),
           "lbm_batch_get_info")
    return {"tiles": t.value, "grid": g.value, "cells": c.value}


def lbm_batch_destroy(h):
    load().lbm_batch_destroy(h)


# ------------------------------------------------------------ convenience

# ------------------------------------------------------------ D3Q19

def make_params3(nx, ny, nz, tau, *, force=(0.0, 0.0, 0.0), bc=(PERIODIC,) * 3, layout="stream",
                 algo="nptl", storage="f32", rounding="rne", seed=0, tile=(0, 0, 0),
                 flags=0, bc_x_east=OUTFLOW_ZG, u_in=(0.0, 0.0, 0.0), rho_out=1.0) -> lbm3_params:
    """bc = (x, y, z), each PERIODIC or WALL; x may also be INLET_EQ or
    INLET_ZOUHE (west; the east face is then bc_x_east: OUTFLOW_ZG, WALL or
    OUTLET_PRESSURE at density rho_out) or OUTFLOW_ZG (both x faces)."""
    p = lbm3_params()
    p.nx, p.ny, p.nz, p.tau = int(nx), int(ny), int(nz), float(tau)
    for a in range(3):
        p.force[a] = float(force[a])
    p.bc_x, p.bc_y, p.bc_z = bc
    p.layout = LAYOUTS[layout] if isinstance(layout, str) else int(layout)
    p.algo = ALGOS[algo] if isinstance(algo, str) else int(algo)
    p.storage = STORAGES[storage] if isinstance(storage, str) else int(storage)
    p.rounding = ROUNDINGS[rounding] if isinstance(rounding, str) else int(rounding)
    p.seed = int(seed)
    p.tile_x, p.tile_y, p.tile_z = tile
    p.flags = int(flags)
    p.bc_x_east = int(bc_x_east)
    for a in range(3):
        p.u_in[a] = float(u_in[a])
    p.rho_out = float(rho_out)
    return p


def lbm3_workspace_bytes(p: lbm3_params) -> int:
    b = ctypes.c_size_t()
    _check(load().lbm3_workspace_bytes(ctypes.byref(p), ctypes.byref(b)), "lbm3_workspace_bytes")
    return b.value


def lbm3_create(p: lbm3_params, mask: np.ndarray, workspace, nbytes: int, stream: int):
    m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    h = ctypes.c_void_p()
    _check(load().lbm3_create(ctypes.byref(p), m.ctypes.data, _ptr(workspace), nbytes, stream,
                              ctypes.byref(h)), "lbm3_create")
    return h


def lbm3_init(h, rho=None, ux=None, uy=None, uz=None):
    arrs = [_f64(a) for a in (rho, ux, uy, uz)]
    _check(load().lbm3_init(h, *[_ptr(a) for a in arrs]), "lbm3_init")


def lbm3_step(h, nsteps: int, want_moments: bool = False):
    _check(load().lbm3_step(h, int(nsteps), 1 if want_moments else 0), "lbm3_step")


def lbm3_sync(h):
    _check(load().lbm3_sync(h), "lbm3_sync")


def lbm3_read_moments(h, N: int):
    out = [np.empty(N) for _ in range(4)]
    _check(load().lbm3_read_moments(h, *[a.ctypes.data for a in out]), "lbm3_read_moments")
    return out


def lbm3_read_populations(h, N: int, as_: str = "f64") -> np.ndarray:
    out = np.empty((19, N), dtype=np.float64 if as_ == "f64" else np.float32)
    _check(load().lbm3_read_populations(h, out.ctypes.data, STORAGES[as_]), "lbm3_read_populations")
    return out


def lbm3_write_populations(h, pops: np.ndarray):
    a = np.ascontiguousarray(pops)
    as_ = "f64" if a.dtype == np.float64 else "f32"
    a = a.astype(np.float64 if as_ == "f64" else np.float32, copy=False)
    _check(load().lbm3_write_populations(h, a.ctypes.data, STORAGES[as_]), "lbm3_write_populations")


def lbm3_mass(h) -> float:
    out = ctypes.c_double()
    _check(load().lbm3_mass(h, ctypes.byref(out)), "lbm3_mass")
    return out.value


def lbm3_force(h, body=None) -> np.ndarray:
    out = (ctypes.c_double * 3)()
    _check(load().lbm3_force(h, _ptr(body), out), "lbm3_force")
    return np.array([out[0], out[1], out[2]])


def lbm3_get_info(h) -> dict:
    i = lbm_info()
    _check(load().lbm3_get_info(h, ctypes.byref(i)), "lbm3_get_info")
    out = {f: getattr(i, f) for f, _ in lbm_info._fields_ if f != "aux"}
    out["wide_addressing"] = bool(i.aux & 1)
    out["node_pairs"] = bool(i.aux & 2)
    return out


def lbm3_destroy(h):
    load().lbm3_destroy(h)


def lbm3_layout_index(layout, N: int, n: int, i: int) -> int:
    lay = LAYOUTS[layout] if isinstance(layout, str) else int(layout)
    return int(load().lbm3_layout_index(lay, int(N), int(n), int(i)))


def _param3_array(params):
    arr = (lbm3_params * len(params))()
    for k, p in enumerate(params):
        arr[k] = p
    return arr


def lbm3_batch_workspace_bytes(params: list) -> int:
    b = ctypes.c_size_t()
    _check(load().lbm3_batch_workspace_bytes(len(params), _param3_array(params), ctypes.byref(b)),
           "lbm3_batch_workspace_bytes")
    return b.value


def lbm3_batch_create(params: list, masks: list, workspace, nbytes: int, stream: int):
    arr = _param3_array(params)
    ms = [np.ascontiguousarray(m, dtype=np.uint8).reshape(-1) for m in masks]
    ptrs = (ctypes.c_void_p * len(ms))(*[m.ctypes.data for m in ms])
    h = ctypes.c_void_p()
    _check(load().lbm3_batch_create(len(params), arr, ptrs, _ptr(workspace), nbytes, stream,
                                    ctypes.byref(h)), "lbm3_batch_create")
    return h, ms


def lbm3_batch_init(h, c: int, rho=None, ux=None, uy=None, uz=None):
    arrs = [_f64(a) for a in (rho, ux, uy, uz)]
    _check(load().lbm3_batch_init(h, int(c), *[_ptr(a) for a in arrs]), "lbm3_batch_init")


def lbm3_batch_step(h, nsteps: int, want_moments: bool = False):
    _check(load().lbm3_batch_step(h, int(nsteps), 1 if want_moments else 0), "lbm3_batch_step")


def lbm3_batch_sync(h):
    _check(load().lbm3_batch_sync(h), "lbm3_batch_sync")


def lbm3_batch_read_moments(h, c: int, N: int):
    out = [np.empty(N) for _ in range(4)]
    _check(load().lbm3_batch_read_moments(h, int(c), *[a.ctypes.data for a in out]),
           "lbm3_batch_read_moments")
    return out


def lbm3_batch_read_populations(h, c: int, N: int, as_: str = "f64") -> np.ndarray:
    out = np.empty((19, N), dtype=np.float64 if as_ == "f64" else np.float32)
    _check(load().lbm3_batch_read_populations(h, int(c), out.ctypes.data, STORAGES[as_]),
           "lbm3_batch_read_populations")
    return out


def lbm3_batch_mass(h, c: int) -> float:
    out = ctypes.c_double()
    _check(load().lbm3_batch_mass(h, int(c), ctypes.byref(out)), "lbm3_batch_mass")
    return out.value


def lbm3_batch_get_info(h) -> dict:
    it, c, f, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    _check(load().lbm3_batch_get_info(h, ctypes.byref(it), ctypes.byref(c), ctypes.byref(f), ctypes.byref(b)),
           "lbm3_batch_get_info")
    return {"items": it.value, "cells": c.value, "fluid_cells": f.value, "bytes_per_update": b.value}


def lbm3_batch_destroy(h):
    load().lbm3_batch_destroy(h)


def _torch():
    import torch
    return torch


def current_stream() -> int:
    return _torch().cuda.current_stream().cuda_stream


class Lattice:
    """One lattice on the current CUDA device; workspace owned by a torch tensor."""

    def __init__(self, nx, ny, tau, mask=None, stream=None, **kw):
        """stream: a torch.cuda.Stream (default: the current stream)."""
        torch = _torch()
        self.params = make_params(nx, ny, tau, **kw)
        self.nx, self.ny = int(nx), int(ny)
        self.N = self.nx * self.ny
        nbytes = lbm_workspace_bytes(self.params)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.torch_stream = stream if stream is not None else torch.cuda.current_stream()
        self.stream = self.torch_stream.cuda_stream
        if mask is None:
            mask = np.zeros(self.N, np.uint8)
        self.h = lbm_create(self.params, mask, self.workspace, nbytes, self.stream)

    def init(self, rho=None, ux=None, uy=None):
        lbm_init(self.h, rho, ux, uy)
        return self

    def step(self, n: int, moments: bool = False):
        lbm_step(self.h, n, moments)
        return self

    def sync(self):
        lbm_sync(self.h)
        return self

    def moments(self, out=None):
        return lbm_read_moments(self.h, self.N, out)

    def populations(self, as_: str = "f64") -> np.ndarray:
        return lbm_read_populations(self.h, self.N, as_)

    def write_populations(self, pops):
        lbm_write_populations(self.h, pops)

    def face_pack(self, x: int, sense: int, buf):
        lbm_face_pack(self.h, x, sense, buf)

    def face_unpack(self, x: int, sense: int, buf):
        lbm_face_unpack(self.h, x, sense, buf)

    def mass(self) -> float:
        return lbm_mass(self.h)

    def force(self, body=None):
        return lbm_force(self.h, body)

    def info(self) -> dict:
        return lbm_get_info(self.h)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent lattices advanced by one persistent launch per update."""

    def __init__(self, params: list, masks: list, stream=None, plan: bool = True,
                 tuning: lbm_tuning | None = None):
        torch = _torch()
        self.params = lbm_batch_plan(params, tuning) if plan else list(params)
        self.N = [p.nx * p.ny for p in self.params]
        nbytes = lbm_batch_workspace_bytes(self.params)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.torch_stream = stream if stream is not None else torch.cuda.current_stream()
        self.stream = self.torch_stream.cuda_stream
        self.h, self._masks = lbm_batch_create(self.params, masks, self.workspace, nbytes, self.stream)

    def init(self, c, rho=None, ux=None, uy=None):
        lbm_batch_init(self.h, c, rho, ux, uy)
        return self

    def step(self, n: int, moments: bool = False):
        lbm_batch_step(self.h, n, moments)
        return self

    def sync(self):
        lbm_batch_sync(self.h)
        return self

    def moments(self, c):
        return lbm_batch_read_moments(self.h, c, self.N[c])

    def populations(self, c, as_: str = "f64"):
        return lbm_batch_read_populations(self.h, c, self.N[c], as_)

    def info(self) -> dict:
        return lbm_batch_get_info(self.h)

    def close(self):
        if getattr(self, "h", None):
            lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Lattice3:
    """One D3Q19 lattice on the current CUDA device; workspace owned by a torch tensor."""

    def __init__(self, nx, ny, nz, tau, mask=None, stream=None, **kw):
        torch = _torch()
        self.params = make_params3(nx, ny, nz, tau, **kw)
        self.shape = (int(nz), int(ny), int(nx))
        self.N = int(nx) * int(ny) * int(nz)
        nbytes = lbm3_workspace_bytes(self.params)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.torch_stream = stream if stream is not None else torch.cuda.current_stream()
        self.stream = self.torch_stream.cuda_stream
        if mask is None:
            mask = np.zeros(self.N, np.uint8)
        self.h = lbm3_create(self.params, mask, self.workspace, nbytes, self.stream)

    def init(self, rho=None, ux=None, uy=None, uz=None):
        lbm3_init(self.h, rho, ux, uy, uz)
        return self

    def step(self, n: int, moments: bool = False):
        lbm3_step(self.h, n, moments)
        return self

    def sync(self):
        lbm3_sync(self.h)
        return self

    def moments(self):
        return lbm3_read_moments(self.h, self.N)

    def populations(self, as_: str = "f64") -> np.ndarray:
        return lbm3_read_populations(self.h, self.N, as_)

    def write_populations(self, pops):
        lbm3_write_populations(self.h, pops)

    def face_pack(self, x: int, sense: int, buf):
        lbm3_face_pack(self.h, x, sense, buf)

    def face_unpack(self, x: int, sense: int, buf):
        lbm3_face_unpack(self.h, x, sense, buf)

    def mass(self) -> float:
        return lbm3_mass(self.h)

    def force(self, body=None):
        """body: device uint8 tensor of N bytes, or None for every solid node."""
        return lbm3_force(self.h, body)

    def info(self) -> dict:
        return lbm3_get_info(self.h)

    def close(self):
        if getattr(self, "h", None):
            lbm3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch3:
    """Independent D3Q19 boxes advanced by one launch per update."""

    def __init__(self, params: list, masks: list, stream=None):
        torch = _torch()
        self.params = list(params)
        self.N = [p.nx * p.ny * p.nz for p in self.params]
        nbytes = lbm3_batch_workspace_bytes(self.params)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.torch_stream = stream if stream is not None else torch.cuda.current_stream()
        self.stream = self.torch_stream.cuda_stream
        self.h, self._masks = lbm3_batch_create(self.params, masks, self.workspace, nbytes, self.stream)

    def init(self, c, rho=None, ux=None, uy=None, uz=None):
        lbm3_batch_init(self.h, c, rho, ux, uy, uz)
        return self

    def step(self, n: int, moments: bool = False):
        lbm3_batch_step(self.h, n, moments)
        return self

    def sync(self):
        lbm3_batch_sync(self.h)
        return self

    def moments(self, c):
        return lbm3_batch_read_moments(self.h, c, self.N[c])

    def populations(self, c, as_: str = "f64"):
        return lbm3_batch_read_populations(self.h, c, self.N[c], as_)

    def mass(self, c) -> float:
        return lbm3_batch_mass(self.h, c)

    def info(self) -> dict:
        return lbm3_batch_get_info(self.h)

    def close(self):
        if getattr(self, "h", None):
            lbm3_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
