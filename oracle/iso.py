"""Marshalling for the isosurface oracle (``iso_oracle.c``) -- TEST INFRASTRUCTURE ONLY.

Field and polygonisation follow Sec. 3.4 as stated in the C source; this module only
converts arrays.
"""
from __future__ import annotations

import ctypes

import numpy as np

_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")


def declare(L):
    L.orc_iso_field.restype = None
    L.orc_iso_field.argtypes = [ctypes.c_int, _f32p, _f64p, _i32p, ctypes.c_double, _i32p, _f32p,
                                ctypes.c_float, _f64p]
    L.orc_iso_polygonize.restype = ctypes.c_longlong
    L.orc_iso_polygonize.argtypes = [_f64p, _i32p, _f64p, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_longlong, _f64p, _i64p]


def grid(lo, hi, cube: float):
    """Corner counts and FP32 corner (0,0,0): origin lo + cube / 2, floor((hi - lo) / cube)
    corners per axis."""
    cube32 = np.float32(cube)
    origin = np.array([np.float32(np.float32(l) + np.float32(0.5) * cube32) for l in lo], np.float32)
    dims = np.array([int(np.floor((float(np.float32(h)) - float(np.float32(l))) / float(cube32)))
                     for l, h in zip(lo, hi)], np.int32)
    return dims, origin


def field(x: np.ndarray, m: np.ndarray, is_fluid: np.ndarray, h: float, dims, origin,
          cube: float) -> np.ndarray:
    """Fluid density at every corner, shape (nz, ny, nx)."""
    from . import lib
    x = np.ascontiguousarray(x, np.float32)
    d = np.ascontiguousarray(dims, np.int32)
    out = np.zeros(int(np.prod(d)), np.float64)
    lib().orc_iso_field(x.shape[0], x, np.ascontiguousarray(m, np.float64),
                        np.ascontiguousarray(is_fluid, np.int32), float(np.float32(h)), d,
                        np.ascontiguousarray(origin, np.float32), float(np.float32(cube)), out)
    return out.reshape(d[2], d[1], d[0])


def polygonize(fld: np.ndarray, origin, cube: float, iso: float, max_tris: int = None):
    """Triangles (n, 3, 3) and their vertices' cube-edge ids (n, 3)."""
    from . import lib
    f = np.ascontiguousarray(fld, np.float64)
    nz, ny, nx = f.shape
    d = np.array([nx, ny, nz], np.int32)
    o = np.ascontiguousarray(origin, np.float64)
    if max_tris is None:
        max_tris = 8 * (nx - 1) * (ny - 1) * (nz - 1)
    xyz = np.zeros(9 * max(max_tris, 1), np.float64)
    vid = np.zeros(3 * max(max_tris, 1), np.int64)
    n = lib().orc_iso_polygonize(f.ravel(), d, o, float(cube), float(iso), int(max_tris), xyz, vid)
    k = min(int(n), max_tris)
    return xyz[:9 * k].reshape(k, 3, 3), vid[:3 * k].reshape(k, 3)
