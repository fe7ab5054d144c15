"""FP64 CPU oracle of the SPH coupling substep -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's ``cpu_baseline`` /
``--impl reference`` legs may import this package.  It shares no code with the CUDA
path; the only common module is the seeded scene generator, which holds none of the
method's arithmetic.

The C source (``sph_oracle.c``) cites the paper passage each function follows; the
Python side below only marshals arrays and drives substeps in the order of Alg. 2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "sph_oracle.c"), os.path.join(_HERE, "mlp_oracle.c"),
        os.path.join(_HERE, "iso_oracle.c")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

KIND_STATIC, KIND_RIGID, KIND_SOFT = 1, 2, 3
CLAMP_PRESSURE = 1
TAIT = 8
VOLUME_BOUNDARY = 16


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, OpenMP, no FMA contraction)."""
    srcs = [s for s in _SRC if os.path.exists(s)]
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in srcs)):
        return _LIB_PATH
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", _LIB_PATH + ".tmp", *srcs, "-lm"]
    subprocess.check_call(cmd)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


_lib_handle = None


def lib():
    global _lib_handle
    if _lib_handle is None:
        build()
        _lib_handle = ctypes.CDLL(_LIB_PATH)
        _declare(_lib_handle)
    return _lib_handle


class Params(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("rho0", ctypes.c_double), ("k", ctypes.c_double),
                ("nu", ctypes.c_double), ("g", ctypes.c_double * 3), ("dt", ctypes.c_double),
                ("visc_eps", ctypes.c_double), ("spring_zeta", ctypes.c_double),
                ("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3), ("cell", ctypes.c_float),
                ("flags", ctypes.c_int)]


class BodyC(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("first", ctypes.c_int), ("n", ctypes.c_int),
                ("grabbed", ctypes.c_int), ("mass", ctypes.c_double),
                ("inertia", ctypes.c_double * 9), ("t", ctypes.c_float * 3),
                ("q", ctypes.c_float * 4), ("v", ctypes.c_float * 3), ("w", ctypes.c_float * 3),
                ("grab_local", ctypes.c_float * 3), ("local", ctypes.POINTER(ctypes.c_float)),
                ("n_springs", ctypes.c_int), ("springs", ctypes.POINTER(ctypes.c_int)),
                ("spring_L0", ctypes.POINTER(ctypes.c_double)),
                ("spring_k", ctypes.POINTER(ctypes.c_double)),
                ("spring_c", ctypes.POINTER(ctypes.c_double)),
                ("anchored", ctypes.POINTER(ctypes.c_int))]


_P = ctypes.POINTER
_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")


def _declare(L):
    L.orc_alpha.restype = ctypes.c_double
    L.orc_alpha.argtypes = [ctypes.c_double]
    L.orc_W.restype = ctypes.c_double
    L.orc_W.argtypes = [ctypes.c_double, ctypes.c_double]
    L.orc_gradW_coef.restype = ctypes.c_double
    L.orc_gradW_coef.argtypes = [ctypes.c_double, ctypes.c_double]
    L.orc_grid_dims.argtypes = [_P(Params), _i32p]
    L.orc_hash.restype = ctypes.c_int
    L.orc_hash.argtypes = [_P(Params), ctypes.c_int, _f32p, _u32p]
    L.orc_counting_sort.argtypes = [ctypes.c_int, _u32p, ctypes.c_int, _u32p, _i32p]
    L.orc_nnbr_brute.argtypes = [_P(Params), ctypes.c_int, _f32p, _i32p]
    L.orc_support2.restype = ctypes.c_float
    L.orc_support2.argtypes = [_P(Params)]
    L.orc_rot_f32.argtypes = [_f32p, _f32p]
    L.orc_body_point_f32.argtypes = [_f32p, _f32p, _f32p, _f32p]
    L.orc_soft_setup.argtypes = [ctypes.c_int, _i32p, _f32p, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, _f64p, _f64p, _f64p]
    L.orc_substep.restype = ctypes.c_int
    L.orc_substep.argtypes = [_P(Params), ctypes.c_int, ctypes.c_int, _f32p, _f32p, _f32p, _i32p,
                              ctypes.c_int, _P(BodyC), ctypes.c_int, _u32p, _i32p, _u32p,
                              _f64p, _f64p, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
    L.orc_boxcar.argtypes = [ctypes.c_int, ctypes.c_int, _f64p, _f64p]
    L.orc_set_threads.restype = None
    L.orc_set_threads.argtypes = [ctypes.c_int]
    if hasattr(L, "orc_mlp_forward"):
        from . import mlp as _mlp
        _mlp.declare(L)
    if hasattr(L, "orc_iso_polygonize"):
        from . import iso as _iso
        _iso.declare(L)


def _f32(x) -> float:
    """The method's parameters are FP32 values; the oracle computes with those values."""
    return float(np.float32(x))


def params(p: dict) -> Params:
    P = Params()
    P.h, P.rho0, P.k, P.nu = _f32(p["h"]), _f32(p["rho0"]), _f32(p["k"]), _f32(p["nu"])
    for a in range(3):
        P.g[a] = _f32(p["g"][a])
        P.lo[a] = p["lo"][a]
        P.hi[a] = p["hi"][a]
    P.dt, P.visc_eps, P.spring_zeta = _f32(p["dt"]), _f32(p["visc_eps"]), _f32(p["spring_zeta"])
    P.cell = p["cell"]
    P.flags = int(p["flags"]) & (CLAMP_PRESSURE | TAIT | VOLUME_BOUNDARY)
    return P


def set_threads(n: int) -> None:
    """Host threads for the oracle's parallel loops (0: all cores)."""
    lib().orc_set_threads(int(n))


def W(r, h):
    return lib().orc_W(float(r), float(h))


def gradW_coef(r, h):
    return lib().orc_gradW_coef(float(r), float(h))


def alpha(h):
    return lib().orc_alpha(float(h))


def grid_dims(p: dict):
    d = np.zeros(3, np.int32)
    lib().orc_grid_dims(ctypes.byref(params(p)), d)
    return d


def hash_keys(p: dict, x: np.ndarray):
    x = np.ascontiguousarray(x, np.float32)
    keys = np.zeros(x.shape[0], np.uint32)
    bad = lib().orc_hash(ctypes.byref(params(p)), x.shape[0], x, keys)
    return keys, bad


def counting_sort(keys: np.ndarray, ncell: int):
    keys = np.ascontiguousarray(keys, np.uint32)
    cs = np.zeros(ncell + 1, np.uint32)
    src = np.zeros(keys.shape[0], np.int32)
    lib().orc_counting_sort(keys.shape[0], keys, ncell, cs, src)
    return cs, src


def nnbr_brute(p: dict, x: np.ndarray):
    x = np.ascontiguousarray(x, np.float32)
    out = np.zeros(x.shape[0], np.int32)
    lib().orc_nnbr_brute(ctypes.byref(params(p)), x.shape[0], x, out)
    return out


def support2(p: dict) -> float:
    return lib().orc_support2(ctypes.byref(params(p)))


def rot_f32(q):
    R = np.zeros(9, np.float32)
    lib().orc_rot_f32(np.ascontiguousarray(q, np.float32), R)
    return R


def body_point_f32(R, t, l):
    out = np.zeros(3, np.float32)
    lib().orc_body_point_f32(np.ascontiguousarray(R, np.float32),
                             np.ascontiguousarray(t, np.float32),
                             np.ascontiguousarray(l, np.float32), out)
    return out


def soft_setup(pairs, rest_xyz, young, spacing, pmass, zeta):
    pairs = np.ascontiguousarray(pairs, np.int32)
    ns = pairs.shape[0]
    L0, ks, cd = np.zeros(ns), np.zeros(ns), np.zeros(ns)
    lib().orc_soft_setup(ns, pairs, np.ascontiguousarray(rest_xyz, np.float32), float(young),
                         float(spacing), float(pmass), float(zeta), L0, ks, cd)
    return L0, ks, cd


def boxcar(wrenches: np.ndarray, window: int) -> np.ndarray:
    w = np.ascontiguousarray(wrenches, np.float64).reshape(-1, 6)
    out = np.zeros_like(w)
    lib().orc_boxcar(w.shape[0], int(window), w, out)
    return out


def particle_mass(rho0, spacing) -> np.float32:
    """SPH mass rho0 * s^3 as the FP32 value the method stores (each product rounded)."""
    s32 = np.float32(spacing)
    return np.float32(np.float32(rho0) * np.float32(np.float32(s32 * s32) * s32))


class System:
    """Particles in the current slot order plus body states, advanced by `substep`.

    The state between substeps is FP32 (the storage precision of the method); each
    substep computes in FP64 from that state and rounds the new state back to FP32.
    """

    def __init__(self, scene, mode: int = 0):
        p = scene.params
        self.p = p
        self.P = params(p)
        self.mode = mode
        rho0 = np.float32(p["rho0"])
        nf = scene.n_fluid

        def pmass(spacing):
            return particle_mass(rho0, spacing)

        xs = [np.asarray(scene.fluid_x, np.float32)]
        vs = [np.asarray(scene.fluid_v, np.float32)]
        ms = [np.full(nf, pmass(scene.fluid_spacing), np.float32)]
        self.bodies = []
        first = nf
        self._keep = []
        self._springs = []          # (body index, pairs, k_s, c_d) of every soft body
        for b in scene.bodies:
            n = b.n
            bc = BodyC()
            bc.kind, bc.first, bc.n, bc.grabbed = int(b.kind), first, n, 0
            bc.mass = float(b.mass)
            inert = np.asarray(b.inertia, np.float64).reshape(9)
            for a in range(9):
                bc.inertia[a] = inert[a]
            pose = np.asarray(b.pose, np.float32)
            vel = np.asarray(b.vel, np.float32)
            for a in range(3):
                bc.t[a] = pose[a]
                bc.v[a] = vel[a]
                bc.w[a] = vel[3 + a]
                bc.grab_local[a] = b.grab_local[a]
            for a in range(4):
                bc.q[a] = pose[3 + a]
            local = np.ascontiguousarray(b.xyz, np.float32)
            self._keep.append(local)
            bc.local = local.ctypes.data_as(_P(ctypes.c_float))
            pm = pmass(b.spacing)
            if b.kind == KIND_SOFT:
                pairs = np.ascontiguousarray(b.springs, np.int32)
                L0, ks, cd = soft_setup(pairs, b.xyz, b.young, b.spacing, float(pm),
                                        p["spring_zeta"])
                self._keep += [pairs, L0, ks, cd]
                bc.n_springs = pairs.shape[0]
                bc.springs = pairs.ctypes.data_as(_P(ctypes.c_int))
                bc.spring_L0 = L0.ctypes.data_as(_P(ctypes.c_double))
                bc.spring_k = ks.ctypes.data_as(_P(ctypes.c_double))
                bc.spring_c = cd.ctypes.data_as(_P(ctypes.c_double))
                self._springs.append((len(self.bodies), pairs, ks, cd))
                if b.anchors is not None and len(b.anchors):
                    anc = np.zeros(n, np.int32)
                    anc[np.asarray(b.anchors)] = 1
                    self._keep.append(anc)
                    bc.anchored = anc.ctypes.data_as(_P(ctypes.c_int))
            xs.append(local if b.kind != KIND_RIGID else np.zeros((n, 3), np.float32))
            vs.append(np.zeros((n, 3), np.float32))
            ms.append(np.full(n, pm, np.float32))
            self.bodies.append(bc)
            first += n
        self.x = np.ascontiguousarray(np.concatenate(xs), np.float32)
        self.v = np.ascontiguousarray(np.concatenate(vs), np.float32)
        self.m = np.ascontiguousarray(np.concatenate(ms), np.float32)
        self.id = np.arange(self.x.shape[0], dtype=np.int32)
        self.nf = nf
        self.n = self.x.shape[0]
        self.grab_body = scene.grab_body
        self.trajectory = scene.trajectory
        self.step_index = 0
        if self.grab_body >= 0:
            self.bodies[self.grab_body].grabbed = 1
        self.body_arr = (BodyC * max(1, len(self.bodies)))(*self.bodies)
        self.dims = grid_dims(p)
        self.ncell = int(np.prod(self.dims))

    def _apply_grab(self):
        if self.grab_body >= 0 and self.trajectory is not None:
            s = min(self.step_index, self.trajectory.shape[0] - 1)
            row = self.trajectory[s]
            b = self.body_arr[self.grab_body]
            for a in range(3):
                b.t[a] = row[a]
                b.v[a] = row[7 + a]
                b.w[a] = row[10 + a]
            for a in range(4):
                b.q[a] = row[3 + a]

    def body_state(self, b: int) -> np.ndarray:
        bc = self.body_arr[b]
        return np.array(list(bc.t) + list(bc.q) + list(bc.v) + list(bc.w), np.float32)

    def substep(self, mode: Optional[int] = None) -> dict:
        mode = self.mode if mode is None else mode
        self._apply_grab()
        n, nb = self.n, len(self.bodies)
        out = dict(key=np.zeros(n, np.uint32), src=np.zeros(n, np.int32),
                   cell_start=np.zeros(self.ncell + 1, np.uint32), rho=np.zeros(n),
                   pres=np.zeros(n), nnbr=np.zeros(n, np.int32), acc=np.zeros(n * 3),
                   x_new=np.zeros(n * 3), v_new=np.zeros(n * 3), wrench=np.zeros(max(1, nb) * 6),
                   body_new=np.zeros(max(1, nb) * 13), diag=np.zeros(8), cond=np.zeros(2 * n))
        out["clamped"] = lib().orc_substep(
            ctypes.byref(self.P), n, self.nf, self.x, self.v, self.m, self.id, nb,
            self.body_arr, mode, out["key"], out["src"], out["cell_start"], out["rho"],
            out["pres"], out["nnbr"], out["acc"], out["x_new"], out["v_new"], out["wrench"],
            out["body_new"], out["diag"], out["cond"])
        for k in ("acc", "x_new", "v_new"):
            out[k] = out[k].reshape(n, 3)
        out["cond"] = out["cond"].reshape(n, 2)
        out["wrench"] = out["wrench"].reshape(-1, 6)[:nb]
        out["body_new"] = out["body_new"].reshape(-1, 13)[:nb]
        src = out["src"]
        out["id"] = self.id[src].copy()
        # advance: new FP32 state in the sorted order
        self.x = np.ascontiguousarray(out["x_new"].astype(np.float32))
        self.v = np.ascontiguousarray(out["v_new"].astype(np.float32))
        self.m = np.ascontiguousarray(self.m[src])
        self.id = np.ascontiguousarray(out["id"], np.int32)
        for b in range(nb):
            bc = self.body_arr[b]
            if bc.kind == KIND_RIGID and not bc.grabbed and bc.mass > 0:
                st = out["body_new"][b].astype(np.float32)
                for a in range(3):
                    bc.t[a] = st[a]
                    bc.v[a] = st[7 + a]
                    bc.w[a] = st[10 + a]
                for a in range(4):
                    bc.q[a] = st[3 + a]
        self.step_index += 1
        return out

    def cut_springs(self, tri, margin: float = 1e-5):
        """Incision: cut (k_s = c_d = 0) every active spring whose segment between its
        particles' current positions (lower id first) meets the closed triangle tri, by
        Moller and Trumbore's test in FP64 with the segment parameter in [0, 1] and
        |det| <= 1e-7 |e1|_1 |d x e2|_1 counted as parallel.  Returns (number cut, per body
        the boolean arrays cut and near -- `near`: the decision is within `margin` of one
        of the test's bounds, where FP32 may decide otherwise)."""
        t = np.asarray(tri, np.float64).reshape(3, 3)
        xid = self.by_id(self.x.astype(np.float64))
        total, out = 0, []
        for bi, pairs, ks, cd in self._springs:
            first = self.bodies[bi].first
            ia = first + pairs[:, 0].astype(np.int64)
            ib = first + pairs[:, 1].astype(np.int64)
            lo, hi = np.minimum(ia, ib), np.maximum(ia, ib)
            a, b = xid[lo], xid[hi]
            e1, e2 = t[1] - t[0], t[2] - t[0]
            d = b - a
            pv = np.cross(d, e2)
            det = pv @ e1
            scale = np.abs(e1).sum() * np.abs(pv).sum(1)
            ok = np.abs(det) > 1e-7 * scale
            inv = np.where(ok, 1.0 / np.where(ok, det, 1.0), 0.0)
            tv = a - t[0]
            u = np.einsum("ij,ij->i", tv, pv) * inv
            qv = np.cross(tv, e1)
            v = np.einsum("ij,ij->i", d, qv) * inv
            w = 1.0 - u - v
            sp = (qv @ e2) * inv
            hit = ok & (u >= 0) & (u <= 1) & (v >= 0) & (w >= 0) & (sp >= 0) & (sp <= 1)
            active = ~((ks == 0.0) & (cd == 0.0))
            cut = hit & active
            near = active & ok & (np.minimum.reduce([np.abs(u), np.abs(1 - u), np.abs(v), np.abs(w),
                                                     np.abs(sp), np.abs(1 - sp)]) < margin)
            # the parallel threshold itself: within a factor 1.5 of it either side
            near |= active & (np.abs(det) > 1e-7 / 1.5 * scale) & (np.abs(det) < 1.5e-7 * scale)
            ks[cut] = 0.0
            cd[cut] = 0.0
            total += int(cut.sum())
            out.append((cut, near))
        return total, out

    def by_id(self, arr: np.ndarray) -> np.ndarray:
        """Reorder a per-particle array of the current (sorted) order into id order."""
        out = np.empty_like(arr)
        out[self.id] = arr
        return out
