"""Python binding of the C ABI in ``include/sph.h`` (argument marshalling only).

Every step of the substep runs in ``libsph_gb300.so``; this module loads it with ctypes,
allocates the workspace as one torch uint8 CUDA tensor and passes plain pointers.  There
is no CPU fallback: without the built library or a CUDA device, construction raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import scenes as _scenes

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsph_gb300.so")
# the same library built with -DSPH_CHECKED (index checks; build.build(checked=True))
CHECKED_LIB_PATH = os.path.join(_HERE, "libsph_gb300_checked.so")

OK, ERR_ARG, ERR_CUDA, ERR_WORKSPACE, ERR_CAPACITY, ERR_NONFINITE, ERR_DOMAIN, ERR_TIMEOUT, \
    ERR_STATE, ERR_BOUNDS = range(10)
FLAG_CLAMP_PRESSURE, FLAG_RECORD, FLAG_NO_GRAPH, FLAG_TAIT, FLAG_VOLUME_BOUNDARY = 1, 2, 4, 8, 16
FLAG_LOW_LATENCY = 32
BODY_STATIC, BODY_RIGID, BODY_SOFT = 1, 2, 3

# Every symbol the header declares (checked by the CPU test suite).
SYMBOLS = ["sph_workspace_bytes", "sph_create", "sph_add_rigid", "sph_add_soft",
           "sph_set_grab_pose", "sph_set_grab_path", "sph_step", "sph_get_grab_wrench",
           "sph_get_body_wrench", "sph_get_wrench_log", "sph_get_body", "sph_get_state",
           "sph_set_state", "sph_get_sort", "sph_get_diag", "sph_get_info", "sph_sync",
           "sph_last_error", "sph_destroy", "sph_set_profiling", "sph_get_kernel_times",
           "sph_batch_workspace_bytes", "sph_batch_create", "sph_batch_configure", "sph_batch_tune",
           "sph_batch_step", "sph_batch_sync", "sph_batch_info", "sph_batch_last_error",
           "sph_batch_destroy", "sph_batch_test_barrier", "sph_get_descriptor",
           "sph_mlp_param_count", "sph_mlp_workspace_bytes", "sph_mlp_create", "sph_mlp_set_params",
           "sph_mlp_get_params", "sph_mlp_forward", "sph_mlp_gradients", "sph_mlp_train_step",
           "sph_mlp_sync", "sph_mlp_last_error", "sph_mlp_destroy", "sph_cell_sort_noalloc",
           "sph_iso_grid", "sph_iso_field", "sph_iso_workspace_bytes", "sph_iso_polygonize",
           "sph_set_anchors", "sph_cut_springs", "sph_checkpoint_bytes", "sph_checkpoint_save",
           "sph_checkpoint_load", "sph_haptic_cycle", "sph_measure_fp32_fma",
           "sph_surrogate_set_scene", "sph_surrogate_anchor", "sph_surrogate_tick",
           "sph_surrogate_features", "sph_surrogate_targets"]
KERNELS = ["hash", "scan_tiles", "scan_apply", "scatter", "rank_gather", "density", "force",
           "wrench"]


class SphError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"sph status {status}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("h", ctypes.c_float), ("rho0", ctypes.c_float), ("k", ctypes.c_float),
                ("nu", ctypes.c_float), ("g", ctypes.c_float * 3), ("dt", ctypes.c_float),
                ("domain_lo", ctypes.c_float * 3), ("domain_hi", ctypes.c_float * 3),
                ("cell", ctypes.c_float), ("visc_eps", ctypes.c_float),
                ("spring_zeta", ctypes.c_float), ("fluid_spacing", ctypes.c_float),
                ("flags", ctypes.c_uint32), ("smooth_window", ctypes.c_int32)]


class Capacity(ctypes.Structure):
    _fields_ = [("max_particles", ctypes.c_int32), ("max_bodies", ctypes.c_int32),
                ("max_springs", ctypes.c_int32), ("max_path", ctypes.c_int32),
                ("max_neighbours", ctypes.c_int32)]


_libs = {}
_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p


def load(path: str = LIB_PATH):
    """Load the sm_103a library; raises if it has not been built."""
    path = os.path.abspath(path)
    if path in _libs:
        return _libs[path]
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2511_15908_gb300.build.build()")
    L = ctypes.CDLL(path)
    st = ctypes.c_int
    L.sph_workspace_bytes.restype = ctypes.c_size_t
    L.sph_workspace_bytes.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Capacity)]
    L.sph_create.restype = st
    L.sph_create.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Capacity), _vp, ctypes.c_size_t,
                             _vp, ctypes.c_int32, _f32p, _f32p, ctypes.POINTER(_vp)]
    L.sph_add_rigid.restype = st
    L.sph_add_rigid.argtypes = [_vp, ctypes.c_int32, _f32p, ctypes.c_float, ctypes.c_float, _f32p,
                                _f32p, _f32p, _i32p]
    L.sph_add_soft.restype = st
    L.sph_add_soft.argtypes = [_vp, ctypes.c_int32, _f32p, ctypes.c_float, ctypes.c_int32, _i32p,
                               ctypes.c_float, ctypes.c_float, _i32p]
    L.sph_set_grab_pose.restype = st
    L.sph_set_grab_pose.argtypes = [_vp, ctypes.c_int32, _f32p, _f32p, _f32p]
    L.sph_set_grab_path.restype = st
    L.sph_set_grab_path.argtypes = [_vp, ctypes.c_int32, _f32p]
    L.sph_step.restype = st
    L.sph_step.argtypes = [_vp, ctypes.c_int32]
    L.sph_get_grab_wrench.restype = st
    L.sph_get_grab_wrench.argtypes = [_vp, _f64p, ctypes.c_int32]
    L.sph_get_body_wrench.restype = st
    L.sph_get_body_wrench.argtypes = [_vp, ctypes.c_int32, _f64p]
    L.sph_get_wrench_log.restype = st
    L.sph_get_wrench_log.argtypes = [_vp, ctypes.c_int32, _f64p]
    L.sph_get_body.restype = st
    L.sph_get_body.argtypes = [_vp, ctypes.c_int32, _f32p]
    L.sph_get_state.restype = st
    L.sph_get_state.argtypes = [_vp, _f32p, _f32p, _f32p, _i32p, _f32p]
    L.sph_set_state.restype = st
    L.sph_set_state.argtypes = [_vp, _f32p, _f32p]
    L.sph_get_sort.restype = st
    L.sph_get_sort.argtypes = [_vp, _u32p, _i32p, _u32p]
    L.sph_get_diag.restype = st
    L.sph_get_diag.argtypes = [_vp, _f64p]
    L.sph_get_info.restype = st
    L.sph_get_info.argtypes = [_vp, _i64p]
    L.sph_set_profiling.restype = st
    L.sph_set_profiling.argtypes = [_vp, ctypes.c_int32]
    L.sph_get_kernel_times.restype = st
    L.sph_get_kernel_times.argtypes = [_vp, _f32p]
    L.sph_batch_workspace_bytes.restype = ctypes.c_size_t
    L.sph_batch_workspace_bytes.argtypes = [ctypes.c_int32]
    L.sph_batch_create.restype = st
    L.sph_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32, _vp, ctypes.c_size_t, _vp,
                                   ctypes.POINTER(_vp)]
    L.sph_batch_configure.restype = st
    L.sph_batch_configure.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32]
    L.sph_batch_tune.restype = st
    L.sph_batch_tune.argtypes = [_vp, ctypes.c_int32, _i32p]
    L.sph_batch_step.restype = st
    L.sph_batch_step.argtypes = [_vp, ctypes.c_int32]
    L.sph_batch_sync.restype = st
    L.sph_batch_sync.argtypes = [_vp]
    L.sph_batch_info.restype = st
    L.sph_batch_info.argtypes = [_vp, _i32p]
    L.sph_batch_test_barrier.restype = st
    L.sph_batch_test_barrier.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32]
    L.sph_batch_last_error.restype = ctypes.c_char_p
    L.sph_batch_last_error.argtypes = [_vp]
    L.sph_batch_destroy.restype = None
    L.sph_batch_destroy.argtypes = [_vp]
    L.sph_get_descriptor.restype = st
    L.sph_get_descriptor.argtypes = [_vp, _vp]
    L.sph_mlp_param_count.restype = ctypes.c_int32
    L.sph_mlp_param_count.argtypes = []
    L.sph_mlp_workspace_bytes.restype = ctypes.c_size_t
    L.sph_mlp_workspace_bytes.argtypes = [ctypes.c_int32]
    L.sph_mlp_create.restype = st
    L.sph_mlp_create.argtypes = [_vp, ctypes.c_size_t, _vp, ctypes.c_int32, ctypes.POINTER(_vp)]
    L.sph_mlp_set_params.restype = st
    L.sph_mlp_set_params.argtypes = [_vp, _f32p, _f32p]
    L.sph_mlp_get_params.restype = st
    L.sph_mlp_get_params.argtypes = [_vp, _f32p]
    L.sph_mlp_forward.restype = st
    L.sph_mlp_forward.argtypes = [_vp, _vp, ctypes.c_int32, _vp]
    L.sph_mlp_gradients.restype = st
    L.sph_mlp_gradients.argtypes = [_vp, _vp, _vp, ctypes.c_int32, _f32p, _f64p]
    L.sph_mlp_train_step.restype = st
    L.sph_mlp_train_step.argtypes = [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_float, _f64p]
    L.sph_mlp_sync.restype = st
    L.sph_mlp_sync.argtypes = [_vp]
    L.sph_mlp_last_error.restype = ctypes.c_char_p
    L.sph_mlp_last_error.argtypes = [_vp]
    L.sph_mlp_destroy.restype = None
    L.sph_mlp_destroy.argtypes = [_vp]
    L.sph_cell_sort_noalloc.restype = st
    L.sph_cell_sort_noalloc.argtypes = [ctypes.POINTER(Params), _vp, ctypes.c_int32, _vp, _vp, _vp, _vp]
    L.sph_surrogate_set_scene.restype = st
    L.sph_surrogate_set_scene.argtypes = [_vp, ctypes.POINTER(Params)]
    L.sph_surrogate_anchor.restype = st
    L.sph_surrogate_anchor.argtypes = [_vp, _vp]
    L.sph_surrogate_tick.restype = st
    L.sph_surrogate_tick.argtypes = [_vp, _f32p, ctypes.c_float, _f64p]
    L.sph_surrogate_features.restype = st
    L.sph_surrogate_features.argtypes = [_vp, _vp, ctypes.c_int32, _vp, ctypes.c_int32, _vp, ctypes.c_int32, _vp]
    L.sph_surrogate_targets.restype = st
    L.sph_surrogate_targets.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp]
    L.sph_measure_fp32_fma.restype = st
    L.sph_measure_fp32_fma.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp,
                                       ctypes.POINTER(ctypes.c_double)]
    L.sph_haptic_cycle.restype = st
    L.sph_haptic_cycle.argtypes = [_vp, ctypes.c_int32, _f32p, _f32p, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.POINTER(ctypes.c_double)]
    L.sph_checkpoint_bytes.restype = ctypes.c_size_t
    L.sph_checkpoint_bytes.argtypes = [_vp]
    L.sph_checkpoint_save.restype = st
    L.sph_checkpoint_save.argtypes = [_vp, _vp, ctypes.c_size_t]
    L.sph_checkpoint_load.restype = st
    L.sph_checkpoint_load.argtypes = [_vp, _vp, ctypes.c_size_t]
    L.sph_set_anchors.restype = st
    L.sph_set_anchors.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _i32p]
    L.sph_cut_springs.restype = st
    L.sph_cut_springs.argtypes = [_vp, _f32p, _i64p]
    L.sph_iso_grid.restype = st
    L.sph_iso_grid.argtypes = [ctypes.POINTER(Params), ctypes.c_float, _i32p, _f32p]
    L.sph_iso_field.restype = st
    L.sph_iso_field.argtypes = [_vp, ctypes.c_float, _vp]
    L.sph_iso_workspace_bytes.restype = ctypes.c_size_t
    L.sph_iso_workspace_bytes.argtypes = [_i32p]
    L.sph_iso_polygonize.restype = st
    L.sph_iso_polygonize.argtypes = [_vp, _i32p, _f32p, ctypes.c_float, ctypes.c_float, _vp,
                                     ctypes.c_size_t, _vp, ctypes.c_int64, _i64p, _vp]
    L.sph_sync.restype = st
    L.sph_sync.argtypes = [_vp]
    L.sph_last_error.restype = ctypes.c_char_p
    L.sph_last_error.argtypes = [_vp]
    L.sph_destroy.restype = None
    L.sph_destroy.argtypes = [_vp]
    _libs[path] = L
    return L


def _ptr(a: Optional[np.ndarray], ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def make_params(p: dict, fluid_spacing: float, flags: Optional[int] = None) -> Params:
    P = Params()
    P.h, P.rho0, P.k, P.nu = p["h"], p["rho0"], p["k"], p["nu"]
    for a in range(3):
        P.g[a] = p["g"][a]
        P.domain_lo[a] = p["lo"][a]
        P.domain_hi[a] = p["hi"][a]
    P.dt, P.cell = p["dt"], p["cell"]
    P.visc_eps, P.spring_zeta = p["visc_eps"], p["spring_zeta"]
    P.fluid_spacing = fluid_spacing
    P.flags = int(p["flags"] if flags is None else flags)
    P.smooth_window = int(p.get("smooth_window", 20))
    return P


class Simulation:
    """One scene on one GPU behind the C ABI.  The workspace is a torch CUDA tensor."""

    def __init__(self, scene: _scenes.Scene, flags: Optional[int] = None, max_path: Optional[int] = None,
                 device: int = 0, stream=None, max_neighbours: int = 0, lib: Optional[str] = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the SPH library needs a CUDA device")
        self.L = load(lib or LIB_PATH)
        self.scene = scene
        self.device = torch.device("cuda", device)
        self.params = make_params(scene.params, scene.fluid_spacing, flags)
        n_springs = sum(0 if b.springs is None else int(b.springs.shape[0]) for b in scene.bodies)
        traj_n = 0 if scene.trajectory is None else int(scene.trajectory.shape[0])
        self.cap = Capacity(scene.n_total, max(1, len(scene.bodies)), n_springs,
                            max_path if max_path is not None else max(traj_n, 4096),
                            int(max_neighbours))
        nbytes = self.L.sph_workspace_bytes(ctypes.byref(self.params), ctypes.byref(self.cap))
        if nbytes == 0:
            raise SphError(ERR_ARG, "invalid parameters or capacities")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        x = np.ascontiguousarray(scene.fluid_x, np.float32)
        v = np.ascontiguousarray(scene.fluid_v, np.float32)
        h = _vp()
        st = self.L.sph_create(ctypes.byref(self.params), ctypes.byref(self.cap),
                               self.workspace.data_ptr(), nbytes, self.stream.cuda_stream,
                               x.shape[0], _ptr(x, ctypes.c_float), _ptr(v, ctypes.c_float),
                               ctypes.byref(h))
        if st != OK:
            raise SphError(st, "sph_create failed")
        self.h = h
        self.body_ids = []
        for b in scene.bodies:
            bid = ctypes.c_int32()
            xyz = np.ascontiguousarray(b.xyz, np.float32)
            if b.kind == _scenes.KIND_SOFT:
                pairs = np.ascontiguousarray(b.springs, np.int32)
                self._check(self.L.sph_add_soft(self.h, b.n, _ptr(xyz, ctypes.c_float), b.spacing,
                                                pairs.shape[0], _ptr(pairs, ctypes.c_int32),
                                                b.young, b.poisson, ctypes.byref(bid)))
                if b.anchors is not None and len(b.anchors):
                    anc = np.ascontiguousarray(b.anchors, np.int32)
                    self._check(self.L.sph_set_anchors(self.h, bid.value, anc.shape[0],
                                                       _ptr(anc, ctypes.c_int32)))
            else:
                mass = b.mass if b.kind == _scenes.KIND_RIGID else 0.0
                inertia = np.ascontiguousarray(b.inertia, np.float32).reshape(9)
                pose = np.ascontiguousarray(b.pose, np.float32)
                vel = np.ascontiguousarray(b.vel, np.float32)
                self._check(self.L.sph_add_rigid(self.h, b.n, _ptr(xyz, ctypes.c_float), b.spacing,
                                                 mass, _ptr(inertia, ctypes.c_float),
                                                 _ptr(pose, ctypes.c_float), _ptr(vel, ctypes.c_float),
                                                 ctypes.byref(bid)))
            self.body_ids.append(bid.value)
        if scene.grab_body >= 0:
            gl = np.ascontiguousarray(scene.bodies[scene.grab_body].grab_local, np.float32)
            traj = scene.trajectory
            pose = np.ascontiguousarray(traj[0, :7] if traj is not None else scene.bodies[scene.grab_body].pose,
                                        np.float32)
            vel = np.ascontiguousarray(traj[0, 7:] if traj is not None else np.zeros(6), np.float32)
            self._check(self.L.sph_set_grab_pose(self.h, self.body_ids[scene.grab_body],
                                                 _ptr(pose, ctypes.c_float), _ptr(vel, ctypes.c_float),
                                                 _ptr(gl, ctypes.c_float)))
            if traj is not None:
                t = np.ascontiguousarray(traj[: self.cap.max_path], np.float32)
                self._check(self.L.sph_set_grab_path(self.h, t.shape[0], _ptr(t, ctypes.c_float)))

    # -- helpers
    def _check(self, st):
        if st != OK:
            msg = self.L.sph_last_error(self.h).decode() if getattr(self, "h", None) else ""
            raise SphError(st, msg)

    @property
    def n(self) -> int:
        return self.info()[0]

    def info(self):
        out = np.zeros(5, np.int64)
        self._check(self.L.sph_get_info(self.h, _ptr(out, ctypes.c_int64)))
        return out

    # -- the calls a user makes
    def step(self, n: int = 1):
        self._check(self.L.sph_step(self.h, int(n)))

    def sync(self):
        self._check(self.L.sph_sync(self.h))

    def grab_wrench(self, smoothed: bool = False) -> np.ndarray:
        out = np.zeros(6, np.float64)
        self._check(self.L.sph_get_grab_wrench(self.h, _ptr(out, ctypes.c_double), int(smoothed)))
        return out

    def body_wrench(self, b: int) -> np.ndarray:
        out = np.zeros(6, np.float64)
        self._check(self.L.sph_get_body_wrench(self.h, b, _ptr(out, ctypes.c_double)))
        return out

    def wrench_log(self, n: int) -> np.ndarray:
        out = np.zeros((n, 6), np.float64)
        self._check(self.L.sph_get_wrench_log(self.h, n, _ptr(out, ctypes.c_double)))
        return out

    def set_grab_pose(self, body: int, pose, vel=None, grab_local=None):
        pose = None if pose is None else np.ascontiguousarray(pose, np.float32)
        vel = None if vel is None else np.ascontiguousarray(vel, np.float32)
        gl = None if grab_local is None else np.ascontiguousarray(grab_local, np.float32)
        self._check(self.L.sph_set_grab_pose(self.h, body, _ptr(pose, ctypes.c_float),
                                             _ptr(vel, ctypes.c_float), _ptr(gl, ctypes.c_float)))

    def haptic_cycle(self, body: int, pose, vel, n_substeps: int = 1, smoothed: bool = False,
                     out: Optional[np.ndarray] = None) -> np.ndarray:
        """Set the grabbed body's pose and velocity, step, and read its wrench, in one call
        (sph_haptic_cycle).  pose: 7 float32 (x, q wxyz), vel: 6 float32; `out` (6 float64)
        may be given to avoid an allocation."""
        pose = np.ascontiguousarray(pose, np.float32)
        vel = np.ascontiguousarray(vel, np.float32)
        if out is None:
            out = np.zeros(6, np.float64)
        self._check(self.L.sph_haptic_cycle(self.h, body, _ptr(pose, ctypes.c_float), _ptr(vel, ctypes.c_float),
                                            int(n_substeps), int(smoothed), _ptr(out, ctypes.c_double)))
        return out

    def set_grab_path(self, path):
        path = np.ascontiguousarray(path, np.float32).reshape(-1, 13)
        self._check(self.L.sph_set_grab_path(self.h, path.shape[0], _ptr(path, ctypes.c_float)))

    def body(self, b: int) -> np.ndarray:
        out = np.zeros(13, np.float32)
        self._check(self.L.sph_get_body(self.h, b, _ptr(out, ctypes.c_float)))
        return out

    def state(self, record: bool = False):
        n = self.n
        x = np.zeros((n, 3), np.float32)
        v = np.zeros((n, 3), np.float32)
        rho = np.zeros(n, np.float32)
        nn = np.zeros(n, np.int32) if record else None
        acc = np.zeros((n, 3), np.float32) if record else None
        self._check(self.L.sph_get_state(self.h, _ptr(x, ctypes.c_float), _ptr(v, ctypes.c_float),
                                         _ptr(rho, ctypes.c_float), _ptr(nn, ctypes.c_int32),
                                         _ptr(acc, ctypes.c_float)))
        return dict(x=x, v=v, rho=rho, nnbr=nn, acc=acc)

    def set_state(self, x=None, v=None):
        x = None if x is None else np.ascontiguousarray(x, np.float32)
        v = None if v is None else np.ascontiguousarray(v, np.float32)
        self._check(self.L.sph_set_state(self.h, _ptr(x, ctypes.c_float), _ptr(v, ctypes.c_float)))

    def sort(self):
        n = self.n
        ncell = int(self.info()[2])
        keys = np.zeros(n, np.uint32)
        ids = np.zeros(n, np.int32)
        cs = np.zeros(ncell + 1, np.uint32)
        self._check(self.L.sph_get_sort(self.h, _ptr(keys, ctypes.c_uint32), _ptr(ids, ctypes.c_int32),
                                        _ptr(cs, ctypes.c_uint32)))
        return keys, ids, cs

    def diag(self) -> np.ndarray:
        out = np.zeros(8, np.float64)
        self._check(self.L.sph_get_diag(self.h, _ptr(out, ctypes.c_double)))
        return out

    def descriptor_into(self, d_out) -> None:
        """Write the 269 surrogate inputs of the last substep into a CUDA float tensor."""
        self._check(self.L.sph_get_descriptor(self.h, d_out.data_ptr()))

    def checkpoint(self) -> np.ndarray:
        """Everything that carries over between substeps, as a uint8 array (sph_checkpoint_save)."""
        n = self.L.sph_checkpoint_bytes(self.h)
        if n == 0:
            raise SphError(ERR_ARG, "sph_checkpoint_bytes failed")
        buf = np.zeros(n, np.uint8)
        self._check(self.L.sph_checkpoint_save(self.h, buf.ctypes.data, n))
        return buf

    def restore(self, buf: np.ndarray) -> None:
        """Continue from a checkpoint of the same scene (sph_checkpoint_load)."""
        b = np.ascontiguousarray(buf, np.uint8)
        self._check(self.L.sph_checkpoint_load(self.h, b.ctypes.data, b.size))

    def save_checkpoint(self, path: str) -> None:
        np.savez(path, checkpoint=self.checkpoint())

    def load_checkpoint(self, path: str) -> None:
        with np.load(path) as f:
            self.restore(f["checkpoint"])

    def cut_springs(self, tri) -> int:
        """Cut every soft-body spring whose segment meets the triangle tri (3 x 3 corners);
        returns how many were cut."""
        t = np.ascontiguousarray(np.asarray(tri, np.float32).reshape(9))
        n = np.zeros(1, np.int64)
        self._check(self.L.sph_cut_springs(self.h, _ptr(t, ctypes.c_float), _ptr(n, ctypes.c_int64)))
        return int(n[0])

    def iso_field(self, cube: float):
        """Fluid density field at the corners of the isosurface grid of edge `cube`
        (CUDA float tensor (nz, ny, nx)); see iso_grid for the corner positions."""
        import torch
        dims, _ = iso_grid(self.scene.params, cube)
        f = torch.empty((dims[2], dims[1], dims[0]), dtype=torch.float32, device=self.device)
        self._check(self.L.sph_iso_field(self.h, ctypes.c_float(cube), f.data_ptr()))
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        f.record_stream(self.stream)
        return f

    def isosurface(self, cube: float, iso: float, max_tris: int = 1 << 20):
        """Triangles (n, 3, 3) of the fluid surface phi = iso on the grid of edge `cube`."""
        dims, origin = iso_grid(self.scene.params, cube)
        return iso_polygonize(self.iso_field(cube), dims, origin, cube, iso, max_tris)

    def descriptor(self) -> np.ndarray:
        import torch
        d = torch.empty(269, dtype=torch.float32, device=self.device)
        self.descriptor_into(d)
        self.stream.synchronize()
        return d.cpu().numpy()

    def set_profiling(self, on=True):
        """on: False / 0 off, True / 1 events around every kernel, 2 around the density
        pass only."""
        self._check(self.L.sph_set_profiling(self.h, int(on)))

    def kernel_times(self) -> np.ndarray:
        out = np.zeros(8, np.float32)
        self._check(self.L.sph_get_kernel_times(self.h, _ptr(out, ctypes.c_float)))
        return out

    def close(self):
        if getattr(self, "h", None):
            self.L.sph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many Simulations advanced by one persistent launch per substep (batched form)."""

    def __init__(self, sims, stream=None):
        import torch
        self.sims = list(sims)
        # the scenes' handles belong to the library that made them
        self.L = self.sims[0].L if self.sims else load()
        if any(sm.L is not self.L for sm in self.sims):
            raise SphError(ERR_ARG, "scenes of a batch must come from one library")
        n = len(self.sims)
        nbytes = self.L.sph_batch_workspace_bytes(n)
        if nbytes == 0:
            raise SphError(ERR_ARG, "empty batch")
        dev = self.sims[0].device
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        handles = (_vp * n)(*[s.h for s in self.sims])
        b = _vp()
        st = self.L.sph_batch_create(handles, n, self.workspace.data_ptr(), nbytes,
                                     self.stream.cuda_stream, ctypes.byref(b))
        if st != OK:
            raise SphError(st, "sph_batch_create failed")
        self.b = b

    def _check(self, st):
        if st != OK:
            raise SphError(st, self.L.sph_batch_last_error(self.b).decode())

    def configure(self, blocks_per_sm: int, tiles_per_fetch: int = 1):
        self._check(self.L.sph_batch_configure(self.b, blocks_per_sm, tiles_per_fetch))

    def tune(self, substeps_per_trial: int = 2):
        out = np.zeros(2, np.int32)
        self._check(self.L.sph_batch_tune(self.b, substeps_per_trial, _ptr(out, ctypes.c_int32)))
        return int(out[0]), int(out[1])

    def step(self, n: int = 1):
        self._check(self.L.sph_batch_step(self.b, int(n)))

    def sync(self):
        self._check(self.L.sph_batch_sync(self.b))

    def info(self):
        out = np.zeros(4, np.int32)
        self._check(self.L.sph_batch_info(self.b, _ptr(out, ctypes.c_int32)))
        return dict(scenes=int(out[0]), sms=int(out[1]), blocks_per_sm=int(out[2]),
                    tiles_per_fetch=int(out[3]))

    def test_barrier(self, missing_blocks: int = 1, spin_limit: int = 4096):
        self._check(self.L.sph_batch_test_barrier(self.b, missing_blocks, spin_limit))

    def close(self):
        if getattr(self, "b", None):
            self.L.sph_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surrogate:
    """The 269-128-128-128-6 BF16 tensor-core MLP behind the sph_mlp_* calls."""

    N_IN, N_OUT = 269, 6

    def __init__(self, max_batch: int = 4096, stream=None, device: int = 0):
        import torch
        self.L = load()
        self.max_batch = max_batch
        self.device = torch.device("cuda", device)
        nbytes = self.L.sph_mlp_workspace_bytes(max_batch)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        m = _vp()
        st = self.L.sph_mlp_create(self.workspace.data_ptr(), nbytes, self.stream.cuda_stream, max_batch,
                                   ctypes.byref(m))
        if st != OK:
            raise SphError(st, "sph_mlp_create failed")
        self.m = m
        self.n_params = int(self.L.sph_mlp_param_count())

    def _check(self, st):
        if st != OK:
            raise SphError(st, self.L.sph_mlp_last_error(self.m).decode())

    def set_params(self, params, norm=None):
        params = np.ascontiguousarray(params, np.float32)
        assert params.size == self.n_params
        norm = None if norm is None else np.ascontiguousarray(norm, np.float32)
        self._check(self.L.sph_mlp_set_params(self.m, _ptr(params, ctypes.c_float), _ptr(norm, ctypes.c_float)))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        self._check(self.L.sph_mlp_get_params(self.m, _ptr(out, ctypes.c_float)))
        return out

    def _enter(self):
        # the model's stream waits for work already queued on torch's current stream
        import torch
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)
        return cur

    def _leave(self, cur):
        if cur != self.stream:
            cur.wait_stream(self.stream)

    def forward(self, x_dev, y_dev=None):
        """x_dev: CUDA float32 tensor (B, 269); returns a (B, 6) CUDA tensor."""
        import torch
        B = int(x_dev.shape[0])
        x_dev = x_dev.contiguous()
        if y_dev is None:
            y_dev = torch.empty((B, 6), dtype=torch.float32, device=self.device)
        cur = self._enter()
        self._check(self.L.sph_mlp_forward(self.m, x_dev.data_ptr(), B, y_dev.data_ptr()))
        self._leave(cur)
        return y_dev

    def gradients(self, x_dev, t_dev):
        g = np.zeros(self.n_params, np.float32)
        loss = np.zeros(1, np.float64)
        x_dev, t_dev = x_dev.contiguous(), t_dev.contiguous()
        self._enter()
        self._check(self.L.sph_mlp_gradients(self.m, x_dev.data_ptr(), t_dev.data_ptr(), int(x_dev.shape[0]),
                                             _ptr(g, ctypes.c_float), _ptr(loss, ctypes.c_double)))
        return g, float(loss[0])

    def train_step(self, x_dev, t_dev, lr: float, want_loss: bool = False):
        loss = np.zeros(1, np.float64) if want_loss else None
        x_dev, t_dev = x_dev.contiguous(), t_dev.contiguous()
        cur = self._enter()
        self._check(self.L.sph_mlp_train_step(self.m, x_dev.data_ptr(), t_dev.data_ptr(), int(x_dev.shape[0]),
                                              float(lr), _ptr(loss, ctypes.c_double)))
        # the inputs must stay alive until the model's stream has consumed them
        x_dev.record_stream(self.stream)
        t_dev.record_stream(self.stream)
        self._leave(cur)
        return float(loss[0]) if want_loss else None

    def sync(self):
        self._check(self.L.sph_mlp_sync(self.m))

    # -- the haptic tick (sph_surrogate_*)
    def _keep_scales(self, params: dict):
        # the FP32 scales the library computes (h, c = sqrt(k), rho0), for the caller's records
        self._scales = {"h": float(np.float32(params["h"])),
                        "c": float(np.sqrt(np.float32(params["k"]), dtype=np.float32)),
                        "rho0": float(np.float32(params["rho0"]))}

    def set_scene(self, params: dict):
        P = make_params(params, 1.0)
        self._check(self.L.sph_surrogate_set_scene(self.m, ctypes.byref(P)))
        self._keep_scales(params)

    def scales(self) -> dict:
        return dict(self._scales)

    def anchor(self, sim: "Simulation"):
        """The last substep of `sim` becomes the start of an update cycle."""
        self._check(self.L.sph_surrogate_anchor(sim.h, self.m))
        self._keep_scales(sim.scene.params)

    def tick(self, pose_vel, elapsed: float, out=None) -> np.ndarray:
        """Wrench at a haptic tick: anchor wrench + predicted change (host, 6 doubles)."""
        pv = np.ascontiguousarray(pose_vel, np.float32)
        out = np.zeros(6, np.float64) if out is None else out
        self._check(self.L.sph_surrogate_tick(self.m, _ptr(pv, ctypes.c_float), float(elapsed),
                                              _ptr(out, ctypes.c_double)))
        return out

    def features(self, ticks_dev, anchors_dev, elapsed_dev):
        """Scale-free inputs of n (tick, anchor) pairs: ticks (n, >= 13), anchors (n, >= 269)
        and elapsed (n) CUDA float tensors; returns (n, 269)."""
        import torch
        n = int(ticks_dev.shape[0])
        out = torch.empty((max(n, 1), 269), dtype=torch.float32, device=self.device)
        ticks_dev, anchors_dev, elapsed_dev = ticks_dev.contiguous(), anchors_dev.contiguous(), elapsed_dev.contiguous()
        cur = self._enter()
        self._check(self.L.sph_surrogate_features(self.m, ticks_dev.data_ptr(), int(ticks_dev.shape[1]),
                                                  anchors_dev.data_ptr(), int(anchors_dev.shape[1]),
                                                  elapsed_dev.data_ptr(), n, out.data_ptr()))
        for t in (ticks_dev, anchors_dev, elapsed_dev):
            t.record_stream(self.stream)
        self._leave(cur)
        return out[:n]

    def targets(self, wrench_dev, anchor_wrench_dev, anchors_dev):
        """Training targets of n pairs: the wrench change since the anchor in the anchor's
        body frame and the scene's force and torque scales; CUDA tensors in, (n, 6) out."""
        import torch
        n = int(wrench_dev.shape[0])
        out = torch.empty((max(n, 1), 6), dtype=torch.float32, device=self.device)
        wrench_dev, anchor_wrench_dev, anchors_dev = (wrench_dev.contiguous(), anchor_wrench_dev.contiguous(),
                                                      anchors_dev.contiguous())
        cur = self._enter()
        self._check(self.L.sph_surrogate_targets(self.m, wrench_dev.data_ptr(), anchor_wrench_dev.data_ptr(),
                                                 anchors_dev.data_ptr(), int(anchors_dev.shape[1]), n,
                                                 out.data_ptr()))
        for t in (wrench_dev, anchor_wrench_dev, anchors_dev):
            t.record_stream(self.stream)
        self._leave(cur)
        return out[:n]

    def close(self):
        if getattr(self, "m", None):
            self.L.sph_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NOALLOC_MAX_PARTICLES = 1 << 18
NOALLOC_MAX_CELLS = 1 << 18


def cell_sort_noalloc(params: dict, x_dev, stream=None, out=None):
    """Allocation-free spatial hash of the particles in x_dev (CUDA float32 tensor (n, 4)):
    returns (keys, order, cell_start) CUDA tensors.  The output tensors are the caller's:
    `out` = (keys[n], order[n], cell_start[cells + 1]) int32 tensors, or allocated here by
    torch when None; the library call itself allocates nothing."""
    import torch
    L = load()
    P = make_params(params, 1.0)
    n = int(x_dev.shape[0])
    x_dev = x_dev.contiguous()
    ncell = int(np.prod(grid_dims(params)))
    if n > NOALLOC_MAX_PARTICLES or ncell > NOALLOC_MAX_CELLS:
        # the library refuses these sizes too; refuse before allocating the outputs
        raise SphError(ERR_CAPACITY, "sph_cell_sort_noalloc: beyond the fixed scratch")
    if out is not None:
        keys, order, cs = out
        if keys.numel() < n or order.numel() < n or cs.numel() < ncell + 1:
            raise ValueError("output tensors too small")
    else:
        keys = torch.empty(max(n, 1), dtype=torch.int32, device=x_dev.device)
        order = torch.empty(max(n, 1), dtype=torch.int32, device=x_dev.device)
        cs = torch.empty(ncell + 1, dtype=torch.int32, device=x_dev.device)
    st = stream if stream is not None else torch.cuda.current_stream(x_dev.device)
    r = L.sph_cell_sort_noalloc(ctypes.byref(P), x_dev.data_ptr(), n, keys.data_ptr(), order.data_ptr(),
                                cs.data_ptr(), st.cuda_stream)
    if r != OK:
        raise SphError(r, "sph_cell_sort_noalloc failed")
    return keys[:n], order[:n], cs


def measure_fp32_fma(device=0, iters=65536, reps=5):
    """FP32 FMA throughput of the GPU in TFLOP/s (best of `reps` launches of the library's
    FMA probe kernel at full occupancy, CUDA events on one stream)."""
    import torch
    L = load()
    props = torch.cuda.get_device_properties(device)
    blocks = props.multi_processor_count * (props.max_threads_per_multi_processor // 256)
    sink = torch.zeros(256, dtype=torch.float32, device=f"cuda:{device}")
    s = torch.cuda.Stream(device=device)
    flops = ctypes.c_double(0.0)
    best = None
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        st = L.sph_measure_fp32_fma(ctypes.c_void_p(s.cuda_stream), blocks, iters, ctypes.c_void_p(sink.data_ptr()),
                                    ctypes.byref(flops))
        if st != OK:
            raise SphError(st, "sph_measure_fp32_fma failed")
        e1.record(s)
        e1.synchronize()
        if r > 0:
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
    return flops.value / best / 1e12


def iso_grid(params: dict, cube: float):
    """Corner counts (nx, ny, nz) and corner (0,0,0) of the isosurface grid of edge cube."""
    L = load()
    P = make_params(params, 1.0)
    dims = np.zeros(3, np.int32)
    org = np.zeros(3, np.float32)
    r = L.sph_iso_grid(ctypes.byref(P), ctypes.c_float(cube), _ptr(dims, ctypes.c_int32),
                       _ptr(org, ctypes.c_float))
    if r != OK:
        raise SphError(r, "sph_iso_grid failed")
    return [int(d) for d in dims], org


def iso_polygonize(field_dev, dims, origin, cube: float, iso: float, max_tris: int = 1 << 20,
                   stream=None):
    """Marching cubes over a CUDA float field (nz, ny, nx); returns the triangles as a CUDA
    tensor (n, 3, 3).  Raises SphError(ERR_CAPACITY) when there are more than max_tris."""
    import torch
    L = load()
    field_dev = field_dev.contiguous()
    d = np.asarray(dims, np.int32)
    o = np.asarray(origin, np.float32)
    nbytes = L.sph_iso_workspace_bytes(_ptr(d, ctypes.c_int32))
    if nbytes == 0:
        raise SphError(ERR_ARG, "invalid isosurface grid")
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=field_dev.device)
    off = (-ws.data_ptr()) % 256
    tris = torch.empty((max(max_tris, 1), 3, 3), dtype=torch.float32, device=field_dev.device)
    n = np.zeros(1, np.int64)
    st = stream if stream is not None else torch.cuda.current_stream(field_dev.device)
    r = L.sph_iso_polygonize(field_dev.data_ptr(), _ptr(d, ctypes.c_int32), _ptr(o, ctypes.c_float),
                             ctypes.c_float(cube), ctypes.c_float(iso), ws.data_ptr() + off, nbytes,
                             tris.data_ptr(), int(max_tris), _ptr(n, ctypes.c_int64), st.cuda_stream)
    if r != OK:
        raise SphError(r, f"sph_iso_polygonize failed ({int(n[0])} triangles)")
    return tris[:int(n[0])]


def grid_dims(params: dict):
    """Cells per axis of the uniform grid (same FP32 formula as the library)."""
    cell = np.float32(params["cell"])
    inv = np.float32(1.0) / cell
    out = []
    for a in range(3):
        o = np.float32(np.float32(params["lo"][a]) - cell)
        u = np.float32(np.float32(np.float32(params["hi"][a]) - o) * inv)
        out.append(int(np.floor(u)) + 2)
    return out
