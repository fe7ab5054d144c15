"""Host-side validation of the C ABI, called directly: every refusal returns its status code
and leaves the handle usable.  (Capacities, setup after the first substep, grabbing a body
that is not rigid, grab paths with nothing grabbed, bad spring pairs, a bad workspace.)"""
import ctypes

import numpy as np
import pytest

from paper_2511_15908_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_15908_gb300 import build, sph as _sph
    build.build()
    _sph.load()
    return _sph


def _f32(a):
    a = np.ascontiguousarray(a, np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _handle(sph, max_particles, max_bodies=2, max_springs=0, max_path=8, n_fluid=8):
    """A bare handle with n_fluid particles on a small lattice and the given capacities."""
    import torch
    L = sph.load()
    p = sph.make_params(scenes.make_params(0.02, 1e-3, (-0.2, -0.2, -0.2), (0.4, 0.4, 0.4)), 0.02)
    cap = sph.Capacity(max_particles, max_bodies, max_springs, max_path, 0)
    nbytes = L.sph_workspace_bytes(ctypes.byref(p), ctypes.byref(cap))
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    x = (np.stack(np.meshgrid(*[np.arange(2)] * 3, indexing="ij"), -1).reshape(-1, 3) * 0.02 + 0.05)[:n_fluid]
    xs, xp = _f32(x)
    h = ctypes.c_void_p()
    st = L.sph_create(ctypes.byref(p), ctypes.byref(cap), ws.data_ptr(), nbytes, stream.cuda_stream,
                      xs.shape[0], xp, None, ctypes.byref(h))
    assert st == sph.OK
    return L, h, (ws, stream, xs)


def _add_rigid(L, h, n, mass=1.0, at=(0.2, 0.2, 0.2)):
    xyz = np.zeros((n, 3), np.float32)
    xyz[:, 0] = np.arange(n) * 0.01
    xyz, xp = _f32(xyz)
    inertia, ip = _f32(np.eye(3) * 0.01)
    pose, pp = _f32([*at, 1, 0, 0, 0])
    bid = ctypes.c_int32(-7)
    return L.sph_add_rigid(h, n, xp, ctypes.c_float(0.01), ctypes.c_float(mass), ip, pp, None,
                           ctypes.byref(bid)), bid.value, (xyz, inertia, pose)


def test_create_refuses_bad_workspace_and_too_many_particles(sph):
    import torch
    L = sph.load()
    p = sph.make_params(scenes.make_params(0.02, 1e-3, (0, 0, 0), (0.2, 0.2, 0.2)), 0.02)
    cap = sph.Capacity(4, 1, 0, 4, 0)
    nbytes = L.sph_workspace_bytes(ctypes.byref(p), ctypes.byref(cap))
    ws = torch.empty(nbytes + 512, dtype=torch.uint8, device="cuda")
    x, xp = _f32(np.full((8, 3), 0.1))
    h = ctypes.c_void_p()
    s = torch.cuda.current_stream().cuda_stream
    assert L.sph_create(ctypes.byref(p), ctypes.byref(cap), ws.data_ptr(), nbytes, s, 8, xp, None,
                        ctypes.byref(h)) == sph.ERR_CAPACITY
    assert L.sph_create(ctypes.byref(p), ctypes.byref(cap), ws.data_ptr(), nbytes - 1, s, 2, xp, None,
                        ctypes.byref(h)) == sph.ERR_WORKSPACE
    assert L.sph_create(ctypes.byref(p), ctypes.byref(cap), ws.data_ptr() + 16, nbytes, s, 2, xp, None,
                        ctypes.byref(h)) == sph.ERR_WORKSPACE
    assert L.sph_create(ctypes.byref(p), ctypes.byref(cap), ws.data_ptr(), nbytes, s, 2, None, None,
                        ctypes.byref(h)) == sph.ERR_ARG


def test_body_capacities_and_setup_after_the_first_substep(sph):
    L, h, keep = _handle(sph, max_particles=8 + 10, max_bodies=1)
    st, bid, _ = _add_rigid(L, h, 11)                 # 8 + 11 > 18 particles
    assert st == sph.ERR_CAPACITY
    st, bid, _ = _add_rigid(L, h, 10)
    assert st == sph.OK and bid == 0
    st, _, _ = _add_rigid(L, h, 1)                    # a second body: max_bodies = 1
    assert st == sph.ERR_CAPACITY
    st, _, _ = _add_rigid(L, h, 1, mass=-1.0)
    assert st == sph.ERR_ARG
    assert L.sph_step(h, 2) == sph.OK
    assert L.sph_sync(h) == sph.OK
    L.sph_destroy(h)
    L, h, keep = _handle(sph, max_particles=64, max_bodies=4)
    assert L.sph_step(h, 1) == sph.OK
    st, _, _ = _add_rigid(L, h, 4)
    assert st == sph.ERR_STATE
    assert b"before the first step" in L.sph_last_error(h)
    assert L.sph_step(h, 1) == sph.OK and L.sph_sync(h) == sph.OK
    L.sph_destroy(h)


def test_soft_body_spring_checks(sph):
    L, h, keep = _handle(sph, max_particles=64, max_bodies=2, max_springs=2)
    xyz, xp = _f32(np.array([[0.2, 0.2, 0.2], [0.21, 0.2, 0.2], [0.22, 0.2, 0.2]]))
    bid = ctypes.c_int32()

    def add(pairs):
        pr = np.ascontiguousarray(pairs, np.int32)
        return L.sph_add_soft(h, 3, xp, ctypes.c_float(0.01), pr.shape[0],
                              pr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                              ctypes.c_float(5e4), ctypes.c_float(0.3), ctypes.byref(bid))

    assert add([[0, 1], [1, 2], [0, 2]]) == sph.ERR_CAPACITY     # 3 springs > 2
    assert add([[0, 0]]) == sph.ERR_ARG                          # self pair
    assert add([[0, 3]]) == sph.ERR_ARG                          # outside the body
    assert add([[0, 1], [1, 2]]) == sph.OK
    assert L.sph_step(h, 3) == sph.OK and L.sph_sync(h) == sph.OK
    L.sph_destroy(h)


def test_grab_checks(sph):
    L, h, keep = _handle(sph, max_particles=64, max_bodies=3, max_path=4)
    st, rigid, _ = _add_rigid(L, h, 4)
    assert st == sph.OK
    st, static, _ = _add_rigid(L, h, 4, mass=0.0, at=(0.3, 0.3, 0.3))
    assert st == sph.OK
    pose, pp = _f32([0.2, 0.2, 0.2, 1, 0, 0, 0])
    path, tp = _f32(np.tile([0.2, 0.2, 0.2, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0], (5, 1)))
    w = (ctypes.c_double * 6)()
    # nothing grabbed yet
    assert L.sph_set_grab_path(h, 2, tp) == sph.ERR_STATE
    assert L.sph_get_grab_wrench(h, w, 0) == sph.ERR_STATE
    # only rigid bodies can be grabbed; ids must exist
    assert L.sph_set_grab_pose(h, static, pp, None, None) == sph.ERR_ARG
    assert L.sph_set_grab_pose(h, 7, pp, None, None) == sph.ERR_ARG
    assert L.sph_set_grab_pose(h, rigid, pp, None, None) == sph.OK
    assert L.sph_set_grab_path(h, 5, tp) == sph.ERR_ARG           # longer than max_path = 4
    assert L.sph_set_grab_path(h, 4, tp) == sph.OK
    assert L.sph_step(h, 3) == sph.OK
    assert L.sph_get_grab_wrench(h, w, 0) == sph.OK
    assert np.all(np.isfinite(np.frombuffer(w, np.float64)))
    # release: the wrench read is refused again, stepping goes on
    assert L.sph_set_grab_pose(h, -1, None, None, None) == sph.OK
    assert L.sph_get_grab_wrench(h, w, 0) == sph.ERR_STATE
    assert L.sph_step(h, 1) == sph.OK and L.sph_sync(h) == sph.OK
    L.sph_destroy(h)
