"""Python marshalling of the FP64 surrogate oracle (oracle/mlp_oracle.c) -- test infrastructure."""
import ctypes

import numpy as np

_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")


def declare(L):
    L.orc_mlp_param_count.restype = ctypes.c_int
    L.orc_mlp_param_count.argtypes = []
    L.orc_bf16.restype = ctypes.c_float
    L.orc_bf16.argtypes = [ctypes.c_float]
    L.orc_gelu.restype = ctypes.c_double
    L.orc_gelu.argtypes = [ctypes.c_double]
    L.orc_gelu_grad.restype = ctypes.c_double
    L.orc_gelu_grad.argtypes = [ctypes.c_double]
    L.orc_mlp_forward.restype = None
    L.orc_mlp_forward.argtypes = [_f32p, _f32p, _f32p, ctypes.c_int, ctypes.c_int, _f64p]
    L.orc_mlp_grad.restype = ctypes.c_double
    L.orc_mlp_grad.argtypes = [_f32p, _f32p, _f32p, _f32p, ctypes.c_int, ctypes.c_int, _f64p]
    L.orc_descriptor.restype = None
    L.orc_descriptor.argtypes = [ctypes.c_int, _f32p, _f64p, _f64p, _f64p, _i32p, _f64p, _f32p,
                                 ctypes.c_float, _f64p]


def _lib():
    from . import lib
    return lib()


def param_count():
    return _lib().orc_mlp_param_count()


def bf16(x):
    return _lib().orc_bf16(float(x))


def gelu(z):
    return _lib().orc_gelu(float(z))


def gelu_grad(z):
    return _lib().orc_gelu_grad(float(z))


def forward(params, norm, X, bf=True):
    X = np.ascontiguousarray(X, np.float32).reshape(-1, 269)
    Y = np.zeros((X.shape[0], 6))
    _lib().orc_mlp_forward(np.ascontiguousarray(params, np.float32), np.ascontiguousarray(norm, np.float32),
                           X, X.shape[0], int(bf), Y)
    return Y


def grad(params, norm, X, T, bf=True):
    X = np.ascontiguousarray(X, np.float32).reshape(-1, 269)
    T = np.ascontiguousarray(T, np.float32).reshape(-1, 6)
    G = np.zeros(param_count())
    loss = _lib().orc_mlp_grad(np.ascontiguousarray(params, np.float32), np.ascontiguousarray(norm, np.float32),
                               X, T, X.shape[0], int(bf), G)
    return loss, G


def descriptor(x, v, rho, m, is_fluid, xg, pose_vel, h):
    x = np.ascontiguousarray(x, np.float32)
    n = x.shape[0]
    out = np.zeros(269)
    _lib().orc_descriptor(n, x, np.ascontiguousarray(v, np.float64), np.ascontiguousarray(rho, np.float64),
                          np.ascontiguousarray(m, np.float64), np.ascontiguousarray(is_fluid, np.int32),
                          np.ascontiguousarray(xg, np.float64), np.ascontiguousarray(pose_vel, np.float32),
                          float(h), out)
    return out
