"""Python binding of the surrogate C ABI (include/surrogate.h): marshalling only.

Device arrays are CUDA torch tensors (float32, contiguous); parameter vectors
are host NumPy float32 arrays of SUR_N_PARAMS entries.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import rcell

SUR_N_IN, SUR_N_H, SUR_N_OUT, SUR_WIDTH = 15, 128, 6, 256
SUR_N_PARAMS = 144 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 144 + 144
EXPORTS = ["sur_create", "sur_set_scaling", "sur_get_params", "sur_set_params", "sur_loss_grad", "sur_train_step",
           "sur_predict", "sur_profile_step", "sur_step", "sur_features", "sur_set_backend", "sur_sync", "sur_info",
           "sur_destroy"]
_bound = False


def _lib():
    global _bound
    L = rcell.load()
    if not _bound:
        vp = C.c_void_p
        sig = {
            "sur_create": ([C.c_int, C.c_int, C.c_int, C.c_uint64, vp, C.POINTER(vp)], C.c_int),
            "sur_set_scaling": ([vp, vp, vp], C.c_int),
            "sur_get_params": ([vp, C.c_int, vp], C.c_int),
            "sur_set_params": ([vp, C.c_int, vp], C.c_int),
            "sur_loss_grad": ([vp, C.c_int, vp, vp, C.c_int, C.c_int, C.POINTER(C.c_double), vp], C.c_int),
            "sur_train_step": ([vp, vp, vp, C.c_int, C.c_int, C.c_float, C.c_float, vp], C.c_int),
            "sur_predict": ([vp, vp, C.c_int, C.c_int, vp], C.c_int),
            "sur_profile_step": ([vp, vp, vp, C.c_int, C.c_int, vp], C.c_int),
            "sur_step": ([vp, vp, C.c_int, vp, C.c_float, vp, vp], C.c_int),
            "sur_features": ([vp, vp, C.c_int, vp, vp], C.c_int),
            "sur_info": ([vp, C.POINTER(C.c_int), C.POINTER(vp)], C.c_int),
            "sur_set_backend": ([vp, C.c_int], C.c_int),
            "sur_sync": ([vp], C.c_int),
            "sur_destroy": ([vp], None),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _bound = True
    return L


def _chk(code, what):
    if code != 0:
        raise rcell.RCellError(code, what)


def _dp(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return C.c_void_p(t.data_ptr())


def sur_create(n_members, max_batch, max_steps, seed=0, stream=None):
    out = C.c_void_p()
    _chk(_lib().sur_create(n_members, max_batch, max_steps, seed, rcell._stream_ptr(stream), C.byref(out)),
         "sur_create")
    return out


def sur_set_scaling(s, u_scale, s_scale):
    u = np.ascontiguousarray(u_scale, dtype=np.float32)
    v = np.ascontiguousarray(s_scale, dtype=np.float32)
    _chk(_lib().sur_set_scaling(s, C.c_void_p(u.ctypes.data), C.c_void_p(v.ctypes.data)), "sur_set_scaling")


def sur_get_params(s, member):
    th = np.zeros(SUR_N_PARAMS, dtype=np.float32)
    _chk(_lib().sur_get_params(s, member, C.c_void_p(th.ctypes.data)), "sur_get_params")
    return th


def sur_set_params(s, member, theta):
    th = np.ascontiguousarray(theta, dtype=np.float32)
    assert th.size == SUR_N_PARAMS
    _chk(_lib().sur_set_params(s, member, C.c_void_p(th.ctypes.data)), "sur_set_params")


def sur_loss_grad(s, member, U, Y):
    B, T = int(U.shape[0]), int(U.shape[1])
    loss = C.c_double(0.0)
    g = np.zeros(SUR_N_PARAMS, dtype=np.float32)
    _chk(_lib().sur_loss_grad(s, member, _dp(U), _dp(Y), B, T, C.byref(loss), C.c_void_p(g.ctypes.data)),
         "sur_loss_grad")
    return loss.value, g


def sur_train_step(s, U, Y, lr, wd=0.01, n_members=1, want_loss=True):
    B, T = int(U.shape[0]), int(U.shape[1])
    loss = np.zeros(n_members)
    _chk(_lib().sur_train_step(s, _dp(U), _dp(Y), B, T, lr, wd, C.c_void_p(loss.ctypes.data) if want_loss else None),
         "sur_train_step")
    return loss if want_loss else None


def sur_predict(s, U, out):
    B, T = int(U.shape[0]), int(U.shape[1])
    _chk(_lib().sur_predict(s, _dp(U), B, T, _dp(out)), "sur_predict")


def sur_profile_step(s, U, Y):
    """Milliseconds of the phases of one training step (not applied): forward
    with the tape, data gradients, weight and bias gradients."""
    B, T = int(U.shape[0]), int(U.shape[1])
    ms = np.zeros(3)
    _chk(_lib().sur_profile_step(s, _dp(U), _dp(Y), B, T, C.c_void_p(ms.ctypes.data)), "sur_profile_step")
    return {"forward_tape": float(ms[0]), "backward": float(ms[1]), "weight_grad": float(ms[2])}


def sur_step(s, u, h, s_floor, s_mean, spread):
    _chk(_lib().sur_step(s, _dp(u), int(u.shape[0]), _dp(h), s_floor, _dp(s_mean), _dp(spread)), "sur_step")


def sur_features(F_prev, F, u, stream=None):
    """F_prev, F: CUDA float64 (n, 3, 3); u: CUDA float32 (n, 15) output."""
    _chk(_lib().sur_features(_dp(F_prev), _dp(F), int(F.shape[0]), _dp(u), rcell._stream_ptr(stream)), "sur_features")


def sur_set_backend(s, backend):
    _chk(_lib().sur_set_backend(s, int(backend)), "sur_set_backend")


def sur_sync(s):
    return _lib().sur_sync(s)


def sur_info(s):
    k = C.c_int(0)
    st = C.c_void_p()
    _chk(_lib().sur_info(s, C.byref(k), C.byref(st)), "sur_info")
    return k.value, st.value


def sur_destroy(s):
    if s:
        _lib().sur_destroy(s)
