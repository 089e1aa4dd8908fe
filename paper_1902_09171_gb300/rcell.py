"""Python binding of the r-cell C ABI (include/rcell.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: it converts NumPy arrays / torch tensors into the
pointers and sizes of the ABI and turns status codes into exceptions.  The
CUDA library must be built (``paper_1902_09171_gb300.build.build()``); there
is no fallback -- importing the binding without the library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

RC_HOST, RC_DEVICE = 0, 1
RC_POT_LJ, RC_POT_SC, RC_POT_KG = 0, 1, 2
RC_UNITS_METAL, RC_UNITS_LJ = 0, 1

STATUS = {0: "RC_OK", 1: "RC_EINVAL", 2: "RC_ENOMEM", 3: "RC_ECUDA", 4: "RC_EDEGEN", 5: "RC_EBOX", 6: "RC_EBOND",
          7: "RC_ELOST", 8: "RC_EOVERFLOW", 9: "RC_ENAN", 10: "RC_ETIMEOUT", 11: "RC_ESTATE"}
CODES = {v: k for k, v in STATUS.items()}


class RCellError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = STATUS.get(code, str(code))


class rcell_params(C.Structure):
    _fields_ = [("potential", C.c_int), ("units", C.c_int), ("eps", C.c_double), ("sigma", C.c_double),
                ("rc", C.c_double), ("n", C.c_double), ("m", C.c_double), ("c", C.c_double),
                ("k_fene", C.c_double), ("R0", C.c_double), ("skin", C.c_double), ("mass", C.c_double),
                ("kT", C.c_double), ("tau", C.c_double), ("dt", C.c_double), ("seed", C.c_uint64),
                ("max_step", C.c_double)]


class rcell_init(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("H0", C.POINTER(C.c_double)), ("x0", C.POINTER(C.c_double)),
                ("v0", C.POINTER(C.c_double)), ("n_bonds", C.c_int), ("bonds", C.POINTER(C.c_int))]


_lib = None
EXPORTS = ["rcell_create", "rcell_set_deformation", "rcell_run", "rcell_stress", "rcell_eval", "rcell_get_energy",
           "rcell_get_atoms", "rcell_get_box", "rcell_get_neighbors", "rcell_get_series", "rcell_sync",
           "rcell_clear_status", "rcell_set_active", "rcell_set_limits", "rcell_set_staging", "rcell_set_tuning", "rcell_minimize", "rcell_stress_static", "rcell_get_rebuilds", "rcell_info", "rcell_profile_kernels", "rcell_fp32_peak", "rcell_checkpoint", "rcell_restore",
           "rcell_stress_reduce_static", "rcell_last_error", "rcell_destroy", "fe_create", "fe_create_tet4", "fe_apply_bc", "fe_set_predictor", "fe_get_F", "fe_update", "fe_step", "fe_step_surrogate", "fe_get_P",
           "fe_get_state", "fe_destroy"]


def load(path: str | None = None):
    """Load librcell.so (built in-tree).  Raises if it is missing: no CPU fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run paper_1902_09171_gb300.build.build())")
    L = C.CDLL(path)
    vp, D, I = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
    sig = {
        "rcell_create": ([C.POINTER(rcell_params), C.c_int, C.POINTER(rcell_init), vp, C.POINTER(vp)], C.c_int),
        "rcell_set_deformation": ([vp, vp, C.c_int], C.c_int),
        "rcell_run": ([vp, C.c_int, C.c_int], C.c_int),
        "rcell_stress": ([vp, vp, vp, vp, C.c_int], C.c_int),
        "rcell_eval": ([vp], C.c_int),
        "rcell_get_energy": ([vp, vp, vp], C.c_int),
        "rcell_get_atoms": ([vp, C.c_int, vp, vp, vp], C.c_int),
        "rcell_get_box": ([vp, C.c_int, vp, vp, vp], C.c_int),
        "rcell_get_neighbors": ([vp, C.c_int, vp, C.c_long, C.POINTER(C.c_long)], C.c_int),
        "rcell_get_series": ([vp, C.c_int, vp, vp, vp], C.c_int),
        "rcell_sync": ([vp], C.c_int),
        "rcell_clear_status": ([vp], C.c_int),
        "rcell_set_active": ([vp, vp, C.c_int], C.c_int),
        "rcell_set_staging": ([vp, C.c_int], C.c_int),
        "rcell_set_limits": ([vp, C.c_int, C.c_int], C.c_int),
        "rcell_set_tuning": ([vp, C.c_int, C.c_int], C.c_int),
        "rcell_info": ([vp, I, C.POINTER(C.c_long), C.POINTER(C.c_long)], C.c_int),
        "rcell_profile_kernels": ([vp, C.c_int, vp], C.c_int),
        "rcell_fp32_peak": ([vp, vp], C.c_int),
        "rcell_get_rebuilds": ([vp, vp], C.c_int),
        "rcell_minimize": ([vp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, vp], C.c_int),
        "rcell_stress_static": ([vp, vp, vp, C.c_int], C.c_int),
        "rcell_checkpoint": ([vp, C.c_int, vp, C.POINTER(C.c_size_t)], C.c_int),
        "rcell_restore": ([vp, C.c_int, vp, C.c_size_t], C.c_int),
        "rcell_stress_reduce_static": ([vp, C.c_int, C.c_int, vp, vp, vp, vp, vp, vp], C.c_int),
        "rcell_last_error": ([vp], C.c_char_p),
        "rcell_destroy": ([vp], None),
        "fe_create": ([vp, C.c_int, vp, C.c_int, vp, vp, C.c_double, C.c_double, C.c_double, C.c_double, vp,
                       C.POINTER(vp)], C.c_int),
        "fe_create_tet4": ([vp, C.c_int, vp, C.c_int, vp, vp, C.c_double, C.c_double, C.c_double, vp,
                            C.POINTER(vp)], C.c_int),
        "fe_apply_bc": ([vp, C.c_double], C.c_int),
        "fe_set_predictor": ([vp, vp], C.c_int),
        "fe_get_F": ([vp, vp, C.c_int], C.c_int),
        "fe_update": ([vp, vp, C.c_int], C.c_int),
        "fe_step": ([vp, vp, C.c_double, C.c_int, C.c_int, vp], C.c_int),
        "fe_step_surrogate": ([vp, vp, vp, C.c_double, C.c_int, C.c_int, C.c_float, C.c_float, C.c_float, C.c_int,
                               vp, vp, vp, vp, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
        "fe_get_P": ([vp, vp, C.c_int], C.c_int),
        "fe_get_state": ([vp, vp, vp], C.c_int),
        "fe_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _arr_ptr(a, dtype=np.float64):
    """(pointer, where, keepalive) for a NumPy array (host) or a torch tensor (host/device)."""
    if a is None:
        return None, RC_HOST, None
    if hasattr(a, "data_ptr"):  # torch tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr()), (RC_DEVICE if a.is_cuda else RC_HOST), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return C.c_void_p(arr.ctypes.data), RC_HOST, arr


def _check(code, ctx=None, what=""):
    if code != 0:
        msg = what
        if ctx is not None:
            msg += ": " + load().rcell_last_error(ctx).decode()
        raise RCellError(code, msg)


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def rcell_create(params: rcell_params, cells, stream=None):
    """cells: list of dicts with H0 (3x3), x0 (n,3), optional v0 (n,3), optional bonds (nb,2)."""
    L = load()
    keep = []
    arr = (rcell_init * len(cells))()
    for k, cdef in enumerate(cells):
        H0 = np.ascontiguousarray(cdef["H0"], dtype=np.float64).reshape(9)
        x0 = np.ascontiguousarray(cdef["x0"], dtype=np.float64).reshape(-1)
        v0 = cdef.get("v0")
        v0 = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float64).reshape(-1)
        b = cdef.get("bonds")
        b = np.zeros(0, np.int32) if b is None else np.ascontiguousarray(b, dtype=np.int32).reshape(-1)
        keep += [H0, x0, v0, b]
        arr[k].n_atoms = x0.size // 3
        arr[k].H0 = H0.ctypes.data_as(C.POINTER(C.c_double))
        arr[k].x0 = x0.ctypes.data_as(C.POINTER(C.c_double))
        arr[k].v0 = v0.ctypes.data_as(C.POINTER(C.c_double)) if v0 is not None else None
        arr[k].n_bonds = b.size // 2
        arr[k].bonds = b.ctypes.data_as(C.POINTER(C.c_int))
    out = C.c_void_p()
    _check(L.rcell_create(C.byref(params), len(cells), arr, _stream_ptr(stream), C.byref(out)), None,
           "rcell_create")
    return out


def rcell_set_deformation(ctx, F):
    p, where, keep = _arr_ptr(F)
    _check(load().rcell_set_deformation(ctx, p, where), ctx, "rcell_set_deformation")


def rcell_run(ctx, n_steps: int, n_avg: int):
    _check(load().rcell_run(ctx, n_steps, n_avg), ctx, "rcell_run")


def rcell_stress(ctx, sigma=None, sigma_stderr=None, P=None):
    """Fill the given buffers (all host NumPy or all device tensors).  With no
    buffers, returns host arrays (sigma, stderr, P)."""
    ret = sigma is None and sigma_stderr is None and P is None
    if ret:
        n = rcell_info(ctx)[0]
        sigma, sigma_stderr, P = np.zeros((n, 6)), np.zeros((n, 6)), np.zeros((n, 3, 3))
    ps = [_arr_ptr(a) for a in (sigma, sigma_stderr, P)]
    wheres = {w for (p, w, k) in ps if p is not None}
    if len(wheres) > 1:
        raise ValueError("all stress outputs must be host or all device")
    where = wheres.pop() if wheres else RC_HOST
    _check(load().rcell_stress(ctx, ps[0][0], ps[1][0], ps[2][0], where), ctx, "rcell_stress")
    if ret:
        return sigma, sigma_stderr, P
    return None


def rcell_eval(ctx):
    _check(load().rcell_eval(ctx), ctx, "rcell_eval")


def rcell_get_energy(ctx):
    n = rcell_info(ctx)[0]
    pe, W = np.zeros(n), np.zeros((n, 3, 3))
    _check(load().rcell_get_energy(ctx, C.c_void_p(pe.ctypes.data), C.c_void_p(W.ctypes.data)), ctx,
           "rcell_get_energy")
    return pe, W


def rcell_get_atoms(ctx, cell: int, n_atoms: int):
    x, v, f = np.zeros((n_atoms, 3)), np.zeros((n_atoms, 3)), np.zeros((n_atoms, 3))
    _check(load().rcell_get_atoms(ctx, cell, C.c_void_p(x.ctypes.data), C.c_void_p(v.ctypes.data),
                                  C.c_void_p(f.ctypes.data)), ctx, "rcell_get_atoms")
    return x, v, f


def rcell_get_box(ctx, cell: int):
    H, Q, R = np.zeros((3, 3)), np.zeros((3, 3)), np.zeros((3, 3))
    _check(load().rcell_get_box(ctx, cell, C.c_void_p(H.ctypes.data), C.c_void_p(Q.ctypes.data),
                                C.c_void_p(R.ctypes.data)), ctx, "rcell_get_box")
    return H, Q, R


def rcell_get_neighbors(ctx, cell: int, max_pairs: int):
    pairs = np.zeros((max_pairs, 2), dtype=np.int32)
    cnt = C.c_long(0)
    _check(load().rcell_get_neighbors(ctx, cell, C.c_void_p(pairs.ctypes.data), max_pairs, C.byref(cnt)), ctx,
           "rcell_get_neighbors")
    return pairs[:cnt.value].copy()


def rcell_get_series(ctx, cell: int, n_avg: int):
    s, pe, ke = np.zeros((n_avg, 6)), np.zeros(n_avg), np.zeros(n_avg)
    _check(load().rcell_get_series(ctx, cell, C.c_void_p(s.ctypes.data), C.c_void_p(pe.ctypes.data),
                                   C.c_void_p(ke.ctypes.data)), ctx, "rcell_get_series")
    return s, pe, ke


def rcell_sync(ctx):
    return load().rcell_sync(ctx)


def rcell_clear_status(ctx):
    _check(load().rcell_clear_status(ctx), ctx, "rcell_clear_status")


def rcell_set_active(ctx, mask):
    """mask: host int array or CUDA int32 tensor, one entry per cell (0 = frozen)."""
    if hasattr(mask, "data_ptr"):
        p, where, keep = _arr_ptr(mask)
    else:
        keep = np.ascontiguousarray(mask, dtype=np.int32)
        p, where = C.c_void_p(keep.ctypes.data), RC_HOST
    _check(load().rcell_set_active(ctx, p, where), ctx, "rcell_set_active")


RC_WAIT_POLLS_DEFAULT = 1 << 22


def rcell_set_limits(ctx, max_neighbors: int = -1, wait_polls: int = -1):
    """Failure-injection limits: per-atom list capacity (0 = as allocated) and polls
    of the staging wait (values < 0 keep the current)."""
    _check(load().rcell_set_limits(ctx, int(max_neighbors), int(wait_polls)), ctx, "rcell_set_limits")


def rcell_set_staging(ctx, staged: int):
    _check(load().rcell_set_staging(ctx, int(staged)), ctx, "rcell_set_staging")


def rcell_set_tuning(ctx, threads_per_atom: int = -1, use_graphs: int = -1):
    _check(load().rcell_set_tuning(ctx, threads_per_atom, use_graphs), ctx, "rcell_set_tuning")


def rcell_info(ctx):
    n, na, kl = C.c_int(0), C.c_long(0), C.c_long(0)
    _check(load().rcell_info(ctx, C.byref(n), C.byref(na), C.byref(kl)), ctx, "rcell_info")
    return n.value, na.value, kl.value


PROFILE_NAMES = ["sort", "nlist", "density", "force", "deform", "remap", "stress", "force_sample"]


def rcell_profile_kernels(ctx, n_steps: int):
    """Mean duration (ms) of one launch of each kernel class (0 = not launched)."""
    out = np.zeros(8)
    _check(load().rcell_profile_kernels(ctx, n_steps, C.c_void_p(out.ctypes.data)), ctx, "rcell_profile_kernels")
    return {n: float(v) for n, v in zip(PROFILE_NAMES, out) if v > 0}


def rcell_minimize(ctx, max_iter, f_tol, dt0, dt_max, dmax=0.0):
    """FIRE relaxation at fixed box (Eq. CGPR1); returns per-cell move counts (-1: not converged)."""
    n = rcell_info(ctx)[0]
    it = np.zeros(n, dtype=np.int32)
    _check(load().rcell_minimize(ctx, int(max_iter), float(f_tol), float(dt0), float(dt_max), float(dmax),
                                 C.c_void_p(it.ctypes.data)), ctx, "rcell_minimize")
    return it


def rcell_stress_static(ctx, sigma=None, P=None):
    """Eq. PK1 stress of every cell from the pair sum: fills / returns (sigma (n,6), P (n,3,3)), host
    numpy arrays or CUDA tensors."""
    n = rcell_info(ctx)[0]
    if sigma is None and P is None:
        sigma, P = np.zeros((n, 6)), np.zeros((n, 3, 3))
    ps, ws, ks = _arr_ptr(sigma) if sigma is not None else (None, RC_HOST, None)
    pp, wp, kp = _arr_ptr(P) if P is not None else (None, ws, None)
    where = ws if sigma is not None else wp
    _check(load().rcell_stress_static(ctx, ps, pp, where), ctx, "rcell_stress_static")
    return sigma, P


def rcell_get_rebuilds(ctx):
    """Neighbour-list builds per cell since creation (uint64 array)."""
    n = rcell_info(ctx)[0]
    out = np.zeros(n, dtype=np.uint64)
    _check(load().rcell_get_rebuilds(ctx, C.c_void_p(out.ctypes.data)), ctx, "rcell_get_rebuilds")
    return out


def rcell_fp32_peak(stream=None) -> float:
    """Measured FP32 FMA throughput of the current GPU in TFLOP/s."""
    out = C.c_double(0.0)
    st = load().rcell_fp32_peak(_stream_ptr(stream), C.byref(out))
    if st != 0:
        raise RCellError(st, "rcell_fp32_peak")
    return out.value


def rcell_checkpoint(ctx, cell: int) -> bytes:
    L = load()
    nb = C.c_size_t(0)
    _check(L.rcell_checkpoint(ctx, cell, None, C.byref(nb)), ctx, "rcell_checkpoint")
    buf = C.create_string_buffer(nb.value)
    _check(L.rcell_checkpoint(ctx, cell, buf, C.byref(nb)), ctx, "rcell_checkpoint")
    return buf.raw


def rcell_restore(ctx, cell: int, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    _check(load().rcell_restore(ctx, cell, buf, len(blob)), ctx, "rcell_restore")


def rcell_stress_reduce_static(series, Q, F, sigma, sigma_stderr=None, P=None, stream=None):
    """Allocation-free stress reduction; all arrays are CUDA float64 tensors of
    the current device, contiguous: series (n_cells, n_avg, 6); Q, F
    (n_cells, 3, 3); outputs preallocated: sigma (n_cells, 6), optional
    sigma_stderr (n_cells, 6) and P (n_cells, 3, 3).  stream=None enqueues on
    torch's current stream of the current device.  Anything else raises
    RCellError(RC_EINVAL) before the library is called."""
    import torch
    if series is None or series.dim() != 3 or series.shape[2] != 6:
        raise RCellError(CODES["RC_EINVAL"], "series must have shape (n_cells, n_avg, 6)")
    n_cells, n_avg = int(series.shape[0]), int(series.shape[1])
    dev = torch.cuda.current_device()
    shapes = {"series": (series, (n_cells, n_avg, 6)), "Q": (Q, (n_cells, 3, 3)), "F": (F, (n_cells, 3, 3)),
              "sigma": (sigma, (n_cells, 6)), "sigma_stderr": (sigma_stderr, (n_cells, 6)),
              "P": (P, (n_cells, 3, 3))}
    for name, (t, shape) in shapes.items():
        if t is None and name in ("sigma_stderr", "P"):
            continue
        if t is None or not hasattr(t, "data_ptr"):
            raise RCellError(CODES["RC_EINVAL"], f"{name} must be a CUDA tensor")
        if not t.is_cuda or t.device.index != dev:
            raise RCellError(CODES["RC_EINVAL"], f"{name} must live on the current CUDA device ({dev})")
        if t.dtype != torch.float64:
            raise RCellError(CODES["RC_EINVAL"], f"{name} must be float64")
        if not t.is_contiguous():
            raise RCellError(CODES["RC_EINVAL"], f"{name} must be contiguous")
        if tuple(t.shape) != shape:
            raise RCellError(CODES["RC_EINVAL"], f"{name} has shape {tuple(t.shape)}, expected {shape}")
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    ptr = [None if a is None else C.c_void_p(a.data_ptr()) for a in (series, Q, F, sigma, sigma_stderr, P)]
    _check(load().rcell_stress_reduce_static(ptr[0], n_cells, n_avg, ptr[1], ptr[2], ptr[3], ptr[4], ptr[5],
                                             _stream_ptr(stream)), None, "rcell_stress_reduce_static")


def rcell_last_error(ctx) -> str:
    return load().rcell_last_error(ctx).decode()


def rcell_destroy(ctx):
    if ctx:
        load().rcell_destroy(ctx)


def fe_create(X, hex_conn, bc_mask, bc_val, rho0, dt, damping, hg_coef, stream=None):
    X = np.ascontiguousarray(X, dtype=np.float64)
    hx = np.ascontiguousarray(hex_conn, dtype=np.int32)
    m = np.ascontiguousarray(bc_mask, dtype=np.int32)
    v = np.ascontiguousarray(bc_val, dtype=np.float64)
    out = C.c_void_p()
    _check(load().fe_create(C.c_void_p(X.ctypes.data), X.shape[0], C.c_void_p(hx.ctypes.data), hx.shape[0],
                            C.c_void_p(m.ctypes.data), C.c_void_p(v.ctypes.data), rho0, dt, damping, hg_coef,
                            _stream_ptr(stream), C.byref(out)), None, "fe_create")
    return out


def fe_create_tet4(X, tet_conn, bc_mask, bc_val, rho0, dt, damping, stream=None):
    """Explicit FE on 4-node tetrahedra (positively oriented); the other fe_* calls are shared."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    tt = np.ascontiguousarray(tet_conn, dtype=np.int32)
    m = np.ascontiguousarray(bc_mask, dtype=np.int32)
    v = np.ascontiguousarray(bc_val, dtype=np.float64)
    out = C.c_void_p()
    _check(load().fe_create_tet4(C.c_void_p(X.ctypes.data), X.shape[0], C.c_void_p(tt.ctypes.data), tt.shape[0],
                                 C.c_void_p(m.ctypes.data), C.c_void_p(v.ctypes.data), rho0, dt, damping,
                                 _stream_ptr(stream), C.byref(out)), None, "fe_create_tet4")
    return out


def fe_apply_bc(fe, lam: float):
    _check(load().fe_apply_bc(fe, lam), None, "fe_apply_bc")


def fe_set_predictor(fe, g):
    """Affine predictor of the load increment (nn x 3 host array), or None to remove it."""
    if g is None:
        _check(load().fe_set_predictor(fe, None), None, "fe_set_predictor")
        return
    arr = np.ascontiguousarray(g, dtype=np.float64)
    _check(load().fe_set_predictor(fe, C.c_void_p(arr.ctypes.data)), None, "fe_set_predictor")


def fe_get_F(fe, F):
    p, where, keep = _arr_ptr(F)
    _check(load().fe_get_F(fe, p, where), None, "fe_get_F")


def fe_update(fe, P):
    p, where, keep = _arr_ptr(P)
    _check(load().fe_update(fe, p, where), None, "fe_update")


def fe_step(fe, rc, lam: float, n_steps: int, n_avg: int, u_out=None):
    p = None if u_out is None else C.c_void_p(u_out.ctypes.data)
    _check(load().fe_step(fe, rc, lam, n_steps, n_avg, p), rc, "fe_step")


def fe_step_surrogate(fe, rc, sur, lam, n_steps, n_avg, spread_on, spread_off, s_floor, force_md, h_state, F_prev,
                      md_flag, spread_out=None, with_replays=False):
    """Device state tensors: h_state (float32, members x ne x 128), F_prev (float64,
    ne x 3 x 3), md_flag (int32, ne), optional spread_out (float32, ne).
    Returns the number of points that ran MD at this increment, or with
    with_replays=True the pair (that number, missed increments replayed)."""
    n, r = C.c_int(0), C.c_int(0)
    ptr = [None if t is None else C.c_void_p(t.data_ptr()) for t in (h_state, F_prev, md_flag, spread_out)]
    _check(load().fe_step_surrogate(fe, rc, sur, lam, n_steps, n_avg, spread_on, spread_off, s_floor, int(force_md),
                                    ptr[0], ptr[1], ptr[2], ptr[3], C.byref(n), C.byref(r)), rc, "fe_step_surrogate")
    return (n.value, r.value) if with_replays else n.value


def fe_get_P(fe, P):
    p, where, keep = _arr_ptr(P)
    _check(load().fe_get_P(fe, p, where), None, "fe_get_P")


def fe_get_state(fe, nn: int):
    d, v = np.zeros((nn, 3)), np.zeros((nn, 3))
    _check(load().fe_get_state(fe, C.c_void_p(d.ctypes.data), C.c_void_p(v.ctypes.data)), None, "fe_get_state")
    return d, v


def fe_destroy(fe):
    if fe:
        load().fe_destroy(fe)


# ---------------------------------------------------------------------------
# parameter helpers for the workloads (values only; no arithmetic of the method)
# ---------------------------------------------------------------------------

def params_lj_cu(tau=0.1, kT=None, dt=0.002, seed=1, skin=0.5):
    """FCC copper-like LJ: eps = 0.415 eV, sigma = 2.277 A, rc = 2.5 sigma, m = 63.546 amu."""
    kT = 300 * 8.617333262e-5 if kT is None else kT
    return rcell_params(RC_POT_LJ, RC_UNITS_METAL, 0.415, 2.277, 2.5 * 2.277, 0, 0, 0, 0, 0, skin, 63.546, kT,
                        tau, dt, seed)


def params_sc_cu(tau=0.1, kT=None, dt=0.002, seed=1, skin=1.5):
    """Sutton-Chen copper: n = 9, m = 6, eps = 1.2382e-2 eV, c = 39.432, a = 3.61 A, rc = 2a."""
    kT = 300 * 8.617333262e-5 if kT is None else kT
    return rcell_params(RC_POT_SC, RC_UNITS_METAL, 1.2382e-2, 3.61, 7.22, 9.0, 6.0, 39.432, 0, 0, skin, 63.546,
                        kT, tau, dt, seed)


def params_kg(tau=2.0, kT=0.3, dt=0.005, seed=1, skin=0.3, max_step=0.0):
    """Kremer-Grest bead-spring (reduced units): LJ rc = 2.5, FENE k = 30, R0 = 1.5; gamma = 1/tau."""
    return rcell_params(RC_POT_KG, RC_UNITS_LJ, 1.0, 1.0, 2.5, 0, 0, 0, 30.0, 1.5, skin, 1.0, kT, tau, dt, seed,
                        max_step)
