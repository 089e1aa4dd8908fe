"""FP64 CPU oracle for the r-cell hot path (arXiv:1902.09171) -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or executes anything here, and this
package shares no code with it: the arithmetic lives in ``rcell_oracle.c``
(plain C, FP64) and, for the learned surrogate, in ``mlp.py`` (plain NumPy,
FP64).

The functions below are thin ctypes marshalling around the C routines; each C
routine names the passage of the paper (or the potential / integrator
definition the paper delegates to its MD engine) that it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rcell_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LJ, SC, KG = 0, 1, 2
METAL, LJUNITS = 0, 1

OR_OK, OR_EINVAL, OR_ENOMEM, OR_EDEGEN, OR_EBOX, OR_EBOND = 0, 1, 2, 4, 5, 6


class OracleError(RuntimeError):
    def __init__(self, code, what=""):
        super().__init__(f"oracle error {code} {what}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (FP64, IEEE semantics: no fast-math)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


class Pot(C.Structure):
    _fields_ = [("kind", C.c_int), ("eps", C.c_double), ("sigma", C.c_double), ("rc", C.c_double),
                ("n", C.c_double), ("m", C.c_double), ("c", C.c_double), ("k_fene", C.c_double),
                ("R0", C.c_double)]


class MD(C.Structure):
    _fields_ = [("units", C.c_int), ("mass", C.c_double), ("kT", C.c_double), ("tau", C.c_double),
                ("dt", C.c_double), ("seed", C.c_uint64)]


def pot_lj(eps, sigma, rc):
    return Pot(LJ, eps, sigma, rc, 0.0, 0.0, 0.0, 0.0, 0.0)


def pot_sc(eps, a, rc, n, m, c):
    return Pot(SC, eps, a, rc, n, m, c, 0.0, 0.0)


def pot_kg(eps=1.0, sigma=1.0, rc=2.5, k_fene=30.0, R0=1.5):
    return Pot(KG, eps, sigma, rc, 0.0, 0.0, 0.0, k_fene, R0)


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        D, I, P = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_uint32)
        L.or_qr.argtypes = [D, D, D]
        L.or_delta_R.argtypes = [D, D, D]
        L.or_remap.argtypes = [C.c_int, D, D]
        L.or_box_widths.argtypes = [D, D]
        L.or_rotate_pk1.argtypes = [D, D, D, D, D]
        L.or_philox4x32_10.argtypes = [P, P, P]
        L.or_normals3.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint64, D]
        L.or_neighbor_pairs.argtypes = [C.c_int, D, D, C.c_double, C.c_int, I, C.c_long]
        L.or_neighbor_pairs.restype = C.c_long
        L.or_forces.argtypes = [C.POINTER(Pot), C.c_int, D, D, C.c_int, I, C.c_int, D, D, D, D]
        L.or_ftm2v.argtypes = [C.c_int]
        L.or_ftm2v.restype = C.c_double
        L.or_pconv.argtypes = [C.c_int]
        L.or_pconv.restype = C.c_double
        L.or_stress_inst.argtypes = [C.c_int, C.c_double, C.c_int, D, D, D, D]
        L.or_md_run.argtypes = [C.POINTER(Pot), C.POINTER(MD), C.c_int, D, D, D, C.c_int, I, C.c_uint32,
                                C.POINTER(C.c_uint64), C.c_int, C.c_int, D, D, D]
        L.or_block_stats.argtypes = [C.c_int, D, C.c_int, D, D]
        L.or_fe_tet_geometry.argtypes = [C.c_int, D, C.c_int, I, C.c_double, D, D, D]
        L.or_fe_tet_F.argtypes = [C.c_int, I, D, D, D]
        L.or_fe_tet_update.argtypes = [C.c_int, C.c_int, I, D, D, D, I, D, C.c_double, C.c_double, D, D, D]
        L.or_pk1_pairs.argtypes = [C.POINTER(Pot), C.c_int, C.c_int, D, D, D, C.c_int, I, D]
        L.or_fire_minimize.argtypes = [C.POINTER(Pot), C.c_int, C.c_double, C.c_int, D, D, C.c_int, I, C.c_double,
                                       C.c_double, C.c_double, C.c_double, C.c_int, I]
        L.or_hex8_geometry.argtypes = [D, D, D]
        L.or_hex8_F.argtypes = [D, D, D]
        L.or_hex8_fint.argtypes = [D, D, C.c_double, D, D, C.c_double, D]
        L.or_fe_geometry.argtypes = [C.c_int, D, C.c_int, I, C.c_double, D, D, D]
        L.or_fe_apply_bc.argtypes = [C.c_int, I, D, C.c_double, D]
        L.or_fe_apply_bc_pred.argtypes = [C.c_int, I, D, D, C.c_double, C.c_double, D]
        L.or_fe_F.argtypes = [C.c_int, I, D, D, D]
        L.or_fe_update.argtypes = [C.c_int, D, C.c_int, I, D, D, D, I, D, C.c_double, C.c_double, C.c_double,
                                   D, D, D]
        _lib = L
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# --- geometry (Sec. 2.1) ---------------------------------------------------

def qr(F):
    """F = Q R, Q orthogonal, R upper triangular with positive diagonal."""
    F = _f64(F, (3, 3))
    Q = np.zeros((3, 3))
    R = np.zeros((3, 3))
    e = lib().or_qr(_dp(F), _dp(Q), _dp(R))
    if e:
        raise OracleError(e, "qr: det F <= 0")
    return Q, R


def delta_R(R_new, R_prev):
    out = np.zeros((3, 3))
    lib().or_delta_R(_dp(_f64(R_new, (3, 3))), _dp(_f64(R_prev, (3, 3))), _dp(out))
    return out


def remap(x, dR):
    x = _f64(x, (-1, 3)).copy()
    lib().or_remap(x.shape[0], _dp(x), _dp(_f64(dR, (3, 3))))
    return x


def box_widths(H):
    w = np.zeros(3)
    lib().or_box_widths(_dp(_f64(H, (3, 3))), _dp(w))
    return w


def rotate_pk1(Q, F, s_md):
    s_fem = np.zeros(6)
    P = np.zeros((3, 3))
    lib().or_rotate_pk1(_dp(_f64(Q, (3, 3))), _dp(_f64(F, (3, 3))), _dp(_f64(s_md, (6,))), _dp(s_fem), _dp(P))
    return s_fem, P


# --- random numbers ----------------------------------------------------------

def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    P = C.POINTER(C.c_uint32)
    lib().or_philox4x32_10(c.ctypes.data_as(P), k.ctypes.data_as(P), o.ctypes.data_as(P))
    return o


def normals3(tag, cell, ev, seed):
    z = np.zeros(3)
    lib().or_normals3(tag, cell, ev, seed, _dp(z))
    return z


# --- forces / neighbours -----------------------------------------------------

def forces(pot, x, H, bonds=None, use_cells=True, per_atom=False):
    """Conservative forces (n,3), pair virial W (3,3) and potential energy."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    H = _f64(H, (3, 3))
    b = np.zeros((0, 2), dtype=np.int32) if bonds is None else np.ascontiguousarray(bonds, dtype=np.int32)
    f = np.zeros((n, 3))
    W = np.zeros((3, 3))
    pe = C.c_double(0.0)
    pa = np.zeros(n) if per_atom else None
    e = lib().or_forces(C.byref(pot), n, _dp(x), _dp(H), b.shape[0], _ip(b), int(use_cells), _dp(f), _dp(W),
                        C.byref(pe), _dp(pa) if per_atom else None)
    if e:
        raise OracleError(e, "forces")
    if per_atom:
        return f, W, pe.value, pa
    return f, W, pe.value


def neighbor_pairs(x, H, rlist, use_cells=True, max_pairs=None):
    """Ordered pairs (i, j) with an image of j within rlist of i."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    if max_pairs is None:
        max_pairs = max(1024, n * 600)
    out = np.zeros((max_pairs, 2), dtype=np.int32)
    k = lib().or_neighbor_pairs(n, _dp(x), _dp(_f64(H, (3, 3))), rlist, int(use_cells), _ip(out), max_pairs)
    if k < 0:
        raise OracleError(-1, "neighbor_pairs")
    return out[:k].copy()


def ftm2v(units):
    return lib().or_ftm2v(units)


def pconv(units):
    return lib().or_pconv(units)


def stress_inst(units, mass, v, W, H):
    v = _f64(v, (-1, 3))
    s = np.zeros(6)
    lib().or_stress_inst(units, mass, v.shape[0], _dp(v), _dp(_f64(W, (3, 3))), _dp(_f64(H, (3, 3))), _dp(s))
    return s


def pk1_pairs(pot, x, H, H0, bonds=None, units=0):
    """Eq. PK1: first Piola-Kirchhoff stress (3,3) from the pair sum with the
    reference separations R_ij = H0 H^{-1} r_ij; potential part, pressure units."""
    x = _f64(x, (-1, 3))
    b = np.zeros((0, 2), dtype=np.int32) if bonds is None else np.ascontiguousarray(bonds, dtype=np.int32)
    P = np.zeros((3, 3))
    e = lib().or_pk1_pairs(C.byref(pot), units, x.shape[0], _dp(x), _dp(_f64(H, (3, 3))), _dp(_f64(H0, (3, 3))),
                           b.shape[0], _ip(b), _dp(P))
    if e:
        raise OracleError(e, "pk1_pairs")
    return P


def fire_minimize(pot, x, H, mass, f_tol, dt0, dt_max, max_iter, bonds=None, units=0, dmax=0.0):
    """Eq. CGPR1 by FIRE at fixed box (per-atom move cap dmax, <= 0: none):
    returns (minimised positions, moves before convergence or -1)."""
    x = _f64(x, (-1, 3)).copy()
    b = np.zeros((0, 2), dtype=np.int32) if bonds is None else np.ascontiguousarray(bonds, dtype=np.int32)
    it = C.c_int(0)
    e = lib().or_fire_minimize(C.byref(pot), units, mass, x.shape[0], _dp(x), _dp(_f64(H, (3, 3))), b.shape[0],
                               _ip(b), f_tol, dt0, dt_max, dmax, max_iter, C.byref(it))
    if e:
        raise OracleError(e, "fire_minimize")
    return x, it.value


def md_run(pot, md, x, v, H, bonds=None, cell=0, ev=0, n_steps=1, n_avg=0):
    """Fixed-box VV + Langevin MD on one cell; returns (x, v, eval, stress, pe, ke)."""
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    n = x.shape[0]
    b = np.zeros((0, 2), dtype=np.int32) if bonds is None else np.ascontiguousarray(bonds, dtype=np.int32)
    na = max(0, min(n_avg, n_steps))
    ss = np.zeros((max(na, 1), 6))
    pe = np.zeros(max(na, 1))
    ke = np.zeros(max(na, 1))
    evc = C.c_uint64(ev)
    e = lib().or_md_run(C.byref(pot), C.byref(md), n, _dp(x), _dp(v), _dp(_f64(H, (3, 3))), b.shape[0], _ip(b),
                        cell, C.byref(evc), n_steps, na, _dp(ss), _dp(pe), _dp(ke))
    if e:
        raise OracleError(e, "md_run")
    return x, v, evc.value, ss[:na], pe[:na], ke[:na]


def block_stats(y):
    y = _f64(y)
    m = C.c_double(0.0)
    s = C.c_double(0.0)
    lib().or_block_stats(y.shape[0], _dp(y), 1, C.byref(m), C.byref(s))
    return m.value, s.value


# --- finite elements (Sec. 2.2, Eq. f) ---------------------------------------

def hex8_geometry(Xe):
    g = np.zeros((8, 3))
    V = C.c_double(0.0)
    e = lib().or_hex8_geometry(_dp(_f64(Xe, (8, 3))), _dp(g), C.byref(V))
    if e:
        raise OracleError(e, "hex8 geometry")
    return g, V.value


def hex8_F(gradN, de):
    F = np.zeros((3, 3))
    lib().or_hex8_F(_dp(_f64(gradN, (8, 3))), _dp(_f64(de, (8, 3))), _dp(F))
    return F


def hex8_fint(Xe, gradN, V0, P, de, hg_coef):
    f = np.zeros((8, 3))
    lib().or_hex8_fint(_dp(_f64(Xe, (8, 3))), _dp(_f64(gradN, (8, 3))), V0, _dp(_f64(P, (3, 3))),
                       _dp(_f64(de, (8, 3))), hg_coef, _dp(f))
    return f


class FEMesh:
    """Explicit hex-8 FE driver state (FP64), mirroring the order of one FE step."""

    def __init__(self, X, conn, bc_mask, bc_val, rho0, dt, damping, hg_coef):
        self.X = _f64(X, (-1, 3))
        self.conn = np.ascontiguousarray(conn, dtype=np.int32).reshape(-1, 8)
        self.nn, self.ne = self.X.shape[0], self.conn.shape[0]
        self.bc_mask = np.ascontiguousarray(bc_mask, dtype=np.int32).reshape(-1, 3)
        self.bc_val = _f64(bc_val, (-1, 3))
        self.dt, self.damping, self.hg = dt, damping, hg_coef
        self.gradN = np.zeros((self.ne, 8, 3))
        self.V0 = np.zeros(self.ne)
        self.mass = np.zeros(self.nn)
        e = lib().or_fe_geometry(self.nn, _dp(self.X), self.ne, _ip(self.conn), rho0, _dp(self.gradN),
                                 _dp(self.V0), _dp(self.mass))
        if e:
            raise OracleError(e, "fe geometry")
        self.d = np.zeros((self.nn, 3))
        self.v = np.zeros((self.nn, 3))

    g = None
    lam_last = 0.0

    def set_predictor(self, g):
        """Affine predictor of the load increment (nn x 3, or None): see or_fe_apply_bc_pred."""
        self.g = None if g is None else _f64(g, (-1, 3)).copy()

    def apply_bc(self, lam):
        if self.g is None:
            lib().or_fe_apply_bc(self.nn, _ip(self.bc_mask), _dp(self.bc_val), lam, _dp(self.d))
        else:
            lib().or_fe_apply_bc_pred(self.nn, _ip(self.bc_mask), _dp(self.bc_val), _dp(self.g), lam,
                                      lam - self.lam_last, _dp(self.d))
        self.lam_last = lam

    def F(self):
        F = np.zeros((self.ne, 3, 3))
        lib().or_fe_F(self.ne, _ip(self.conn), _dp(self.gradN), _dp(self.d), _dp(F))
        return F

    def update(self, P):
        P = _f64(P, (self.ne, 3, 3))
        fint = np.zeros((self.nn, 3))
        lib().or_fe_update(self.nn, _dp(self.X), self.ne, _ip(self.conn), _dp(self.gradN), _dp(self.V0),
                           _dp(self.mass), _ip(self.bc_mask), _dp(P), self.hg, self.dt, self.damping, _dp(self.d),
                           _dp(self.v), _dp(fint))
        return fint


class FETetMesh:
    """Explicit 4-node tetrahedron FE driver state (FP64), the same step order as FEMesh."""

    g = None
    lam_last = 0.0
    set_predictor = FEMesh.set_predictor

    def __init__(self, X, conn, bc_mask, bc_val, rho0, dt, damping):
        self.X = _f64(X, (-1, 3))
        self.conn = np.ascontiguousarray(conn, dtype=np.int32).reshape(-1, 4)
        self.nn, self.ne = self.X.shape[0], self.conn.shape[0]
        self.bc_mask = np.ascontiguousarray(bc_mask, dtype=np.int32).reshape(-1, 3)
        self.bc_val = _f64(bc_val, (-1, 3))
        self.dt, self.damping = dt, damping
        self.gradN = np.zeros((self.ne, 4, 3))
        self.V0 = np.zeros(self.ne)
        self.mass = np.zeros(self.nn)
        e = lib().or_fe_tet_geometry(self.nn, _dp(self.X), self.ne, _ip(self.conn), rho0, _dp(self.gradN),
                                     _dp(self.V0), _dp(self.mass))
        if e:
            raise OracleError(e, "fe tet geometry")
        self.d = np.zeros((self.nn, 3))
        self.v = np.zeros((self.nn, 3))

    def apply_bc(self, lam):
        if self.g is None:
            lib().or_fe_apply_bc(self.nn, _ip(self.bc_mask), _dp(self.bc_val), lam, _dp(self.d))
        else:
            lib().or_fe_apply_bc_pred(self.nn, _ip(self.bc_mask), _dp(self.bc_val), _dp(self.g), lam,
                                      lam - self.lam_last, _dp(self.d))
        self.lam_last = lam

    def F(self):
        F = np.zeros((self.ne, 3, 3))
        lib().or_fe_tet_F(self.ne, _ip(self.conn), _dp(self.gradN), _dp(self.d), _dp(F))
        return F

    def update(self, P):
        P = _f64(P, (self.ne, 3, 3))
        fint = np.zeros((self.nn, 3))
        lib().or_fe_tet_update(self.nn, self.ne, _ip(self.conn), _dp(self.gradN), _dp(self.V0), _dp(self.mass),
                               _ip(self.bc_mask), _dp(P), self.dt, self.damping, _dp(self.d), _dp(self.v),
                               _dp(fint))
        return fint
