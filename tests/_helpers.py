"""Shared helpers of the GPU parity tests (test-side only)."""
import numpy as np

import oracle
from paper_1902_09171_gb300 import inputs, rcell

KB = inputs.KB_EV
M_CU = 63.546


def min_image_diff(a, b, H):
    """Minimum-image difference a - b of positions in the periodic box H."""
    d = np.asarray(a) - np.asarray(b)
    s = d @ np.linalg.inv(H).T
    s -= np.round(s)
    return s @ H.T


def oracle_pot(prm):
    if prm.potential == rcell.RC_POT_LJ:
        return oracle.pot_lj(prm.eps, prm.sigma, prm.rc)
    if prm.potential == rcell.RC_POT_SC:
        return oracle.pot_sc(prm.eps, prm.sigma, prm.rc, prm.n, prm.m, prm.c)
    return oracle.pot_kg(prm.eps, prm.sigma, prm.rc, prm.k_fene, prm.R0)


def oracle_md(prm):
    return oracle.MD(prm.units, prm.mass, prm.kT, prm.tau, prm.dt, prm.seed)


def force_err(f_gpu, f_ref):
    """Per-atom error relative to max(|f_i|, f_rms(cell)) -- the force tolerance reading."""
    frms = np.sqrt((f_ref ** 2).sum(1).mean())
    scale = np.maximum(np.linalg.norm(f_ref, axis=1), frms)
    return (np.linalg.norm(f_gpu - f_ref, axis=1) / scale).max()


def lj_cell(nc=4, jit=0.05, seed=1, T=300.0):
    x, H = inputs.fcc(nc, nc, nc, 3.615)
    x = inputs.to_f32(inputs.jitter(x, jit, seed))
    v = inputs.to_f32(inputs.maxwell(len(x), M_CU, T * KB, 0, seed))
    return dict(H0=H, x0=x, v0=v)


def voigt_rotate_series(Q, series):
    out = np.zeros_like(series)
    for t in range(len(series)):
        out[t], _ = oracle.rotate_pk1(Q, np.eye(3), series[t])
    return out
