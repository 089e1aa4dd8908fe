"""Drivers for the multi-increment workloads: loop control around the C ABI.

Every numerical step runs in the CUDA library (r-cell MD, deformation, stress,
surrogate features / training / inference, FE update); these functions only
sequence the calls, move the seeded inputs in and the results out, and keep
the timings.

  * prepare_kg_batch  : Kremer-Grest melts -> equilibrated r-cell batch
  * generate_dataset  : S1 -- strain paths run through batched r-cells, labelled
                        with the time-averaged FE-frame stress of each increment
  * train             : AdamW over BPTT of every ensemble member (cosine lr)
  * fe_compare        : the same FE load history with all-MD r-cells and with
                        the surrogate + ensemble-spread MD fallback
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs, rcell
from . import surrogate as S


def _torch():
    import torch
    return torch


def prepare_kg_batch(n_cells, n_chains=100, chain_len=50, density=0.85, seed=3, stream=None, soft_steps=2000,
                     eq_steps=2000, kT=0.3, skin=0.3, n_distinct=4, tpa=1, cells=None, starmap=None):
    """Melts -> soft start (dt 0.002, strong friction, T = 1, displacement limited to
    0.02 sigma per step) -> equilibration at the production temperature.  Returns (ctx, cells) with ctx holding the equilibrated
    production batch (dt = 0.005, gamma = 0.5).  cells: prebuilt melts (dicts of
    inputs.kg_cells) instead of generating them; starmap: parallel melt generation."""
    if cells is None:
        cells = inputs.kg_cells(n_cells, n_chains, chain_len, density, seed, n_distinct, starmap=starmap)
    soft = rcell.params_kg(tau=0.5, kT=1.0, dt=0.002, seed=seed, skin=skin, max_step=0.02)
    ctx = rcell.rcell_create(soft, cells, stream=stream)
    rcell.rcell_set_tuning(ctx, tpa, 1)
    rcell.rcell_run(ctx, soft_steps, 0)
    st = rcell.rcell_sync(ctx)
    if st != 0:
        raise rcell.RCellError(st, "soft start: " + rcell.rcell_last_error(ctx))
    eq_cells = []
    for k, c in enumerate(cells):
        x, v, _ = rcell.rcell_get_atoms(ctx, k, len(c["x0"]))
        eq_cells.append(dict(H0=c["H0"], x0=x, v0=v, bonds=c["bonds"]))
    rcell.rcell_destroy(ctx)
    prod = rcell.params_kg(tau=2.0, kT=kT, dt=0.005, seed=seed + 1, skin=skin)
    ctx = rcell.rcell_create(prod, eq_cells, stream=stream)
    rcell.rcell_set_tuning(ctx, tpa, 1)
    if eq_steps:
        rcell.rcell_run(ctx, eq_steps, 0)
    st = rcell.rcell_sync(ctx)
    if st != 0:
        raise rcell.RCellError(st, "equilibration: " + rcell.rcell_last_error(ctx))
    final = []
    for k, c in enumerate(eq_cells):
        x, v, _ = rcell.rcell_get_atoms(ctx, k, len(c["x0"]))
        final.append(dict(H0=c["H0"], x0=x, v0=v, bonds=c["bonds"]))
    return ctx, final


def generate_dataset(ctx, F_paths, n_steps, n_avg, stream=None):
    """Run every path (one r-cell each) through its increments: for t = 1..T
    deform to F[:, t], run n_steps MD steps, take the stress averaged over the
    last n_avg.  Returns device tensors U (n, T, 15) of surrogate inputs and
    Y (n, T, 6) of stresses, plus the atom-steps spent."""
    torch = _torch()
    n, T1 = F_paths.shape[0], F_paths.shape[1]
    T = T1 - 1
    dev = torch.device("cuda")
    Fd = torch.tensor(F_paths, dtype=torch.float64, device=dev).contiguous()
    U = torch.zeros((T, n, 15), dtype=torch.float32, device=dev)
    Y = torch.zeros((T, n, 6), dtype=torch.float32, device=dev)
    sig = torch.zeros((n, 6), dtype=torch.float64, device=dev)
    n_atoms = rcell.rcell_info(ctx)[1]
    for t in range(1, T1):
        Ft = Fd[:, t].contiguous()
        rcell.rcell_set_deformation(ctx, Ft)
        rcell.rcell_run(ctx, n_steps, n_avg)
        rcell.rcell_stress(ctx, sig)
        Y[t - 1].copy_(sig.float())
        S.sur_features(Fd[:, t - 1].contiguous(), Ft, U[t - 1], stream=stream)
    st = rcell.rcell_sync(ctx)
    if st != 0:
        raise rcell.RCellError(st, "dataset: " + rcell.rcell_last_error(ctx))
    return U.transpose(0, 1).contiguous(), Y.transpose(0, 1).contiguous(), n_atoms * n_steps * T


def feature_scales(U, Y):
    """Input scales: per-feature standard deviations, floored at 10 % of the largest
    one of the same block (the 9 increment components, the 6 strain components), so
    that a component the training paths barely excite is not blown up to O(1)
    inputs when a quadrature point does excite it.  Output scale: one common RMS
    over all six stress components, so that components a path barely drives (pure
    sampling noise) keep their small weight in the loss."""
    u = U.reshape(-1, U.shape[-1]).std(0)
    for a, b in ((0, 9), (9, 15)):
        u[a:b] = u[a:b].clamp_min(0.1 * float(u[a:b].max()) + 1e-12)
    y = float((Y ** 2).mean().sqrt().clamp_min(1e-4))
    return u.cpu().numpy(), np.full(6, y, dtype=np.float32)


def train(sur, U, Y, steps, lr=1e-3, wd=0.01, n_members=4, log_every=0):
    """AdamW with a cosine learning-rate schedule over `steps` full-batch steps."""
    losses = []
    for k in range(steps):
        lr_k = 0.5 * lr * (1.0 + math.cos(math.pi * k / steps))
        want = log_every and (k % log_every == 0 or k == steps - 1)
        l = S.sur_train_step(sur, U, Y, lr_k, wd, n_members=n_members, want_loss=bool(want))
        if want:
            losses.append((k, l.tolist()))
    return losses


def relative_error(sur, U, Y, n_members, s_floor=0.0, with_spread=False):
    """RMS error of the ensemble-mean prediction over the RMS of the targets; with
    with_spread, also quantiles of the ensemble spread
    ||std over members|| / max(||mean||, s_floor) over all (path, increment)."""
    torch = _torch()
    B, T = U.shape[0], U.shape[1]
    out = torch.zeros((n_members, B, T, 6), dtype=torch.float32, device=U.device)
    S.sur_predict(sur, U, out)
    mean = out.mean(0)
    err = float(((mean - Y) ** 2).mean().sqrt() / (Y ** 2).mean().sqrt())
    if not with_spread:
        return err
    sd = out.std(0, unbiased=True).norm(dim=-1) / mean.norm(dim=-1).clamp_min(s_floor)
    q = torch.quantile(sd.flatten().float(), torch.tensor([0.1, 0.5, 0.9, 0.99], device=sd.device))
    return err, [float(v) for v in q]


def fe_compare_surrogate_only(ctx_sg, sur, fe_sg, n_members, lambdas, n_steps, n_avg, spread_on, spread_off, s_floor,
                              reference, md_first=2, stream=None):
    """The surrogate half of fe_compare against a stored all-MD reference
    (axial stress curve, milliseconds)."""
    torch = _torch()
    ne = rcell.rcell_info(ctx_sg)[0]
    dev = torch.device("cuda")
    st = stream or torch.cuda.current_stream()
    h = torch.zeros((n_members, ne, 128), dtype=torch.float32, device=dev)
    Fp = torch.eye(3, dtype=torch.float64, device=dev).repeat(ne, 1, 1).contiguous()
    flag = torch.zeros(ne, dtype=torch.int32, device=dev)
    P = torch.zeros((ne, 3, 3), dtype=torch.float64, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    P_sg, n_md = [], []
    e0.record(st)
    for k, lam in enumerate(lambdas):
        n, r = rcell.fe_step_surrogate(fe_sg, ctx_sg, sur, lam, n_steps, n_avg, spread_on, spread_off, s_floor,
                                       k < md_first, h, Fp, flag, with_replays=True)
        n_md.append(n + r)  # MD cell-increments: this increment's and the replayed ones
        rcell.fe_get_P(fe_sg, P)
        P_sg.append(P[:, 0, 0].mean())
    e1.record(st)
    torch.cuda.synchronize()
    a, b = np.array(reference[0]), np.array([float(v) for v in P_sg])
    return {"ms_sg": e0.elapsed_time(e1), "axial_sg": b.tolist(), "n_md": n_md,
            "max_rel_dev": float(np.abs(a - b).max() / max(np.abs(a).max(), 1e-30)),
            "md_fraction": float(sum(n_md) / (ne * len(lambdas)))}


def fe_compare(ctx_md, ctx_sg, sur, fe_md, fe_sg, n_members, lambdas, n_steps, n_avg, spread_on=0.02,
               spread_off=0.01, s_floor=0.05, md_first=2, stream=None):
    """Drive two identical FE bars through the same load history: one with all
    r-cells on MD (fe_step), one with the surrogate + MD fallback
    (fe_step_surrogate).  Returns per-increment system-averaged axial stresses,
    MD counts and the wall time of each run (CUDA-event timed)."""
    torch = _torch()
    ne = rcell.rcell_info(ctx_md)[0]
    dev = torch.device("cuda")
    st = stream or torch.cuda.current_stream()
    res = {"axial_md": [], "axial_sg": [], "n_md": []}
    P = torch.zeros((ne, 3, 3), dtype=torch.float64, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    P_md = []
    e0.record(st)
    for lam in lambdas:
        rcell.fe_step(fe_md, ctx_md, lam, n_steps, n_avg, None)
        rcell.fe_get_P(fe_md, P)
        P_md.append(P[:, 0, 0].mean())
    e1.record(st)
    torch.cuda.synchronize()
    res["ms_md"] = e0.elapsed_time(e1)
    res["axial_md"] = [float(v) for v in P_md]
    h = torch.zeros((n_members, ne, 128), dtype=torch.float32, device=dev)
    Fp = torch.eye(3, dtype=torch.float64, device=dev).repeat(ne, 1, 1).contiguous()
    flag = torch.zeros(ne, dtype=torch.int32, device=dev)
    spread = torch.zeros(ne, dtype=torch.float32, device=dev)
    P_sg, sp = [], []
    e0.record(st)
    for k, lam in enumerate(lambdas):
        n, r = rcell.fe_step_surrogate(fe_sg, ctx_sg, sur, lam, n_steps, n_avg, spread_on, spread_off, s_floor,
                                       k < md_first, h, Fp, flag, spread, with_replays=True)
        n += r  # MD cell-increments: this increment's and the replayed ones
        rcell.fe_get_P(fe_sg, P)
        P_sg.append(P[:, 0, 0].mean())
        sp.append(spread.median())
        res["n_md"].append(n)
    e1.record(st)
    torch.cuda.synchronize()
    res["ms_sg"] = e0.elapsed_time(e1)
    res["axial_sg"] = [float(v) for v in P_sg]
    res["spread_median"] = [float(v) for v in sp]
    a, b = np.array(res["axial_md"]), np.array(res["axial_sg"])
    res["max_rel_dev"] = float(np.abs(a - b).max() / max(np.abs(a).max(), 1e-30))
    res["md_fraction"] = float(sum(res["n_md"]) / (ne * len(lambdas)))
    return res


def fe_compare_md_only(ctx, fe, lambdas, n_steps, n_avg, stream=None):
    """The all-MD half of fe_compare on its own (another bar, e.g. another Langevin
    seed, to state the MD noise of the axial stress curve)."""
    torch = _torch()
    ne = rcell.rcell_info(ctx)[0]
    st = stream or torch.cuda.current_stream()
    P = torch.zeros((ne, 3, 3), dtype=torch.float64, device=torch.device("cuda"))
    out = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for lam in lambdas:
        rcell.fe_step(fe, ctx, lam, n_steps, n_avg, None)
        rcell.fe_get_P(fe, P)
        out.append(P[:, 0, 0].mean())
    e1.record(st)
    torch.cuda.synchronize()
    return {"ms_md": e0.elapsed_time(e1), "axial_md": [float(v) for v in out]}


def tensile_F(eps, nu=0.5):
    """Uniaxial stretch along x with lateral contraction (1 + eps)^-nu."""
    lam = 1.0 + eps
    return np.diag([lam, lam ** -nu, lam ** -nu])


def pbc_tensile(ctx, rate, dt, n_chunks, chunk_steps, nu=0.5, eps0=0.0):
    """Direct periodic-box MD tensile test of every r-cell (the comparison run of
    Sec. 3.2): the box follows a uniaxial engineering strain that grows at `rate`
    per unit time, applied as a new deformation (QR, remap) every `chunk_steps` MD
    steps, each chunk averaging the stress over its steps.  Returns the strains
    and the per-cell FE-frame stresses (n_chunks, n_cells, 6)."""
    n = rcell.rcell_info(ctx)[0]
    eps, sig = [], []
    for k in range(1, n_chunks + 1):
        e = eps0 + rate * dt * chunk_steps * k
        rcell.rcell_set_deformation(ctx, np.tile(tensile_F(e, nu), (n, 1, 1)))
        rcell.rcell_run(ctx, chunk_steps, chunk_steps)
        s, _, _ = rcell.rcell_stress(ctx)
        eps.append(e)
        sig.append(s)
    return np.array(eps), np.array(sig)
