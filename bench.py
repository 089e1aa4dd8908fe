"""Benchmark of the r-cell hot path on GB300.

Workload (default, --workload necking_bar): the necking bar -- a 32x4x4 hex
mesh with one quadrature point per element = 512 r-cells of 20 000
Kremer-Grest beads each (400 chains of 50, melt density 0.85, T = 0.3,
Langevin gamma = 0.5, dt = 0.005), 10.24 million beads on one GPU, with a 5 %
cross-section imperfection at mid-length; uniaxial tension to 60 % in 150
increments, 1000 MD steps per increment with the stress averaged over the last
500.  The Verlet skin and the lanes per atom are chosen by the autotuner.

One bench step = one FE load increment through the whole path: boundary
conditions -> element F -> QR / box / remap -> 1000 MD steps (neighbour lists,
forces, Verlet + Langevin, per-cell virial) -> time-averaged stress -> rotation
and P -> FE internal force and explicit update.  With --gpus N the 512 cells
are split over the ranks (atom-balanced), every rank advances the same FE mesh
and the stresses are all-gathered once per increment (strong scaling).

  value : atom-steps/s with everything resident in HBM (fe_step, device F).
  e2e   : the same increments through the public API with host buffers: the FE's
          F copied to the host, handed to the r-cells from host memory, sigma,
          its standard error and P copied back, P handed to the FE update from
          host memory (the coupling of an FE code running on the host).

Other workloads: copper_bar (32 Sutton-Chen cells), kg_bar (64 uneven KG
cells), surrogate_fe, surrogate_train, kg_statics, kg_tensile.

`--impl reference` times the FP64 CPU oracle on this machine's host cores on a
bounded sample of the same workload (the reference arm of this benchmark).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1902_09171_gb300 import inputs  # noqa: E402

A_LAT = 3.615
NC = 10                 # unit cells per edge of one r-cell
MESH = (8, 2, 2)
N_INC = 25
STRAIN = 0.05
MD_STEPS = 1000
N_AVG = 500
KT = 300 * inputs.KB_EV
MASS = 63.546
SC = dict(eps=1.2382e-2, a=3.61, rc=7.22, n=9.0, m=6.0, c=39.432)
WORKLOAD = "copper_bar_sc_eam_32x4000"


def make_cells(n_cells, seed0=1000):
    x, H = inputs.fcc(NC, NC, NC, A_LAT)
    x = inputs.to_f32(x)
    return [dict(H0=H, x0=x, v0=inputs.to_f32(inputs.maxwell(len(x), MASS, KT, 0, seed0 + c))) for c in range(n_cells)]


def mesh(element="hex8"):
    """The bar's mesh: 8 x 2 x 2 hexahedra, or the same box in 6 tetrahedra per
    hexahedron (the paper's C3D4 element)."""
    L = NC * A_LAT
    gen = inputs.tet_mesh if element == "tet4" else inputs.hex_mesh
    X, conn = gen(*MESH, MESH[0] * L, MESH[1] * L, MESH[2] * L)
    mask, val = inputs.uniaxial_bc(X, MESH[0] * L)
    return X, conn, mask, val


# FE of the copper bar in units consistent with the r-cell stress: P in GPa,
# lengths in A, time in ps, so that P * area (GPa A^2) = mass * acceleration
# needs masses in units of 1e-25 kg = 60.2214 amu.  E_CU is the modulus used to
# size the explicit step (0.5 h / c, c = sqrt(E / rho0)), the mass-proportional
# damping (critical for the bar's fundamental mode) and the hourglass stiffness
# (0.05 E).
AMU_PER_FE_MASS = 60.2214
E_CU = 130.0  # GPa


def fe_params():
    rho0 = 4 * MASS / A_LAT ** 3 / AMU_PER_FE_MASS
    c = np.sqrt(E_CU / rho0)  # A / ps
    h = NC * A_LAT
    dt = 0.5 * h / c
    damping = np.pi * c / (MESH[0] * h)  # 2 omega_1 of a bar fixed at one end
    return rho0, dt, damping, 0.05 * E_CU


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard(n_units, world, rank):
    """Contiguous, balanced split of n_units independent units over ranks."""
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.f:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            p = [q.strip() for q in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes (read + write) of one k_force<SC> launch on this workload (128 000
# atoms, skin 1.5 A), from an ncu capture of the current kernel (the variant
# without a stress sample; the other one reads the same list): 121.91 MB read
# + 2.72 MB written.  Mostly the Verlet list, re-read from DRAM every
# launch.
K_FORCE_DRAM_BYTES = 124.63e6


def fp32_unit_peak_tflops():
    """FP32 FMA peak from unit counts and the maximum SM clock: 152 SMs x 128
    FP32 lanes x 2 FLOP per FMA x 2070 MHz."""
    return 152 * 128 * 2 * 2.070e9 / 1e12


def sc_algorithmic_flops_per_atom_step(rho):
    """Algorithmic FP32 work of one Sutton-Chen atom-step, counted once per
    unordered pair inside rc (FMA = 2 FLOP): density pass 14 FLOP/pair (r^2,
    (a/r)^m through r^-6); force pass 30 FLOP/pair for the (a/r)^9, (a/r)^6
    combination and the force scalar, 12 for the f_i / f_j accumulation and 12
    for the six virial components on the steps that record a stress sample;
    40 FLOP/atom for the integrator and the Langevin force.  Returns
    (density_per_atom, force_per_atom without sample, force_per_atom with sample)."""
    half_pairs = rho * 4.0 / 3.0 * np.pi * SC["rc"] ** 3 / 2.0
    return 14.0 * half_pairs, 42.0 * half_pairs + 40.0, 54.0 * half_pairs + 40.0


NECK_MESH = (32, 4, 4)
NECK_BEADS, NECK_CHAIN, NECK_DENSITY = 20000, 50, 0.85
NECK_INC, NECK_STRAIN, NECK_MD, NECK_AVG = 150, 0.6, 1000, 500
NECK_IMPERFECTION = 0.05
NECK_WORKLOAD = "necking_bar_kg_512x20000"
NECK_SKINS, NECK_TPAS = (0.4, 0.5, 0.6, 0.7), (0, 1)  # lanes per atom 0: the lean walk
# the KG bar's uneven batch (761 300 beads, under a tenth of the necking bar)
# fills fewer warps per SM, so its search also offers the smallest skin and
# two lanes per bead
KG_BAR_SKINS, KG_BAR_TPAS = (0.3, 0.4, 0.5, 0.6, 0.8), (0, 1, 2)
NECK_TUNE_CELLS = 128  # a quarter of the bar: 20 000 tiles, enough waves to behave like the whole

# DRAM bytes (read + write) per bead of one k_force<KG> launch (the lean walk,
# non-sampling variant), by Verlet skin, from ncu captures of 16 necking-bar
# cells (320 000 beads; mean of two launches): skin 0.4: 146.78 + 4.62 MB,
# skin 0.5: 160.24 + 4.51 MB.  A launch's traffic grows in proportion to its
# beads (lists, positions and velocities are per bead); the list length
# depends on the skin.
K_FORCE_KG_DRAM_BYTES_PER_ATOM = {0.4: 151.40e6 / 320000, 0.5: 164.75e6 / 320000}


def kg_algorithmic_flops_per_atom_step(rho, bonds_per_atom):
    """Algorithmic FP32 work of one Kremer-Grest bead-step, counted once per
    unordered pair inside rc (FMA = 2 FLOP): 26 FLOP per non-bonded LJ pair
    (displacement 3, r^2 5, 1/r^2 1, r^-6 2, force scalar 3, f_i / f_j 12) plus
    12 for its six virial components on the steps that record a stress sample,
    40 per FENE + WCA bond, 40 per bead for the integrator and the Langevin
    force.  Returns (without sample, with sample) per bead."""
    half = rho * 4.0 / 3.0 * np.pi * 2.5 ** 3 / 2.0 - bonds_per_atom
    return 26.0 * half + 40.0 * bonds_per_atom + 40.0, 38.0 * half + 40.0 * bonds_per_atom + 40.0


def necking_cells(ne, n_distinct, procs, seed=5):
    """The bar's r-cells (512 for the full mesh): n_distinct seeded 20 000-bead melts
    (generated in a spawned process pool), each cell a copy shifted by a seeded
    periodic translation."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(max(1, min(procs, n_distinct))) as pool:
        return inputs.kg_cells(ne, NECK_BEADS // NECK_CHAIN, NECK_CHAIN, NECK_DENSITY, seed, n_distinct,
                               starmap=pool.starmap)


def axial_predictor(X):
    """Affine predictor of a uniaxial load increment along x: g = (X_x, 0, 0)."""
    g = np.zeros_like(X)
    g[:, 0] = X[:, 0]
    return g


class CudaFE:
    """The FE context behind the interface of dist.fe_step_sharded (device tensors)."""

    def __init__(self, fe, ne, torch):
        from paper_1902_09171_gb300 import rcell
        self.rc, self.fe = rcell, fe
        self.Fbuf = torch.zeros((ne, 3, 3), dtype=torch.float64, device="cuda")

    def apply_bc(self, lam):
        self.rc.fe_apply_bc(self.fe, lam)

    def F(self):
        self.rc.fe_get_F(self.fe, self.Fbuf)
        return self.Fbuf

    def update(self, P):
        self.rc.fe_update(self.fe, P)


def run_necking_bar(args):
    import torch

    from paper_1902_09171_gb300 import autotune, build, pipeline, rcell
    from paper_1902_09171_gb300 import dist as rdist

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    rcell.load()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    mesh = tuple(int(v) for v in args.mesh.split(",")) if args.mesh else NECK_MESH
    ne = int(np.prod(mesh))
    bounds = rdist.shard_by_atoms([NECK_BEADS] * ne, world)
    a, b = bounds[rank]
    t_prep = time.time()
    cells = necking_cells(ne, args.distinct, args.procs)[a:b]
    # soft start and equilibration of this rank's cells (input preparation)
    ctx0, eq = pipeline.prepare_kg_batch(b - a, stream=stream, seed=7 + rank, soft_steps=args.soft_steps,
                                         eq_steps=args.eq_steps, cells=cells)
    rcell.rcell_destroy(ctx0)
    # autotuned Verlet skin and lanes per atom, timed on 128 of this rank's cells
    # (on 32 cells, under three waves of tiles, a longer list looked cheaper than
    # it is on the whole bar) over 400 MD steps (a few list rebuilds per cell),
    # the last 200 sampling the stress as the increments do
    make = lambda skin: rcell.params_kg(seed=11 + rank, skin=skin)  # noqa: E731
    if args.skin_kg > 0:
        tuned, hit = {"skin": args.skin_kg, "tpa": args.tpa if args.tpa >= 0 else 1, "table": []}, False
    else:
        tuned, hit = autotune.tune(make, eq[:NECK_TUNE_CELLS], stream, skins=NECK_SKINS, tpas=NECK_TPAS, n_steps=400,
                                   n_avg=200)
    ctx = rcell.rcell_create(make(tuned["skin"]), eq, stream=stream)
    rcell.rcell_set_tuning(ctx, int(tuned["tpa"]), 1)
    h = NECK_BEADS ** (1.0 / 3.0) / NECK_DENSITY ** (1.0 / 3.0)
    X, conn = inputs.necking_mesh(*mesh, h, NECK_IMPERFECTION)
    mask, val = inputs.uniaxial_bc(X, mesh[0] * h)
    fe = rcell.fe_create(X, conn, mask, val, NECK_DENSITY, 2.0, 1.0, 1.0, stream=stream)
    rcell.fe_set_predictor(fe, axial_predictor(X))
    t_prep = time.time() - t_prep
    md, navg = args.md_steps, min(NECK_AVG, args.md_steps // 2)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    P_local = torch.zeros((b - a, 3, 3), dtype=torch.float64, device="cuda")
    cfe = CudaFE(fe, ne, torch)

    def run_cells(F_local):
        rcell.rcell_set_deformation(ctx, F_local)
        rcell.rcell_run(ctx, md, navg)
        rcell.rcell_stress(ctx, P=P_local)
        return P_local

    def lam_of(k):
        return NECK_STRAIN * ((k % NECK_INC) + 1) / NECK_INC

    def one_step(k):
        if world == 1:
            rcell.fe_step(fe, ctx, lam_of(k), md, navg, None)
        else:
            rdist.fe_step_sharded(cfe, run_cells, lam_of(k), bounds, rank)

    for k in range(args.warmup):
        one_step(k)
    torch.cuda.synchronize()
    if rcell.rcell_sync(ctx) != 0:
        raise RuntimeError("warm-up failed: " + rcell.rcell_last_error(ctx))
    fp32_peak = rcell.rcell_fp32_peak(stream)
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    rb0 = rcell.rcell_get_rebuilds(ctx)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            ev[k][0].record(stream)
            one_step(args.warmup + k)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    st = rcell.rcell_sync(ctx)
    if st != 0:
        raise RuntimeError("timed run failed: " + rcell.rcell_last_error(ctx))
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
    rebuilds = float(np.mean(rcell.rcell_get_rebuilds(ctx) - rb0)) / args.steps
    if world > 1:
        ms = rdist_max(ms)
        torch.distributed.barrier()
    n_atoms_total = NECK_BEADS * ne
    atom_steps = n_atoms_total * md * args.steps
    value = atom_steps / (ms / 1e3)
    launches_run = rcell.rcell_info(ctx)[2]
    # deform + remap, stress, FE (bc, F, fint, update): fe_step; the sharded step
    # launches the same kernels through the individual calls
    launches_per_step = launches_run + 2 + 1 + 4

    # ---- e2e: host F out of the FE and into the r-cells, host sigma / stderr / P back,
    # host P into the FE update (the same kernels as fe_step, host copies timed) ----
    pin = lambda shape: torch.zeros(shape, dtype=torch.float64).pin_memory()  # noqa: E731
    F_h, sig_h, se_h = pin((ne, 3, 3)), pin((b - a, 6)), pin((b - a, 6))
    P_h = pin((ne, 3, 3)) if world == 1 else pin((b - a, 3, 3))
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    e2e_ms = 0.0
    k0 = args.warmup + args.steps
    for k in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rcell.fe_apply_bc(fe, lam_of(k0 + k))
        rcell.fe_get_F(fe, F_h)  # device -> host, synchronous
        rcell.rcell_set_deformation(ctx, F_h[a:b])
        rcell.rcell_run(ctx, md, navg)
        rcell.rcell_stress(ctx, sig_h, se_h, P_h)  # device -> host, synchronous
        if world == 1:
            rcell.fe_update(fe, P_h)
        else:
            P_local.copy_(P_h, non_blocking=False)
            rcell.fe_update(fe, rdist.gather_cells(P_local, bounds))
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    if world > 1:
        e2e_ms = rdist_max(e2e_ms)
    e2e = n_atoms_total * md * e2e_steps / (e2e_ms / 1e3)
    h2d = (b - a) * 72 + (ne if world == 1 else b - a) * 72
    d2h = ne * 72 + (b - a) * (48 + 48 + 72)

    # ---- per-kernel durations and the roofline of the dominant kernel ----
    prof = rcell.rcell_profile_kernels(ctx, args.profile_steps)
    Fe = np.zeros((ne, 3, 3))
    rcell.fe_get_F(fe, Fe)
    rho = NECK_DENSITY / float(np.mean(np.linalg.det(Fe)))
    bpa = (NECK_CHAIN - 1) / NECK_CHAIN
    f_ns, f_s = kg_algorithmic_flops_per_atom_step(rho, bpa)
    n_ns, n_s = md - navg, navg
    t_ns, t_s = prof["force"], prof.get("force_sample", prof["force"])
    n_local = NECK_BEADS * (b - a)
    achieved = (n_ns * f_ns + n_s * f_s) * n_local / ((n_ns * t_ns + n_s * t_s) / 1e3) / 1e12
    per_bead = K_FORCE_KG_DRAM_BYTES_PER_ATOM.get(float(tuned["skin"])) if int(tuned["tpa"]) == 0 else None
    traffic = round(per_bead * n_local) if per_bead is not None else None
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / fp32_peak, 4), "traffic": traffic,
                "kernel": "k_force<KG> (LJ + FENE/WCA forces, Verlet/Langevin, virial on sampling steps)",
                "peak_source": "measured: FFMA probe on this GPU (rcell_fp32_peak), %.2f TFLOP/s; unit-count "
                               "figure 152 SMs x 128 lanes x 2 FLOP x 2070 MHz = %.2f TFLOP/s"
                               % (fp32_peak, fp32_unit_peak_tflops())}
    Fxx = (float(Fe[:, 0, 0].min()), float(Fe[:, 0, 0].max()))
    rcell.fe_destroy(fe)
    rcell.rcell_destroy(ctx)
    out = None
    if rank == 0:
        out = {
            "metric": "atom-steps/s batched r-cell MD (necking bar, %d Kremer-Grest r-cells x 20000 beads)" % ne,
            "value": value, "unit": "atom-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": "f32 (pair math) / f64 (QR, remap, virial accumulation, FE)",
            "data": "synthetic (seeded melts, GPU-equilibrated)",
            "config": {"workload": NECK_WORKLOAD if mesh == NECK_MESH else "necking_bar_kg_%dx20000" % ne,
                       "cells": ne, "atoms_per_cell": NECK_BEADS, "atoms": n_atoms_total, "mesh": list(mesh), "imperfection": NECK_IMPERFECTION,
                       "increments_timed": [args.warmup + 1, args.warmup + args.steps], "of_increments": NECK_INC,
                       "strain_per_increment": NECK_STRAIN / NECK_INC, "md_steps_per_increment": md, "n_avg": navg,
                       "skin": tuned["skin"], "threads_per_atom": int(tuned["tpa"]),
                       "autotune": "cache hit" if hit else ("fixed by --skin-kg" if args.skin_kg > 0 else "searched"),
                       "autotune_ms_per_step": {f"skin {r['skin']} lanes {r['tpa']}": round(r["ms_per_step"], 4)
                                                for r in tuned.get("table", [])},
                       "distinct_melts": args.distinct, "l2": "flushed (256 MB write) between steps",
                       "fe_predictor": "affine, g = (X_x, 0, 0)",
                       "parallelism": f"cells split over {world} GPUs, P all-gathered" if world > 1 else "single GPU"},
            "fe_load_steps_per_s": args.steps / (ms / 1e3),
            "list_rebuilds_per_cell_per_increment": round(rebuilds, 2),
            "element_F_xx_range": Fxx,
            "e2e": {"value": e2e, "unit": "atom-steps/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "steps": e2e_steps},
            "gpu_launches": int(launches_per_step * args.steps),
            "kernel_ms": {k: round(v, 5) for k, v in prof.items()},
            "roofline": roofline,
            "clocks": clk.summary(),
            "prep_s": round(t_prep, 1),
        }
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def rdist_max(v):
    import torch
    t = torch.tensor([v], device="cuda", dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


_NECK_ORACLE_CELL = []


def neck_oracle_cell():
    """One of the necking bar's 20 000-bead melts (host-generated, the first of the
    distinct melts), relaxed by 100 iterations of the oracle's FIRE so that MD at
    the production time step keeps every FENE bond below R0 (a pushed-off melt that
    has not gone through the GPU's soft start stretches one past R0 within a few
    steps).  Input preparation of the timing sample, computed once."""
    import oracle
    if not _NECK_ORACLE_CELL:
        x, H, bonds = inputs.kg_melt(NECK_BEADS // NECK_CHAIN, NECK_CHAIN, NECK_DENSITY, seed=5 * 1000)
        x, _ = oracle.fire_minimize(oracle.pot_kg(), x, H, 1.0, 1.0, 0.001, 0.01, 100, bonds=bonds, units=1,
                                    dmax=0.05)
        x = inputs.to_f32(np.mod(x, H[0, 0]))
        v = inputs.to_f32(inputs.maxwell(len(x), 1.0, 0.3, 1, 5))
        _NECK_ORACLE_CELL.append((x, v, H, bonds))
    return _NECK_ORACLE_CELL[0]


def neck_oracle_sample(threads, md_steps):
    """Time the FP64 oracle on a bounded sample of the necking bar: `threads` copies
    of one of its 20 000-bead melts (neck_oracle_cell), md_steps MD steps each with
    the production parameters, one cell (with its own Langevin stream) per host
    thread.  Returns (atom_steps, seconds)."""
    import concurrent.futures as cf

    import oracle
    x, v, H, bonds = neck_oracle_cell()
    pot = oracle.pot_kg()
    mdp = oracle.MD(1, 1.0, 0.3, 2.0, 0.005, 11)

    def one(c):
        oracle.md_run(pot, mdp, x, v, H, bonds=bonds, cell=c, ev=0, n_steps=md_steps, n_avg=md_steps)

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, range(threads)))
    return threads * NECK_BEADS * md_steps, time.perf_counter() - t0


def neck_cpu_baseline(target_s=15.0):
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    try:
        a, t = neck_oracle_sample(1, 1)
        steps = int(max(1, min(30, target_s / max(t, 1e-3))))
        a, t = neck_oracle_sample(threads, steps)
    except Exception as e:  # the GPU line is printed with the reason instead
        return {"value": None, "unit": "atom-steps/s", "cores": threads, "kind": "oracle", "error": str(e)[:200]}
    return {"value": a / t, "unit": "atom-steps/s", "cores": threads, "kind": "oracle",
            "sample": f"{threads} copies of one 20000-bead necking-bar melt (FIRE-relaxed, 100 iterations), "
                      f"{steps} MD steps each with the production parameters, one cell per host thread, FP64"}


def run_ours(args):
    import torch

    from paper_1902_09171_gb300 import build, rcell

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    rcell.load()
    stream = torch.cuda.Stream()  # a dedicated stream: library kernels, flushes and events all on it
    torch.cuda.set_stream(stream)
    X, conn, mask, val = mesh(args.element)
    n_total = len(conn)  # one r-cell per element
    # weak scaling: each rank runs a full copper bar (its own independent cells)
    cells = make_cells(n_total, seed0=1000 + rank * n_total)
    prm = rcell.params_sc_cu(tau=0.1, kT=KT, dt=0.002, seed=12345 + rank, skin=args.skin)
    ctx = rcell.rcell_create(prm, cells, stream=stream)
    if args.tpa >= 0:
        rcell.rcell_set_tuning(ctx, args.tpa, -1)
    rho0, dt_fe, damp_fe, hg_fe = fe_params()
    if args.element == "tet4":  # tetrahedra: shorter altitudes, half the step; no hourglass control
        fe = rcell.fe_create_tet4(X, conn, mask, val, rho0, 0.5 * dt_fe, damp_fe, stream=stream)
    else:
        fe = rcell.fe_create(X, conn, mask, val, rho0, dt_fe, damp_fe, hg_fe, stream=stream)
    n_atoms = sum(len(c["x0"]) for c in cells)
    md = args.md_steps
    navg = min(N_AVG, md // 2)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def one_step(k):
        lam = STRAIN * ((k % N_INC) + 1) / N_INC
        rcell.fe_step(fe, ctx, lam, md, navg, None)

    for k in range(args.warmup):
        one_step(k)
    torch.cuda.synchronize()
    if rcell.rcell_sync(ctx) != 0:
        raise RuntimeError("warm-up failed: " + rcell.rcell_last_error(ctx))
    fp32_peak = rcell.rcell_fp32_peak(stream)  # roofline denominator, measured with warm clocks
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            ev[k][0].record(stream)
            one_step(args.warmup + k)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    st = rcell.rcell_sync(ctx)
    if st != 0:
        raise RuntimeError("timed run failed: " + rcell.rcell_last_error(ctx))
    ms = sum(a.elapsed_time(b) for a, b in ev)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        torch.distributed.barrier()
    atom_steps = n_atoms * md * args.steps * world
    value = atom_steps / (ms / 1e3)
    launches_run = rcell.rcell_info(ctx)[2]
    launches_per_step = launches_run + 2 + 1 + 4  # deform + remap, stress, FE (bc, F, fint, update)

    # ---- e2e: host F in, host sigma / stderr / P out, through the r-cell API ----
    pin = lambda shape: torch.zeros(shape, dtype=torch.float64).pin_memory()  # noqa: E731
    F_h = pin((n_total, 3, 3))
    sig_h, se_h, P_h = pin((n_total, 6)), pin((n_total, 6)), pin((n_total, 3, 3))
    e2e_ms = 0.0
    for k in range(args.steps):
        lam = STRAIN * ((k % N_INC) + 1) / N_INC
        F_h.copy_(torch.from_numpy(np.tile(np.diag([1 + lam, 1 - 0.3 * lam, 1 - 0.3 * lam]), (n_total, 1, 1))))
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rcell.rcell_set_deformation(ctx, F_h)
        rcell.rcell_run(ctx, md, navg)
        rcell.rcell_stress(ctx, sig_h, se_h, P_h)
        e2e_ms += (time.perf_counter() - t0) * 1e3
    if world > 1:
        t = torch.tensor([e2e_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e = atom_steps / (e2e_ms / 1e3)

    # ---- per-kernel durations (CUDA events around each launch, same stream) ----
    prof = rcell_kernel_profile(ctx, stream, n_steps=args.profile_steps)
    rho = NC ** 3 * 4 / (NC * A_LAT) ** 3
    _, force_ns, force_s = sc_algorithmic_flops_per_atom_step(rho)
    # one load increment: md - navg force launches without a stress sample, navg with one
    n_ns, n_s = md - navg, navg
    t_ns, t_s = prof["force"], prof.get("force_sample", prof["force"])
    achieved = (n_ns * force_ns + n_s * force_s) * n_atoms / ((n_ns * t_ns + n_s * t_s) / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / fp32_peak, 4), "traffic": K_FORCE_DRAM_BYTES if (args.skin == 1.5 and args.element == "hex8") else None,
                "kernel": "k_force<SC> (force + Verlet/Langevin (+ virial on sampling steps))",
                "peak_source": "measured: FFMA probe on this GPU (rcell_fp32_peak), %.2f TFLOP/s; unit-count "
                               "figure 152 SMs x 128 lanes x 2 FLOP x 2070 MHz = %.2f TFLOP/s"
                               % (fp32_peak, fp32_unit_peak_tflops())}

    rcell.fe_destroy(fe)
    rcell.rcell_destroy(ctx)
    out = None
    if rank == 0:
        out = {
            "metric": "atom-steps/s batched r-cell MD (copper bar, Sutton-Chen EAM, %d x 4000 atoms)" % n_total,
            "value": value, "unit": "atom-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (pair math) / f64 (QR, remap, virial accumulation, FE)", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.element == "hex8" else "copper_bar_sc_eam_tet4_%dx4000" % n_total,
                       "element": args.element, "cells": n_total * world, "atoms_per_cell": NC ** 3 * 4,
                       "md_steps_per_increment": md, "n_avg": navg, "mesh": list(MESH), "l2": "flushed (256 MB write)",
                       "parallelism": f"{world} independent cell batches" if world > 1 else "single GPU"},
            "fe_load_steps_per_s": args.steps / (ms / 1e3),
            "e2e": {"value": e2e, "unit": "atom-steps/s", "h2d_bytes_per_step": int(F_h.numel() * 8),
                    "d2h_bytes_per_step": int((sig_h.numel() + se_h.numel() + P_h.numel()) * 8)},
            "gpu_launches": int(launches_per_step * args.steps),
            "kernel_ms": {k: round(v, 5) for k, v in prof.items()},
            "roofline": roofline,
            "clocks": clk.summary(),
        }
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def rcell_kernel_profile(ctx, stream, n_steps=100):
    """Mean duration of one launch of each kernel class over n_steps MD steps,
    from CUDA events recorded around every launch on the library's stream."""
    from paper_1902_09171_gb300 import rcell
    return rcell.rcell_profile_kernels(ctx, n_steps)


def run_oracle_sample(n_cells_sample, md_steps, threads):
    """Time the FP64 oracle on a bounded sample of the workload: n_cells_sample
    r-cells of the copper bar, one load increment each (QR, remap, md_steps MD
    steps, stress), one cell per host thread.  Returns (atom_steps, seconds)."""
    import concurrent.futures as cf

    import oracle

    cells = make_cells(n_cells_sample)
    pot = oracle.pot_sc(SC["eps"], SC["a"], SC["rc"], SC["n"], SC["m"], SC["c"])
    mdp = oracle.MD(0, MASS, KT, 0.1, 0.002, 12345)
    lam = STRAIN / N_INC
    F = np.diag([1 + lam, 1.0, 1.0])

    def one(c):
        Q, R = oracle.qr(F)
        x = oracle.remap(cells[c]["x0"], oracle.delta_R(R, np.eye(3)))
        _, _, _, ss, _, _ = oracle.md_run(pot, mdp, x, cells[c]["v0"], R @ cells[c]["H0"], cell=c, ev=0,
                                          n_steps=md_steps, n_avg=max(1, md_steps // 2))
        s_fem = np.array([oracle.rotate_pk1(Q, F, s)[0] for s in ss])
        return s_fem.mean(0)

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, range(n_cells_sample)))
    dt = time.perf_counter() - t0
    return n_cells_sample * len(cells[0]["x0"]) * md_steps, dt


def cpu_baseline(target_s=15.0):
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    threads = min(cores, MESH[0] * MESH[1] * MESH[2])
    # calibrate: one cell, 2 steps
    a, t = run_oracle_sample(1, 2, 1)
    per_atom_step = t / a
    steps = max(2, int(target_s * threads / (per_atom_step * 4000 * threads)))
    steps = min(steps, MD_STEPS)
    a, t = run_oracle_sample(threads, steps, threads)
    return {"value": a / t, "unit": "atom-steps/s", "cores": threads, "kind": "oracle",
            "sample": f"{threads} of the 32 copper-bar r-cells (4000 atoms, Sutton-Chen), one increment of "
                      f"{steps} MD steps each (QR, remap, MD, stress), one cell per host thread, FP64"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    if args.workload == "necking_bar":
        threads, md = cores, 2
        for _ in range(args.warmup):
            neck_oracle_sample(threads, 1)
        tot_a, tot_t = 0, 0.0
        for _ in range(args.steps):
            a, t = neck_oracle_sample(threads, md)
            tot_a += a
            tot_t += t
        value = tot_a / tot_t
        return {"impl": "reference",
                "metric": "atom-steps/s batched r-cell MD (necking bar, %d Kremer-Grest r-cells x 20000 beads)" % int(np.prod(NECK_MESH)),
                "value": value, "unit": "atom-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": tot_t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": NECK_WORKLOAD, "cells": int(np.prod(NECK_MESH)), "atoms_per_cell": NECK_BEADS},
                "cpu_baseline": {"value": value, "unit": "atom-steps/s", "cores": threads, "kind": "oracle",
                                 "sample": f"each step: {threads} copies of one 20000-bead melt (FIRE-relaxed) x {md} "
                                           f"MD steps (FP64 oracle, one cell per host thread)"},
                "e2e": {"value": value, "unit": "atom-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    threads = min(cores, MESH[0] * MESH[1] * MESH[2])
    md = 3
    for _ in range(args.warmup):
        run_oracle_sample(threads, 1, threads)
    tot_a, tot_t = 0, 0.0
    for _ in range(args.steps):
        a, t = run_oracle_sample(threads, md, threads)
        tot_a += a
        tot_t += t
    value = tot_a / tot_t
    return {"impl": "reference", "metric": "atom-steps/s batched r-cell MD (copper bar, Sutton-Chen EAM, 32 x 4000 atoms)",
            "value": value, "unit": "atom-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot_t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": MESH[0] * MESH[1] * MESH[2], "atoms_per_cell": NC ** 3 * 4},
            "cpu_baseline": {"value": value, "unit": "atom-steps/s", "cores": threads, "kind": "oracle",
                             "sample": f"each step: {threads} r-cells x {md} MD steps (FP64 oracle)"},
            "e2e": {"value": value, "unit": "atom-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _kg_melt_job(n_chains, chain_len, density, seed, pushoff):
    return inputs.kg_melt(n_chains, chain_len, density, seed=seed, pushoff_iters=pushoff)


def run_kg_bar(args):
    """Uneven Kremer-Grest r-cells (sizes U[5000, 20000] beads in chains of 50, seed 3)
    on a 4x4x4 hex mesh, one FE increment = one bench step (uniaxial tension to 30 %
    in 60 increments, 1000 MD steps each, last 500 averaged)."""
    import torch

    from paper_1902_09171_gb300 import build, pipeline, rcell
    build.build()
    rcell.load()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sizes = inputs.uniform_sizes(args.kg_cells, 5000, 20000, 50, 3)
    # the seeded melts (NumPy push-off of overlapping beads) in a spawned process pool
    import multiprocessing as mp
    jobs = [(int(n) // 50, 50, 0.85, 300 + k, args.pushoff) for k, n in enumerate(sizes)]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        melts = pool.starmap(_kg_melt_job, jobs)
    cells = [dict(H0=H, x0=inputs.to_f32(x), bonds=b) for x, H, b in melts]
    # melt preparation (as for the surrogate data): displacement-limited soft start,
    # then equilibration with the production parameters; the timed increments
    # start from these states
    soft = rcell.params_kg(tau=0.5, kT=1.0, dt=0.002, seed=3, max_step=0.02)
    ctx = rcell.rcell_create(soft, cells, stream=stream)
    rcell.rcell_run(ctx, 2000, 0)
    st = rcell.rcell_sync(ctx)
    if st != 0:
        raise RuntimeError("KG soft start: " + rcell.rcell_last_error(ctx))
    eq = []
    for k, c in enumerate(cells):
        x, v, _ = rcell.rcell_get_atoms(ctx, k, len(c["x0"]))
        eq.append(dict(H0=c["H0"], x0=x, v0=v, bonds=c["bonds"]))
    rcell.rcell_destroy(ctx)
    # autotuned Verlet skin and lanes per atom (timed on the bar's own cells)
    from paper_1902_09171_gb300 import autotune
    make = lambda skin: rcell.params_kg(skin=skin)  # noqa: E731
    tuned, hit = autotune.tune(make, eq, stream, skins=KG_BAR_SKINS, tpas=KG_BAR_TPAS, n_steps=400, n_avg=200)
    ctx = rcell.rcell_create(make(tuned["skin"]), eq, stream=stream)
    rcell.rcell_set_tuning(ctx, int(tuned["tpa"]), 1)
    rcell.rcell_run(ctx, 2000, 0)
    st = rcell.rcell_sync(ctx)
    if st != 0:
        raise RuntimeError("KG equilibration: " + rcell.rcell_last_error(ctx))
    L = float(np.mean([c["H0"][0, 0] for c in cells]))
    m = int(round(len(cells) ** (1 / 3)))
    X, conn = inputs.hex_mesh(m, m, m, m * L, m * L, m * L)
    mask, val = inputs.uniaxial_bc(X, m * L)
    fe = rcell.fe_create(X, conn, mask, val, 0.85, 2.0, 1.0, 1.0, stream=stream)
    md = args.md_steps
    for k in range(args.warmup):
        rcell.fe_step(fe, ctx, 0.3 * (k + 1) / 60, md, md // 2, None)
    torch.cuda.synchronize()
    st = rcell.rcell_sync(ctx)
    if st != 0:
        raise RuntimeError("KG warm-up increments: " + rcell.rcell_last_error(ctx))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    rb0 = rcell.rcell_get_rebuilds(ctx)
    for k in range(args.steps):
        ev[k][0].record(stream)
        rcell.fe_step(fe, ctx, 0.3 * (args.warmup + k + 1) / 60, md, md // 2, None)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    st = rcell.rcell_sync(ctx)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    rebuilds = (rcell.rcell_get_rebuilds(ctx) - rb0) / float(args.steps)  # per cell and increment
    prof = rcell.rcell_profile_kernels(ctx, args.profile_steps)
    n_atoms = int(sizes.sum())
    Fe = np.zeros((len(cells), 3, 3))
    rcell.fe_get_F(fe, Fe)
    out = {"metric": "atom-steps/s batched r-cell MD (Kremer-Grest bar, uneven cells)",
           "value": n_atoms * md * args.steps / (ms / 1e3), "unit": "atom-steps/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "status": rcell.STATUS[st], "data": "synthetic",
           "config": {"workload": f"kg_bar_{len(cells)}_cells_5k_20k", "atoms": n_atoms, "md_steps": md,
                      "skin": tuned["skin"], "threads_per_atom": int(tuned["tpa"]),
                      "autotune": "cache hit" if hit else "searched", "autotune_table": tuned.get("table")},
           "fe_load_steps_per_s": args.steps / (ms / 1e3),
           "element_F_xx_range": [float(Fe[:, 0, 0].min()), float(Fe[:, 0, 0].max())],
           "list_rebuilds_per_cell_per_increment": round(float(np.mean(rebuilds)), 2),
           "kernel_ms": {k: round(v, 5) for k, v in prof.items()}}
    rcell.fe_destroy(fe)
    rcell.rcell_destroy(ctx)
    return out


def run_kg_statics(args):
    """The paper's molecular-statics r-cell route (Sec. 2.2, Eqs. CGPR1-CGPR3, PK1)
    on amorphous Kremer-Grest cells: 32 cells of 5000 beads, quenched to a local
    energy minimum; one bench step = one load increment of uniaxial stretch (0.5 %)
    through rcell_set_deformation (the Cauchy-Born guess), FIRE relaxation of every
    cell to max |f| < 1e-2 and the pair-sum first Piola-Kirchhoff stress."""
    import torch

    import oracle
    from paper_1902_09171_gb300 import build, rcell
    build.build()
    rcell.load()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    n_cells, f_tol, dt0, dt_max, dmax, max_iter = 32, 1e-2, 0.005, 0.05, 0.05, 50000
    cells = inputs.kg_cells(n_cells, 100, 50, 0.85, seed=400, n_distinct=4)
    soft = rcell.params_kg(tau=0.5, kT=1.0, dt=0.002, seed=4, max_step=0.02)
    ctx = rcell.rcell_create(soft, cells, stream=stream)
    rcell.rcell_run(ctx, 1000, 0)
    glass = []
    for k, c in enumerate(cells):
        x, _, _ = rcell.rcell_get_atoms(ctx, k, len(c["x0"]))
        glass.append(dict(H0=c["H0"], x0=x, v0=np.zeros_like(x), bonds=c["bonds"]))
    rcell.rcell_destroy(ctx)
    prm = rcell.params_kg(skin=0.3)
    ctx = rcell.rcell_create(prm, glass, stream=stream)
    rcell.rcell_minimize(ctx, max_iter, f_tol, dt0, dt_max, dmax)  # the unstrained minimum
    n_atoms = np.array([len(c["x0"]) for c in glass])
    sig = torch.zeros((n_cells, 6), dtype=torch.float64, device="cuda")

    def increment(k):
        eps = 0.005 * (k + 1)
        rcell.rcell_set_deformation(ctx, np.tile(np.diag([1.0 + eps, 1.0, 1.0]), (n_cells, 1, 1)))
        it = rcell.rcell_minimize(ctx, max_iter, f_tol, dt0, dt_max, dmax)
        rcell.rcell_stress_static(ctx, sig)
        return it

    for k in range(args.warmup):
        increment(k)
    torch.cuda.synchronize()
    work, ms, iters = 0, 0.0, []
    for k in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it = increment(args.warmup + k)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        iters.append(int(it.max()))
        work += int((n_atoms * (np.maximum(it, 0) + 1)).sum())  # force evaluations of cells still moving
    st = rcell.rcell_sync(ctx)
    value = work / (ms / 1e3)
    # oracle on a bounded sample: one cell, the same relaxation, at most 30 iterations
    pot = oracle.pot_kg()
    H, _, _ = rcell.rcell_get_box(ctx, 0)
    x0 = rcell.rcell_get_atoms(ctx, 0, int(n_atoms[0]))[0] @ np.diag([1.005, 1.0, 1.0]).T
    t0 = time.perf_counter()
    oracle.fire_minimize(pot, x0, np.diag([1.005, 1.0, 1.0]) @ H, 1.0, f_tol, dt0, dt_max, 30,
                         bonds=glass[0]["bonds"], units=1, dmax=dmax)
    cpu_s = time.perf_counter() - t0
    out = {"metric": "atom force-evaluations/s, batched r-cell molecular statics (Kremer-Grest glass)",
           "value": value, "unit": "atom-evaluations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms / args.steps, "higher_is_better": True, "status": rcell.STATUS[st], "data": "synthetic",
           "dtype": "f32 (pair math) / f64 (cell sums, stress)",
           "config": {"workload": f"kg_statics_{n_cells}x5000", "f_tol": f_tol, "dmax": dmax, "strain_per_increment": 0.005,
                      "fire_iterations_per_increment": iters},
           "fe_load_steps_per_s": args.steps / (ms / 1e3),
           "cpu_baseline": {"value": int(n_atoms[0]) * 31 / cpu_s, "unit": "atom-evaluations/s", "cores": 1,
                            "kind": "oracle", "sample": "one 5000-bead cell, 30 FIRE iterations, FP64"}}
    rcell.rcell_destroy(ctx)
    return out


def run_surrogate_train(args):
    """The learned surrogate's tensor-core kernels at the training shapes (4
    members, batch 4096, 60 increments, synthetic features and targets): one
    bench step = one AdamW step of every member side by side (whole-forward
    tcgen05 kernel with the BPTT tape, whole-backward tcgen05 kernel, tcgen05
    weight and bias gradients).  The roofline is that of the slower of the two
    fused kernels, timed by sur_profile_step; the ensemble prediction of the
    same batch is timed beside it."""
    import torch

    from paper_1902_09171_gb300 import build, rcell
    from paper_1902_09171_gb300 import surrogate as S
    build.build()
    rcell.load()
    st = torch.cuda.Stream()
    torch.cuda.set_stream(st)
    B, T, K = 4096, 60, 4
    rng = np.random.default_rng(0)
    U = torch.tensor(rng.standard_normal((B, T, 15)), dtype=torch.float32, device="cuda")
    Y = torch.tensor(rng.standard_normal((B, T, 6)), dtype=torch.float32, device="cuda")
    s = S.sur_create(K, B, T, 1, stream=st)
    for _ in range(args.warmup):
        S.sur_train_step(s, U, Y, 1e-3, want_loss=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        S.sur_train_step(s, U, Y, 1e-3, want_loss=False)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    P = torch.zeros((K, B, T, 6), dtype=torch.float32, device="cuda")
    for _ in range(3):
        S.sur_predict(s, U, P)
    torch.cuda.synchronize()
    n_pred = 10
    e0.record(st)
    for _ in range(n_pred):
        S.sur_predict(s, U, P)
    e1.record(st)
    torch.cuda.synchronize()
    ms_pred = e0.elapsed_time(e1) / n_pred
    phases = [S.sur_profile_step(s, U, Y) for _ in range(3)][-1]
    err = S.sur_sync(s)
    S.sur_destroy(s)
    flop_fwd = 2.0 * B * T * (144 * 256 + 2 * 256 * 256 + 256 * 144) * K
    try:
        peaks = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")))
        peak, peak_src = float(peaks["bf16_tflops"]), "measured bf16 burst (MEASURED_PEAKS.json)"
    except (OSError, ValueError, KeyError):
        peak, peak_src = 1900.0, "fallback: 1.9 PFLOP/s bf16 burst of an earlier GB300 measurement"
    # both fused kernels run the four products of every step of every member:
    # the forward's FLOPs (the backward skips nothing but dZ of step 0)
    dom = "backward" if phases["backward"] >= phases["forward_tape"] else "forward_tape"
    achieved = flop_fwd / (phases[dom] / 1e3) / 1e12
    return {"metric": "surrogate training throughput (sequence-increments/s, 4-member ensemble)",
            "value": B * T * K / (ms / 1e3), "unit": "sequence-increments/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "status": err, "data": "synthetic",
            "dtype": "bf16 operands, f32 accumulation / master weights",
            "config": {"workload": "surrogate_train_4x4096x60", "members": K, "batch": B, "increments": T},
            "train_tflops": 3 * flop_fwd / (ms / 1e3) / 1e12,
            "predict_ms": ms_pred, "predict_tflops": round(flop_fwd / (ms_pred / 1e3) / 1e12, 2),
            "phase_ms": {k: round(v, 4) for k, v in phases.items()},
            "roofline": {"bound": "tensor", "achieved": round(achieved, 2), "peak": peak, "unit": "TFLOP/s",
                         "frac": round(achieved / peak, 4), "traffic": None,
                         "kernel": "k_backward_ws (BPTT data gradients)" if dom == "backward"
                         else "k_forward_ws (forward with the BPTT tape)",
                         "peak_source": peak_src}}


def run_kg_tensile(args):
    """The paper's direct periodic-box MD tensile comparison (Sec. 3.2): 32
    Kremer-Grest cells of 5000 beads at T = 0.1 (below the glass transition),
    stretched along x at the engineering strain rate 0.01 / tau with lateral
    contraction (1 + eps)^-1/2, a new deformation every 50 MD steps (dt 0.005),
    to 15 % strain.  One bench step = one chunk (deformation, 50 MD steps, stress)."""
    import torch

    from paper_1902_09171_gb300 import build, pipeline, rcell
    build.build()
    rcell.load()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    n_cells, rate, dt, chunk = 32, 0.01, 0.005, 50
    n_chunks = int(round(0.15 / (rate * dt * chunk)))
    ctx0, cells = pipeline.prepare_kg_batch(n_cells, stream=stream)
    rcell.rcell_destroy(ctx0)
    ctx = rcell.rcell_create(rcell.params_kg(kT=0.1, seed=7), cells, stream=stream)
    rcell.rcell_run(ctx, 2000, 0)  # cool to T = 0.1
    for _ in range(args.warmup):
        rcell.rcell_run(ctx, chunk, chunk)
    st = rcell.rcell_sync(ctx)
    if st != 0:
        raise RuntimeError("KG tensile preparation: " + rcell.rcell_last_error(ctx))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    eps, sig = pipeline.pbc_tensile(ctx, rate, dt, n_chunks, chunk)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = rcell.rcell_sync(ctx)
    n_atoms = rcell.rcell_info(ctx)[1]
    sxx = sig[:, :, 0].mean(1)
    out = {"metric": "atom-steps/s, periodic-box MD tensile test (Kremer-Grest glass, T = 0.1)",
           "value": n_atoms * chunk * n_chunks / (ms / 1e3), "unit": "atom-steps/s", "n_gpus": 1,
           "steps": n_chunks, "warmup": args.warmup, "ms_per_step": ms / n_chunks, "higher_is_better": True,
           "status": rcell.STATUS[st], "data": "synthetic", "dtype": "f32 (pair math) / f64 (stress)",
           "config": {"workload": f"kg_tensile_{n_cells}x5000", "strain_rate": rate, "md_steps_per_chunk": chunk,
                      "final_strain": float(eps[-1])},
           "stress_xx_at_strain": {f"{e:.3f}": round(float(v), 4) for e, v in zip(eps[4::6], sxx[4::6])},
           "strain_at_max_stress": float(eps[int(np.argmax(sxx))])}
    rcell.rcell_destroy(ctx)
    return out


def run_surrogate_fe(args):
    """The learned surrogate against plain r-cell MD on an FE bar of Kremer-Grest
    r-cells (5000 beads each): S1 data generation through batched r-cells, BF16
    training of a 4-member ensemble, then the same FE load history with all-MD
    r-cells and with the surrogate + 2 % ensemble-spread MD fallback."""
    import torch

    from paper_1902_09171_gb300 import build, pipeline, rcell
    from paper_1902_09171_gb300 import surrogate as S
    build.build()
    rcell.load()
    st = torch.cuda.Stream()
    torch.cuda.set_stream(st)
    NP, T, NMD, NAVG, K = args.paths, 60, 400, 300, 4
    t0 = time.time()
    ctx, _ = pipeline.prepare_kg_batch(NP, stream=st)
    F = inputs.strain_paths(NP, T, seed=11)
    U, Y, data_steps = pipeline.generate_dataset(ctx, F, NMD, NAVG, stream=st)
    rcell.rcell_destroy(ctx)
    torch.cuda.synchronize()
    t_data = time.time() - t0
    ntr = int(NP * 0.9)
    sur = S.sur_create(K, NP, T, seed=5, stream=st)
    us, ys = pipeline.feature_scales(U[:ntr], Y[:ntr])
    S.sur_set_scaling(sur, us, ys)
    t0 = time.time()
    pipeline.train(sur, U[:ntr].contiguous(), Y[:ntr].contiguous(), args.train_steps, lr=1e-3, n_members=K)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    s_floor = 0.5 * float(ys[0])  # half the RMS stress of the training data
    err_ho, spread_q = pipeline.relative_error(sur, U[ntr:].contiguous(), Y[ntr:].contiguous(), K, s_floor=s_floor,
                                               with_spread=True)
    ne = 32
    ctx_md, cells = pipeline.prepare_kg_batch(ne, stream=st, seed=21)
    # the surrogate bar starts from the same states with the same Langevin seed as the
    # all-MD bar (prepare_kg_batch's production seed is seed + 1); a third all-MD bar
    # with another seed states the MD noise of the axial stress curve
    ctx_sg = rcell.rcell_create(rcell.params_kg(seed=22), cells, stream=st)
    ctx_nz = rcell.rcell_create(rcell.params_kg(seed=99), cells, stream=st)
    L = cells[0]["H0"][0, 0]
    X, conn = inputs.hex_mesh(8, 2, 2, 8 * L, 2 * L, 2 * L)
    mask, val = inputs.uniaxial_bc(X, 8 * L)
    fe_md = rcell.fe_create(X, conn, mask, val, 0.85, 2.0, 1.0, 1.0, stream=st)
    fe_sg = rcell.fe_create(X, conn, mask, val, 0.85, 2.0, 1.0, 1.0, stream=st)
    fe_nz = rcell.fe_create(X, conn, mask, val, 0.85, 2.0, 1.0, 1.0, stream=st)
    for fe in (fe_md, fe_sg, fe_nz):
        rcell.fe_set_predictor(fe, axial_predictor(X))
    lams = [0.3 * (k + 1) / 60 for k in range(60)]
    res = pipeline.fe_compare(ctx_md, ctx_sg, sur, fe_md, fe_sg, K, lams, NMD, NAVG, s_floor=s_floor, stream=st)
    nz = pipeline.fe_compare_md_only(ctx_nz, fe_nz, lams, NMD, NAVG, stream=st)
    a0, a2 = np.array(res["axial_md"]), np.array(nz["axial_md"])
    md_noise = float(np.abs(a0 - a2).max() / max(np.abs(a0).max(), 1e-30))
    for h in (fe_md, fe_sg, fe_nz):
        rcell.fe_destroy(h)
    for c in (ctx_md, ctx_sg, ctx_nz):
        rcell.rcell_destroy(c)
    S.sur_destroy(sur)
    return {"metric": "FE load-steps/s, surrogate + MD fallback vs all-MD r-cells",
            "value": len(lams) / (res["ms_sg"] / 1e3), "unit": "load-steps/s", "n_gpus": 1,
            "all_md_value": len(lams) / (res["ms_md"] / 1e3), "speedup": res["ms_md"] / res["ms_sg"],
            "max_rel_axial_stress_dev": res["max_rel_dev"], "md_noise_max_rel_axial_dev": md_noise,
            "md_fraction": res["md_fraction"], "n_md_per_increment": res["n_md"],
            "axial_md": res["axial_md"], "axial_sg": res["axial_sg"],
            "heldout_rel_rms_error": err_ho, "heldout_spread_quantiles_10_50_90_99": spread_q,
            "data_atom_steps": data_steps, "data_s": t_data, "train_s": t_train, "higher_is_better": True,
            "data": "synthetic",
            "config": {"workload": f"kg_surrogate_fe_8x2x2_{NP}_paths", "paths": NP, "increments": T,
                       "md_steps": NMD, "n_avg": NAVG, "members": K, "train_steps": args.train_steps,
                       "spread_on": 0.02, "spread_off": 0.01, "s_floor": s_floor,
                       "fe_predictor": "affine, g = (X_x, 0, 0)"}}


def run_surrogate_fe_cu(args):
    """The learned surrogate against plain r-cell MD on the copper bar: the
    surrogate's training set of copper-bar-style r-cells read as the copper bar's
    own Sutton-Chen r-cells (4000 atoms, 300 K).  Data: `--paths` cells driven along
    seeded bar-like deformation histories (25 increments, --sur-md MD steps each,
    stress averaged over the second half) through the batched r-cell engine;
    BF16 training of a 4-member ensemble on 90 % of them; then the copper bar's
    FE load history (8 x 2 x 2 hexahedra, 32 r-cells, 5 % in 25 increments, affine
    load predictor, gradient-flow damping) with
    all-MD r-cells (fe_step) and with the surrogate + 2 % ensemble-spread MD
    fallback (fe_step_surrogate: MD forced on the first 2 increments, trip above
    2 %, release below 1 %, missed increments replayed on return).  Both bars
    start from the same cells with the same Langevin seed; a third all-MD bar with
    another seed states the MD noise of the axial stress curve."""
    import torch

    from paper_1902_09171_gb300 import build, pipeline, rcell
    from paper_1902_09171_gb300 import surrogate as S
    build.build()
    rcell.load()
    st = torch.cuda.Stream()
    torch.cuda.set_stream(st)
    NP, T, K = args.paths, N_INC, 4
    NMD = args.sur_md
    NAVG = NMD // 2
    t0 = time.time()
    prm = rcell.params_sc_cu(tau=0.1, kT=KT, dt=0.002, seed=77)
    ctx = rcell.rcell_create(prm, make_cells(NP, seed0=5000), stream=st)
    F = inputs.bar_strain_paths(NP, T, seed=13, max_axial=0.08, max_shear=0.02, max_lateral=0.03)
    U, Y, data_steps = pipeline.generate_dataset(ctx, F, NMD, NAVG, stream=st)
    rcell.rcell_destroy(ctx)
    torch.cuda.synchronize()
    t_data = time.time() - t0
    ntr = int(NP * 0.9)
    sur = S.sur_create(K, max(NP, 32), T, seed=5, stream=st)
    us, ys = pipeline.feature_scales(U[:ntr], Y[:ntr])
    S.sur_set_scaling(sur, us, ys)
    t0 = time.time()
    pipeline.train(sur, U[:ntr].contiguous(), Y[:ntr].contiguous(), args.train_steps, lr=1e-3, n_members=K)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    s_floor = args.s_floor if args.s_floor > 0 else 0.5 * float(ys[0])  # half the RMS training stress
    err_ho, spread_q = pipeline.relative_error(sur, U[ntr:].contiguous(), Y[ntr:].contiguous(), K, s_floor=s_floor,
                                               with_spread=True)
    X, conn, mask, val = mesh("hex8")
    ne = len(conn)
    rho0, dt_fe, damp_fe, hg_fe = fe_params()
    bars = []
    for seed in (21, 21, 22):  # all-MD, surrogate (same cells, same seed), all-MD with another seed
        c = rcell.rcell_create(rcell.params_sc_cu(tau=0.1, kT=KT, dt=0.002, seed=seed), make_cells(ne), stream=st)
        # gradient-flow FE (c dt / 2 = 1: no memory of the previous velocity), so that the
        # thermal stress of the 300 K cells relaxes without ringing
        fe = rcell.fe_create(X, conn, mask, val, rho0, dt_fe, 2.0 / dt_fe, hg_fe, stream=st)
        rcell.fe_set_predictor(fe, axial_predictor(X))
        bars.append((c, fe))
    lams = [STRAIN * (k + 1) / N_INC for k in range(N_INC)]
    res = pipeline.fe_compare(bars[0][0], bars[1][0], sur, bars[0][1], bars[1][1], K, lams, NMD, NAVG,
                              spread_on=0.02, spread_off=0.01, s_floor=s_floor, stream=st)
    Fe = np.zeros((ne, 3, 3))
    rcell.fe_get_F(bars[0][1], Fe)
    noise = pipeline.fe_compare_md_only(bars[2][0], bars[2][1], lams, NMD, NAVG, stream=st)
    a0, a2 = np.array(res["axial_md"]), np.array(noise["axial_md"])
    md_noise = float(np.abs(a0 - a2).max() / max(np.abs(a0).max(), 1e-30))
    for c, fe in bars:
        rcell.fe_destroy(fe)
        rcell.rcell_destroy(c)
    S.sur_destroy(sur)
    return {"metric": "FE load-steps/s, surrogate + MD fallback vs all-MD r-cells (copper bar)",
            "value": len(lams) / (res["ms_sg"] / 1e3), "unit": "load-steps/s", "n_gpus": 1,
            "all_md_value": len(lams) / (res["ms_md"] / 1e3), "speedup": res["ms_md"] / res["ms_sg"],
            "max_rel_axial_stress_dev": res["max_rel_dev"], "md_noise_max_rel_axial_dev": md_noise,
            "md_fraction": res["md_fraction"], "md_cell_increments": int(sum(res["n_md"])),
            "all_md_cell_increments": ne * len(lams),
            "heldout_rel_rms_error": err_ho, "heldout_spread_quantiles_10_50_90_99": spread_q,
            "axial_md": res["axial_md"], "axial_sg": res["axial_sg"], "n_md_per_increment": res["n_md"],
            "element_F_range": {"xx": [float(Fe[:, 0, 0].min()), float(Fe[:, 0, 0].max())],
                                "max_abs_shear": float(np.abs(Fe - np.diag(np.diag(Fe[0])) * 0 - np.eye(3))[:, [0, 0, 1, 2], [1, 2, 0, 0]].max())},
            "data_atom_steps": data_steps, "data_s": t_data, "train_s": t_train, "higher_is_better": True,
            "data": "synthetic",
            "config": {"workload": f"cu_surrogate_fe_8x2x2_{NP}_paths", "paths": NP, "increments": T,
                       "md_steps": NMD, "n_avg": NAVG, "members": K, "train_steps": args.train_steps,
                       "spread_on": 0.02, "spread_off": 0.01, "s_floor_gpa": s_floor,
                       "fe_predictor": "affine, g = (X_x, 0, 0)", "fe_damping": "c dt / 2 = 1"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="necking_bar",
                    choices=["necking_bar", "copper_bar", "kg_bar", "surrogate_fe", "surrogate_fe_cu", "kg_statics",
                             "surrogate_train", "kg_tensile"])
    ap.add_argument("--md-steps", type=int, default=MD_STEPS)
    ap.add_argument("--skin", type=float, default=1.5, help="copper bar: Verlet skin (A)")
    ap.add_argument("--skin-kg", type=float, default=0.0, help="necking bar: fixed skin (0 = autotuned)")
    ap.add_argument("--element", default="hex8", choices=["hex8", "tet4"],
                    help="FE element of the copper bar: 8-node hexahedra (32 r-cells) or 4-node tetrahedra (192)")
    ap.add_argument("--tpa", type=int, default=-1, help="lanes per atom (0: the lean walk; -1: default / autotuned)")
    ap.add_argument("--profile-steps", type=int, default=100)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--distinct", type=int, default=16, help="necking bar: distinct seeded melts")
    ap.add_argument("--mesh", default="", help="necking bar: another mesh nx,ny,nz (a smaller bar for profiling)")
    ap.add_argument("--procs", type=int, default=16, help="host processes for the melts")
    ap.add_argument("--soft-steps", type=int, default=1000)
    ap.add_argument("--eq-steps", type=int, default=1000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--kg-cells", type=int, default=64)
    ap.add_argument("--pushoff", type=int, default=300)
    ap.add_argument("--paths", type=int, default=1024)
    ap.add_argument("--train-steps", type=int, default=2500)
    ap.add_argument("--sur-md", type=int, default=400, help="copper surrogate: MD steps per increment")
    ap.add_argument("--s-floor", type=float, default=0.0,
                    help="copper surrogate: spread floor (GPa; 0 = half the RMS stress of the training data)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        out = run_reference(args)
        if out is not None:
            print(json.dumps(out))
        return
    if args.workload == "necking_bar":
        out = run_necking_bar(args)
        if out is not None:
            if not args.no_cpu_baseline and out["n_gpus"] == 1:
                out["cpu_baseline"] = neck_cpu_baseline(args.cpu_seconds)
            print(json.dumps(out))
        return
    if args.workload != "copper_bar":
        run = {"kg_bar": run_kg_bar, "surrogate_fe": run_surrogate_fe, "surrogate_fe_cu": run_surrogate_fe_cu,
               "kg_statics": run_kg_statics,
               "surrogate_train": run_surrogate_train, "kg_tensile": run_kg_tensile}[args.workload]
        out = run(args)
        print(json.dumps(out))
        return
    out = run_ours(args)
    if out is not None:
        if not args.no_cpu_baseline and out["n_gpus"] == 1:
            out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(out))


if __name__ == "__main__":
    main()
