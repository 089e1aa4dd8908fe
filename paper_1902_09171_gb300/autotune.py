"""Autotuner for the batched r-cell MD launches.

Tunables: the Verlet skin (list size versus rebuild frequency; fixed at
context creation) and the number of lanes that share one atom's list
(1, 2, 4 or 8 with the software-pipelined walk, or 0 for the lean walk;
switchable on a live context).  Each candidate is timed on the
caller's own batch -- the captured MD loop of `n_steps` steps after one warm-up
run, with CUDA events on the batch's stream -- and the fastest is cached per
(GPU name, potential, atom-count bucket) in a JSON file, so later runs on the
same kind of GPU and workload skip the search.
"""
from __future__ import annotations

import json
import os
import threading

from . import rcell

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "_autotune_cache.json")
_lock = threading.Lock()


def bucket(n_atoms: int) -> str:
    """Power-of-two bucket of the batch's atom count."""
    b = 1
    while b < n_atoms:
        b <<= 1
    return str(b)


def key(gpu: str, potential: int, n_atoms: int) -> str:
    return f"{gpu}|pot{potential}|n{bucket(n_atoms)}"


def load_cache(path: str = CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store(k: str, value: dict, path: str = CACHE) -> None:
    with _lock:
        c = load_cache(path)
        c[k] = value
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def search(make_params, cells, time_candidate, skins, tpas):
    """Generic search: time_candidate(params, tpa) -> ms per MD step (or None if the
    candidate is invalid); returns the best (skin, tpa, ms) and the full table."""
    table = []
    for skin in skins:
        prm = make_params(skin)
        for tpa in tpas:
            ms = time_candidate(prm, cells, tpa)
            if ms is not None:
                table.append({"skin": skin, "tpa": tpa, "ms_per_step": ms})
    if not table:
        raise RuntimeError("no valid autotune candidate")
    best = min(table, key=lambda r: r["ms_per_step"])
    return best, table


def cuda_timer(stream, n_steps=100, n_avg=0):
    """Candidate timer for a CUDA batch: builds the context, runs one warm-up
    (captures the graph), then times one run of n_steps steps that records a
    stress sample on the last n_avg of them (as a load increment does: sampling
    steps evaluate the virial too, which makes long lists costlier)."""
    import torch

    def run(prm, cells, tpa):
        try:
            ctx = rcell.rcell_create(prm, cells, stream=stream)
        except rcell.RCellError:
            return None  # e.g. skin too large for the box (r_list > w / 2)
        try:
            rcell.rcell_set_tuning(ctx, tpa, 1)
            rcell.rcell_run(ctx, n_steps, n_avg)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rcell.rcell_run(ctx, n_steps, n_avg)
            e1.record(stream)
            torch.cuda.synchronize()
            if rcell.rcell_sync(ctx) != 0:
                return None
            return e0.elapsed_time(e1) / n_steps
        finally:
            rcell.rcell_destroy(ctx)

    return run


def tune(make_params, cells, stream, skins=(1.0, 1.5, 2.0), tpas=(1, 2, 4), n_steps=100, use_cache=True,
         path: str = CACHE, n_avg=0):
    """Best (skin, tpa) for this GPU and workload, from the cache or by search
    (each candidate timed over n_steps MD steps, the last n_avg sampling)."""
    import torch
    gpu = torch.cuda.get_device_name()
    prm0 = make_params(skins[0])
    n_atoms = sum(len(c["x0"]) for c in cells)
    k = key(gpu, prm0.potential, n_atoms)
    if use_cache:
        hit = load_cache(path).get(k)
        if hit:
            return hit, True
    best, table = search(make_params, cells, cuda_timer(stream, n_steps, n_avg), skins, tpas)
    value = dict(best, table=table)
    store(k, value, path)
    return value, False
