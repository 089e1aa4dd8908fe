"""Failure paths of the r-cell engine that host-made inputs reach, on the GPU.

Every failure here is made on the host -- a list capacity set too small, a wait
limit of zero polls, an input with a non-finite or absurd value -- and turned
into a status code by the library's own checks: bounded writes, bounded waits
that let their copies land before the block exits, per-cell status words.
Nothing faults, traps or hangs the GPU.  After each failure the context (or a
new one) keeps working.
"""
import numpy as np
import pytest

import oracle
from _helpers import force_err, lj_cell, oracle_pot
from paper_1902_09171_gb300 import rcell

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1902_09171_gb300 import build
    build.build()
    rcell.load()


def test_list_capacity_overflow_is_reported_and_recoverable():
    prm = rcell.params_lj_cu()
    cell = lj_cell(5, jit=0.1, seed=5)
    ctx = rcell.rcell_create(prm, [cell])
    try:
        with pytest.raises(rcell.RCellError) as e:
            rcell.rcell_set_limits(ctx, 6)  # not a multiple of 4
        assert e.value.name == "RC_EINVAL"
        rcell.rcell_set_limits(ctx, 8)  # about 90 neighbours per atom within r_list
        rcell.rcell_eval(ctx)
        assert rcell.STATUS[rcell.rcell_sync(ctx)] == "RC_EOVERFLOW"
        rcell.rcell_clear_status(ctx)
        rcell.rcell_set_limits(ctx, 0)  # the capacity allocated at creation
        rcell.rcell_eval(ctx)
        assert rcell.rcell_sync(ctx) == 0
        x, _, f = rcell.rcell_get_atoms(ctx, 0, len(cell["x0"]))
        H, _, _ = rcell.rcell_get_box(ctx, 0)
        fo, _, _ = oracle.forces(oracle_pot(prm), x, H)
        assert force_err(f, fo) <= 1e-5
    finally:
        rcell.rcell_destroy(ctx)


def test_non_finite_inputs_are_refused_before_any_launch():
    prm = rcell.params_lj_cu()
    for key in ("x0", "v0"):
        cell = lj_cell(4, seed=2)
        cell[key] = cell[key].copy()
        cell[key][17, 1] = np.nan if key == "x0" else np.inf
        with pytest.raises(rcell.RCellError) as e:
            rcell.rcell_create(prm, [cell])
        assert e.value.name == "RC_EINVAL"
    cell = lj_cell(4, seed=2)
    ctx = rcell.rcell_create(prm, [cell])
    try:
        F = np.diag([1.01, 1.0, 1.0])[None].copy()
        F[0, 2, 1] = np.nan
        with pytest.raises(rcell.RCellError) as e:
            rcell.rcell_set_deformation(ctx, F)
        assert e.value.name == "RC_EINVAL"
        # nothing was launched: the box is unchanged and the context runs on
        H, _, _ = rcell.rcell_get_box(ctx, 0)
        assert np.array_equal(H, cell["H0"].astype(np.float32).astype(np.float64))  # the FP32-held box
        rcell.rcell_run(ctx, 10, 5)
        sig, _, _ = rcell.rcell_stress(ctx)
        assert np.all(np.isfinite(sig))
    finally:
        rcell.rcell_destroy(ctx)


@pytest.mark.parametrize("speed,code", [(1.0e4, "RC_ELOST"), (1.0e30, "RC_ENAN")])
def test_runaway_atom_stops_only_its_own_cell(speed, code):
    # one atom of cell 1 moves farther than half the skin in one step (ELOST), or
    # so fast that its squared step overflows FP32 (ENAN); cell 0 of the same
    # batch runs on, bit for bit as it does alone
    prm = rcell.params_lj_cu()
    good = lj_cell(4, seed=3)
    bad = lj_cell(4, seed=4)
    bad["v0"] = bad["v0"].copy()
    bad["v0"][7] = [speed, 0.0, 0.0]
    n = len(good["x0"])
    both = rcell.rcell_create(prm, [good, bad])
    alone = rcell.rcell_create(prm, [good])
    try:
        rcell.rcell_run(both, 8, 4)
        rcell.rcell_run(alone, 8, 4)
        assert rcell.STATUS[rcell.rcell_sync(both)] == code
        assert rcell.rcell_sync(alone) == 0
        x2, v2, _ = rcell.rcell_get_atoms(both, 0, n)
        x1, v1, _ = rcell.rcell_get_atoms(alone, 0, n)
        assert np.array_equal(x1, x2) and np.array_equal(v1, v2)
    finally:
        rcell.rcell_destroy(both)
        rcell.rcell_destroy(alone)


def test_staging_wait_that_gives_up_reports_timeout_and_recovers():
    # the shared-memory staging wait with a limit of zero polls gives up at once;
    # the block still waits (bounded) for its issued copy before it exits
    prm = rcell.params_lj_cu()
    cells = [lj_cell(4, seed=6), lj_cell(5, seed=7)]
    ctx = rcell.rcell_create(prm, cells)
    try:
        rcell.rcell_set_staging(ctx, 1)
        rcell.rcell_set_limits(ctx, -1, 0)
        rcell.rcell_run(ctx, 6, 3)
        assert rcell.STATUS[rcell.rcell_sync(ctx)] == "RC_ETIMEOUT"
        rcell.rcell_clear_status(ctx)
        rcell.rcell_set_limits(ctx, -1, rcell.RC_WAIT_POLLS_DEFAULT)
        rcell.rcell_run(ctx, 6, 3)
        sig, _, _ = rcell.rcell_stress(ctx)
        assert np.all(np.isfinite(sig))
    finally:
        rcell.rcell_destroy(ctx)
