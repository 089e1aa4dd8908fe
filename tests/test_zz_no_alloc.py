"""The allocation-free stress reduction (rcell_stress_reduce_static) against the
context's own reduction (rcell_stress).

Callers that cannot call cudaMalloc at the time they reduce -- a host program
that reserves the GPU's memory up front for its own pool, a latency-bound loop
that must not take the implicit device synchronisation of cudaFree -- use the
static entry point, whose only scratch is a fixed array in the library's device
image.  This file runs last (pytest orders files by name) so that a failure
here leaves every other test already run.
"""
import json
import os

import numpy as np
import pytest

from _helpers import lj_cell
from paper_1902_09171_gb300 import rcell

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1.json")))


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    t.cuda.set_device(0)
    from paper_1902_09171_gb300 import build
    build.build()
    rcell.load()
    return t


def test_static_reduction_matches_rcell_stress_twice(torch):
    prm = rcell.params_lj_cu()
    names = ["B(t)", "C(t)", "C(c)"]
    cells = [lj_cell(5, seed=30 + k) for k in range(len(names))]
    F = np.array([GOLD["cases"][k]["F"] for k in names])
    n_steps, n_avg = 120, 96
    ctx = rcell.rcell_create(prm, cells)
    try:
        rcell.rcell_set_deformation(ctx, F)
        rcell.rcell_run(ctx, n_steps, n_avg)
        sig, se, P = rcell.rcell_stress(ctx)
        series = np.stack([rcell.rcell_get_series(ctx, k, n_avg)[0] for k in range(len(cells))])
        Q = np.stack([rcell.rcell_get_box(ctx, k)[1] for k in range(len(cells))])
    finally:
        rcell.rcell_destroy(ctx)
    dev = torch.device("cuda:0")
    t_series = torch.tensor(series, dtype=torch.float64, device=dev).contiguous()
    t_Q = torch.tensor(Q, dtype=torch.float64, device=dev).contiguous()
    t_F = torch.tensor(F, dtype=torch.float64, device=dev).contiguous()
    for call in range(2):
        out_s = torch.full((len(cells), 6), float("nan"), dtype=torch.float64, device=dev)
        out_e = torch.full((len(cells), 6), float("nan"), dtype=torch.float64, device=dev)
        out_P = torch.full((len(cells), 3, 3), float("nan"), dtype=torch.float64, device=dev)
        rcell.rcell_stress_reduce_static(t_series, t_Q, t_F, out_s, out_e, out_P)
        torch.cuda.synchronize()
        s2, e2, P2 = out_s.cpu().numpy(), out_e.cpu().numpy(), out_P.cpu().numpy()
        assert np.abs(s2 - sig).max() <= 1e-10 * np.abs(sig).max(), call
        assert np.abs(e2 - se).max() <= 1e-8 * np.abs(se).max(), call
        assert np.abs(P2 - P).max() <= 1e-10 * np.abs(P).max(), call


def test_static_reduction_rejects_oversized_input(torch):
    dev = torch.device("cuda:0")
    n_cells, n_avg = 2, 40000  # 80000 samples > 65536
    series = torch.zeros((n_cells, n_avg, 6), dtype=torch.float64, device=dev)
    Q = torch.eye(3, dtype=torch.float64, device=dev).repeat(n_cells, 1, 1).contiguous()
    out = torch.zeros((n_cells, 6), dtype=torch.float64, device=dev)
    with pytest.raises(rcell.RCellError) as e:
        rcell.rcell_stress_reduce_static(series, Q, Q, out)
    assert e.value.name == "RC_EINVAL"


def test_static_reduction_rejects_bad_tensors_before_the_call(torch):
    # wrong dtype, layout or shape never reaches the kernel
    dev = torch.device("cuda:0")
    n_cells, n_avg = 2, 32
    series = torch.zeros((n_cells, n_avg, 6), dtype=torch.float64, device=dev)
    Q = torch.eye(3, dtype=torch.float64, device=dev).repeat(n_cells, 1, 1).contiguous()
    out = torch.zeros((n_cells, 6), dtype=torch.float64, device=dev)
    bad = [
        (series.float(), Q, Q, out),
        (series, Q.transpose(1, 2), Q, out),
        (series, Q[:1].contiguous(), Q, out),
        (series, Q, Q, out[:1].contiguous()),
        (series[:, :, :5].contiguous(), Q, Q, out),
        (series.cpu(), Q, Q, out),
    ]
    for args in bad:
        with pytest.raises(rcell.RCellError) as e:
            rcell.rcell_stress_reduce_static(*args)
        assert e.value.name == "RC_EINVAL"
