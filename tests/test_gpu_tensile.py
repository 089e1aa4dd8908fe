"""Direct periodic-box MD tensile test (the comparison run of Sec. 3.2): a box
deformed in chunks of MD steps follows the same trajectory as the FP64 oracle
doing the same remaps and the same Langevin steps (same Philox counters)."""
import numpy as np
import pytest

import oracle
from _helpers import lj_cell, min_image_diff, oracle_md, oracle_pot
from paper_1902_09171_gb300 import inputs, pipeline, rcell

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


def test_chunked_tensile_deformation_matches_oracle():
    prm = rcell.params_lj_cu()
    cell = lj_cell(5, jit=0.05, seed=90)
    n = len(cell["x0"])
    chunk, n_chunks, rate = 5, 3, 1.0  # 1 / ps: 1 % strain per chunk of 5 steps of 2 fs
    ctx = rcell.rcell_create(prm, [cell])
    try:
        eps, sig = pipeline.pbc_tensile(ctx, rate, prm.dt, n_chunks, chunk, nu=0.5)
        x_g, v_g, _ = rcell.rcell_get_atoms(ctx, 0, n)
        H_g, _, _ = rcell.rcell_get_box(ctx, 0)
    finally:
        rcell.rcell_destroy(ctx)
    assert np.allclose(eps, [0.01, 0.02, 0.03])
    # the oracle: remap x <- Delta R x into the box R H0 (FP32-rounded, as the MD box is
    # held), then the same MD steps, chunk by chunk
    pot, md = oracle_pot(prm), oracle_md(prm)
    x, v, ev = inputs.to_f32(cell["x0"]).astype(np.float64), cell["v0"].astype(np.float64), 0
    R_prev = np.eye(3)
    for k in range(n_chunks):
        F = pipeline.tensile_F(eps[k], 0.5)
        Q, R = oracle.qr(F)
        x = oracle.remap(x, oracle.delta_R(R, R_prev))
        R_prev = R
        H = (R @ cell["H0"]).astype(np.float32).astype(np.float64)
        x, v, ev, s, _, _ = oracle.md_run(pot, md, x, v, H, cell=0, ev=ev, n_steps=chunk, n_avg=chunk)
        s_mean = s.mean(0)
        assert np.abs(sig[k][0] - s_mean).max() <= 2e-3 * np.abs(s_mean).max(), (k, sig[k][0], s_mean)
    assert np.allclose(H_g, H, rtol=1e-7, atol=0)
    assert np.abs(min_image_diff(x_g, x, H)).max() < 2e-4
    assert np.abs(v_g - v).max() < 2e-3 * np.abs(v).max()
