"""What the trained surrogate gains over the method without it, on the GPU.

A small copper bar (4 x 1 x 1 hexahedra, one Sutton-Chen r-cell of 2048 atoms
per element, 300 K; affine load predictor, gradient-flow damping) is loaded in
16 increments to 4 % twice from the same cells and the same Langevin seed: once
with every point on r-cell MD (fe_step), once with the learned surrogate and
the MD fallback (fe_step_surrogate, MD forced on the first two increments, trip
above 2 % ensemble spread, release below 1 %, spread floor half the RMS stress
of the training data, missed increments replayed on return).  The surrogate
was trained on the GPU by the library's own kernels, on r-cell trajectories the
library generated along seeded bar-like deformation histories.

Gain: fewer MD cell-increments (the replayed ones included) than all-MD, at a
system-averaged axial stress curve within 2 % of the all-MD one (max |dP_xx| /
max |P_xx|), the criterion of the surrogate target.
"""
import numpy as np
import pytest

from paper_1902_09171_gb300 import inputs, pipeline, rcell
from paper_1902_09171_gb300 import surrogate as S

pytestmark = pytest.mark.gpu

KB = 8.617333262e-5
M_CU = 63.546


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


def cu_cells(n, seed0):
    x, H = inputs.fcc(8, 8, 8, 3.615)
    x = inputs.to_f32(x)
    return [dict(H0=H, x0=x, v0=inputs.to_f32(inputs.maxwell(len(x), M_CU, 300 * KB, 0, seed0 + c))) for c in range(n)]


def test_surrogate_takes_fewer_md_increments_at_two_percent(torch):
    st = torch.cuda.Stream()
    torch.cuda.set_stream(st)
    T, n_steps, n_avg, K, NP = 16, 300, 150, 4, 256
    kT = 300 * KB
    try:
        # training data: r-cells driven along bar-like histories, then a 4-member ensemble
        ctx = rcell.rcell_create(rcell.params_sc_cu(tau=0.1, kT=kT, seed=31), cu_cells(NP, 700), stream=st)
        F = inputs.bar_strain_paths(NP, T, seed=17, max_axial=0.06, max_shear=0.02, max_lateral=0.03)
        U, Y, _ = pipeline.generate_dataset(ctx, F, n_steps, n_avg, stream=st)
        rcell.rcell_destroy(ctx)
        sur = S.sur_create(K, NP, T, seed=9, stream=st)
        us, ys = pipeline.feature_scales(U, Y)
        S.sur_set_scaling(sur, us, ys)
        pipeline.train(sur, U, Y, 3000, lr=1e-3, n_members=K)
        s_floor = 0.5 * float(ys[0])  # half the RMS stress of the training data
        assert S.sur_sync(sur) == 0
        # the bar, twice from the same cells and seed
        cells = cu_cells(4, 100)
        L = cells[0]["H0"][0, 0]
        X, conn = inputs.hex_mesh(4, 1, 1, 4 * L, L, L)
        mask, val = inputs.uniaxial_bc(X, 4 * L)
        rho0 = 4 * M_CU / 3.615 ** 3 / 60.2214
        c = np.sqrt(130.0 / rho0)
        dt_fe = 0.5 * L / c
        g = np.zeros_like(X)
        g[:, 0] = X[:, 0]  # affine predictor of the uniaxial increments
        bars = []
        for _ in range(2):
            fe = rcell.fe_create(X, conn, mask, val, rho0, dt_fe, 2.0 / dt_fe, 6.5, stream=st)  # gradient flow
            rcell.fe_set_predictor(fe, g)
            bars.append((rcell.rcell_create(rcell.params_sc_cu(tau=0.1, kT=kT, seed=41), cells, stream=st), fe))
        try:
            lams = [0.04 * (k + 1) / T for k in range(T)]
            res = pipeline.fe_compare(bars[0][0], bars[1][0], sur, bars[0][1], bars[1][1], K, lams, n_steps, n_avg,
                                      spread_on=0.02, spread_off=0.01, s_floor=s_floor, stream=st)
            for ctx_, _ in bars:
                assert rcell.rcell_sync(ctx_) == 0
        finally:
            for ctx_, fe in bars:
                rcell.fe_destroy(fe)
                rcell.rcell_destroy(ctx_)
            S.sur_destroy(sur)
    finally:
        torch.cuda.set_stream(torch.cuda.default_stream())
    md_increments = sum(res["n_md"])
    all_md = 4 * T
    assert md_increments < all_md, res
    assert res["max_rel_dev"] <= 0.02, (res["max_rel_dev"], res["axial_md"], res["axial_sg"])
