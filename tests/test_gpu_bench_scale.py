"""Parity at the sizes and launch configuration the benchmark runs.

* Copper bar: 32 r-cells of 4000 Sutton-Chen atoms in one batch (1024 tiles of
  128 atoms; the pair kernels' grid is padded to a multiple of the SM count and
  its blocks remapped to tiles), skin 1.5 A, the default lanes per atom, CUDA
  graphs and programmatic dependent launch on: forces, energy and virial of
  four cells; a 20-step Langevin trajectory whose first ten steps take the
  force variant without virial (no stress sample) and whose last ten sample
  the stress; one load increment's time-averaged stress of four cells.
* Kremer-Grest: the chunked periodic-box tensile deformation of Sec. 3.2's
  comparison run at T = 0.1, bonds and all.
* Surrogate: the ensemble forward and one member-batched AdamW step at the
  training shape (4 members, batch 4096, 60 increments).

Inputs are seeded and generated on the host for both sides; tolerances as in
test_gpu_parity.py (forces 1e-5 of max(|f_i|, f_rms), virial 1e-4 of its
scale, trajectories to FP32 accuracy, averaged stress within max(2 %, 3 sigma))
and test_gpu_surrogate.py (BF16 operands).
"""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle
from _helpers import KB, M_CU, force_err, min_image_diff, oracle_md, oracle_pot
from oracle import mlp
from paper_1902_09171_gb300 import inputs, pipeline, rcell
from paper_1902_09171_gb300 import surrogate as S
from test_gpu_surrogate import bf16, bf16_weights

pytestmark = pytest.mark.gpu

N_BAR = 32


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


def copper_bar_cells(jit):
    """The benchmark's r-cells: 10x10x10 FCC copper (a = 3.615 A), Maxwell 300 K per
    cell (seed 1000 + c), positions jittered by up to `jit` A (seed 500 + c) and
    wrapped into the box on the host, so that the engine's own wrap moves no atom
    (an FP32 wrap would shift a coordinate by up to half an ulp of the box length)."""
    x, H = inputs.fcc(10, 10, 10, 3.615)
    kT = 300 * KB
    L = H[0, 0]
    return [dict(H0=H, x0=inputs.to_f32(np.mod(inputs.jitter(x, jit, 500 + c), L)),
                 v0=inputs.to_f32(inputs.maxwell(len(x), M_CU, kT, 0, 1000 + c))) for c in range(N_BAR)]


def f32_box(H):
    """The MD box as the engine holds it: the FP64 box rounded once to FP32."""
    return np.asarray(H, dtype=np.float64).astype(np.float32).astype(np.float64)


def test_copper_bar_forces_at_bench_layout(torch):
    prm = rcell.params_sc_cu(skin=1.5)
    cells = copper_bar_cells(0.1)
    ctx = rcell.rcell_create(prm, cells)
    try:
        rcell.rcell_eval(ctx)
        pe, W = rcell.rcell_get_energy(ctx)
        for c in (0, 11, 22, 31):
            _, _, f = rcell.rcell_get_atoms(ctx, c, 4000)
            fo, Wo, eo = oracle.forces(oracle_pot(prm), cells[c]["x0"], f32_box(cells[c]["H0"]))
            assert force_err(f, fo) <= 1e-5, (c, force_err(f, fo))
            assert abs(pe[c] - eo) <= 1e-5 * abs(eo), (c, pe[c], eo)
            assert np.abs(W[c] - Wo).max() <= 1e-4 * np.abs(Wo).max(), c
    finally:
        rcell.rcell_destroy(ctx)


def test_copper_bar_trajectory_at_bench_layout(torch):
    prm = rcell.params_sc_cu(skin=1.5)
    cells = copper_bar_cells(0.05)
    n_steps, n_avg = 20, 10
    ctx = rcell.rcell_create(prm, cells)
    try:
        rcell.rcell_run(ctx, n_steps, n_avg)  # graph capture on first use
        assert rcell.rcell_sync(ctx) == 0
        got = {}
        for c in (3, 17):
            H = f32_box(cells[c]["H0"])
            x, v, _ = rcell.rcell_get_atoms(ctx, c, 4000)
            s, pe, ke = rcell.rcell_get_series(ctx, c, n_avg)
            got[c] = (H, x, v, s, pe, ke)
    finally:
        rcell.rcell_destroy(ctx)

    def ref(c):
        return oracle.md_run(oracle_pot(prm), oracle_md(prm), cells[c]["x0"], cells[c]["v0"], got[c][0], cell=c,
                             ev=0, n_steps=n_steps, n_avg=n_avg)

    with cf.ThreadPoolExecutor(2) as ex:
        refs = dict(zip(got, ex.map(ref, list(got))))
    for c, (H, x, v, s, pe, ke) in got.items():
        xo, vo, ev, so, peo, keo = refs[c]
        assert ev == n_steps + 1
        assert np.abs(min_image_diff(x, xo, H)).max() < 1e-4, c
        assert np.abs(v - vo).max() < 1e-3 * np.abs(vo).max(), c
        assert np.abs(s - so).max() <= 1e-4 * np.abs(so).max(), c
        assert np.abs(pe - peo).max() <= 1e-5 * np.abs(peo).max(), c
        assert np.abs(ke - keo).max() <= 1e-4 * np.abs(keo).max(), c


def test_copper_bar_increment_stress_at_bench_layout(torch):
    # the bar's first load increment (0.2 % uniaxial stretch) on every cell, stress
    # averaged over the second half of the MD run; four cells against the oracle
    prm = rcell.params_sc_cu(skin=1.5)
    cells = copper_bar_cells(0.0)
    n_steps, n_avg = 400, 200
    F = np.diag([1.002, 1.0, 1.0])
    ctx = rcell.rcell_create(prm, cells)
    try:
        rcell.rcell_set_deformation(ctx, np.tile(F, (N_BAR, 1, 1)))
        rcell.rcell_run(ctx, n_steps, n_avg)
        sig, se, P = rcell.rcell_stress(ctx)
    finally:
        rcell.rcell_destroy(ctx)
    Q, R = oracle.qr(F)
    H = {c: f32_box(R @ cells[c]["H0"]) for c in range(N_BAR)}

    def ref(c):
        x = oracle.remap(cells[c]["x0"], oracle.delta_R(R, np.eye(3)))
        _, _, _, so, _, _ = oracle.md_run(oracle_pot(prm), oracle_md(prm), x, cells[c]["v0"], H[c], cell=c, ev=0,
                                          n_steps=n_steps, n_avg=n_avg)
        so_fem = np.array([oracle.rotate_pk1(Q, F, s)[0] for s in so])
        return np.array([oracle.block_stats(so_fem[:, j]) for j in range(6)])

    subset = (0, 9, 18, 31)
    with cf.ThreadPoolExecutor(len(subset)) as ex:
        refs = dict(zip(subset, ex.map(ref, subset)))
    for c in subset:
        r = refs[c]
        tol = np.maximum(0.02 * np.abs(r[:, 0]), 3 * np.sqrt(se[c] ** 2 + r[:, 1] ** 2))
        assert np.all(np.abs(sig[c] - r[:, 0]) <= tol), (c, sig[c], r[:, 0], tol)


def test_kremer_grest_chunked_tensile_trajectory_matches_oracle(torch):
    # Sec. 3.2's periodic-box comparison run on a bead-spring melt at T = 0.1:
    # three chunks of 5 steps, each after a 1 % uniaxial stretch with lateral
    # contraction, FENE + WCA bonds and the non-bonded LJ, same Philox stream
    prm = rcell.params_kg(kT=0.1, seed=8)
    x0, H0, bonds = inputs.kg_melt(20, 50, 0.85, seed=12, pushoff_iters=300)
    # a pushed-off melt still holds near-overlaps whose forces would stretch bonds
    # past R0 within a few steps: relax it first (host side, the oracle's FIRE)
    x0, _ = oracle.fire_minimize(oracle_pot(prm), x0, H0, 1.0, 1.0, 0.001, 0.01, 2000, bonds=bonds, units=1,
                                 dmax=0.05)
    x0 = inputs.to_f32(np.mod(x0, H0[0, 0]))
    v0 = inputs.to_f32(inputs.maxwell(len(x0), 1.0, 0.1, 1, 12))
    cell = dict(H0=H0, x0=x0, v0=v0, bonds=bonds)
    n = len(x0)
    chunk, n_chunks = 5, 3
    rate = 0.01 / (chunk * prm.dt)
    ctx = rcell.rcell_create(prm, [cell])
    try:
        eps, sig = pipeline.pbc_tensile(ctx, rate, prm.dt, n_chunks, chunk, nu=0.5)
        x_g, v_g, _ = rcell.rcell_get_atoms(ctx, 0, n)
        H_g, _, _ = rcell.rcell_get_box(ctx, 0)
    finally:
        rcell.rcell_destroy(ctx)
    assert np.allclose(eps, [0.01, 0.02, 0.03])
    pot, md = oracle_pot(prm), oracle_md(prm)
    x, v, ev = x0.astype(np.float64), v0.astype(np.float64), 0
    R_prev = np.eye(3)
    for k in range(n_chunks):
        F = pipeline.tensile_F(eps[k], 0.5)
        Q, R = oracle.qr(F)
        x = oracle.remap(x, oracle.delta_R(R, R_prev))
        R_prev = R
        H = (R @ H0).astype(np.float32).astype(np.float64)
        x, v, ev, s, _, _ = oracle.md_run(pot, md, x, v, H, bonds=bonds, cell=0, ev=ev, n_steps=chunk, n_avg=chunk)
        s_mean = s.mean(0)
        assert np.abs(sig[k][0] - s_mean).max() <= 2e-3 * np.abs(s_mean).max(), (k, sig[k][0], s_mean)
    assert np.allclose(H_g, H, rtol=1e-7, atol=0)
    assert np.abs(min_image_diff(x_g, x, H)).max() < 2e-4
    assert np.abs(v_g - v).max() < 2e-3 * np.abs(v).max()


def training_problem(B, T, K):
    rng = np.random.default_rng(2024)
    U = rng.standard_normal((B, T, mlp.N_IN))
    Y = 0.5 * np.cumsum(U[:, :, :mlp.N_OUT], axis=1) / np.sqrt(np.arange(1, T + 1))[None, :, None]
    thetas = [mlp.init_params(900 + k).astype(np.float32) for k in range(K)]
    return U, Y, thetas


def test_surrogate_forward_at_training_shape(torch):
    # 4 members x 4096 sequences x 60 increments in one launch (128 row tiles);
    # 48 rows of every member compared with the oracle's recurrence
    B, T, K = 4096, 60, 4
    U, _, thetas = training_problem(B, T, K)
    s = S.sur_create(K, B, T, 0)
    try:
        for k in range(K):
            S.sur_set_params(s, k, thetas[k])
        dU = torch.tensor(U, dtype=torch.float32, device="cuda")
        out = torch.zeros((K, B, T, 6), dtype=torch.float32, device="cuda")
        S.sur_predict(s, dU, out)
        assert S.sur_sync(s) == 0
        got = out.cpu().numpy()
    finally:
        S.sur_destroy(s)
    rows = np.sort(np.random.default_rng(7).choice(B, 48, replace=False))
    rows[0], rows[-1] = 0, B - 1  # first and last tile
    for k in range(K):
        ref, _ = mlp.forward(bf16_weights(thetas[k].astype(np.float64)), bf16(U[rows]))
        scale = np.abs(ref).max()
        err = np.abs(got[k, rows] - ref)
        assert err[:, :40].max() <= 3e-2 * scale, (k, err[:, :40].max() / scale)
        assert err.max() <= 1e-1 * scale, (k, err.max() / scale)
        assert err.mean() <= 5e-3 * scale, (k, err.mean() / scale)


def test_surrogate_training_step_at_training_shape(torch):
    # one AdamW step of every member side by side on the full batch: each member's
    # loss against the oracle, and its first move against the oracle gradient's
    # signs (for lr >> eps the first AdamW step is -lr sign(g), weight decay off)
    B, T, K, lr = 4096, 60, 4, 1e-3
    U, Y, thetas = training_problem(B, T, K)
    s = S.sur_create(K, B, T, 0)
    try:
        for k in range(K):
            S.sur_set_params(s, k, thetas[k])
        dU = torch.tensor(U, dtype=torch.float32, device="cuda")
        dY = torch.tensor(Y, dtype=torch.float32, device="cuda")
        loss = S.sur_train_step(s, dU, dY, lr, wd=0.0, n_members=K)
        assert S.sur_sync(s) == 0
        after = [S.sur_get_params(s, k) for k in range(K)]
    finally:
        S.sur_destroy(s)

    def ref(k):
        # the loss is a mean over rows: the full-batch loss and gradient are the
        # row-count-weighted sums over chunks of 512 rows (bounded host memory)
        th = bf16_weights(thetas[k].astype(np.float64))
        L, g = 0.0, np.zeros(th.size)
        for r0 in range(0, B, 512):
            Lc, gc = mlp.loss_and_grad(th, bf16(U[r0:r0 + 512]), Y[r0:r0 + 512])
            w = min(512, B - r0) / B
            L += w * Lc
            g += w * gc
        return L, g

    with cf.ThreadPoolExecutor(K) as ex:
        refs = list(ex.map(ref, range(K)))
    for k in range(K):
        Lr, gr = refs[k]
        assert abs(loss[k] - Lr) <= 2e-2 * Lr, (k, loss[k], Lr)
        step = after[k].astype(np.float64) - thetas[k].astype(np.float64)
        big = np.abs(gr) > 1e-2 * np.abs(gr).max()
        agree = np.mean(np.sign(step[big]) == -np.sign(gr[big]))
        assert agree > 0.99, (k, agree)
        assert np.abs(step[big]).max() <= 1.01 * lr
