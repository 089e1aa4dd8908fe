"""GPU-vs-oracle parity of the r-cell hot path, called through the C ABI.

Tolerances (floating point; integers and index sets are compared exactly):
  * QR / box / Delta R (FP64 on both sides): 1e-13 absolute.
  * remapped positions: FP32 rounding of the stored coordinates, 4e-6 relative.
  * forces: |df_i| <= 1e-5 max(|f_i|, f_rms) per atom.
  * instantaneous virial / energy: 1e-4 of the virial scale.
  * neighbour lists: identical sets of (i, j) tag pairs within r_list, on
    configurations with no pair within 1e-5 r_list of the list radius.
"""
import json
import os

import numpy as np
import pytest

import oracle
from _helpers import KB, M_CU, force_err, lj_cell, min_image_diff, oracle_md, oracle_pot
from paper_1902_09171_gb300 import inputs, rcell

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1.json")))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1902_09171_gb300 import build
    build.build()
    rcell.load()


class Ctx:
    def __init__(self, prm, cells):
        self.prm = prm
        self.cells = cells
        self.h = rcell.rcell_create(prm, cells)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        rcell.rcell_destroy(self.h)


def test_geometry_matches_oracle_on_table1():
    prm = rcell.params_lj_cu()
    names = list(GOLD["cases"])
    cells = [lj_cell(5, seed=k) for k in range(len(names))]
    F = np.array([GOLD["cases"][k]["F"] for k in names])
    with Ctx(prm, cells) as c:
        rcell.rcell_set_deformation(c.h, F)
        assert rcell.rcell_sync(c.h) == 0
        for k, name in enumerate(names):
            H, Q, R = rcell.rcell_get_box(c.h, k)
            Qo, Ro = oracle.qr(F[k])
            assert np.abs(Q - Qo).max() < 1e-13 and np.abs(R - Ro).max() < 1e-13
            # the MD box is R H0 rounded once to FP32 (positions and box are FP32)
            assert np.abs(H - Ro @ cells[k]["H0"]).max() <= 6e-8 * np.abs(H).max()
            assert np.array_equal(H, inputs.to_f32(H))
            # Table 1 values themselves (3 printed decimals)
            assert np.abs(Q - np.array(GOLD["cases"][name]["Q"])).max() <= 5e-4
            x, _, _ = rcell.rcell_get_atoms(c.h, k, len(cells[k]["x0"]))
            xo = oracle.remap(cells[k]["x0"], oracle.delta_R(Ro, np.eye(3)))
            assert np.abs(x - xo).max() <= 4e-6 * np.abs(xo).max()


def test_incremental_remap_composes():
    # successive deformations: positions follow R(t) H0 S through Delta R (Eq. LAMMPS2)
    prm = rcell.params_lj_cu()
    cell = lj_cell(5, jit=0.0)
    with Ctx(prm, [cell]) as c:
        R_prev = np.eye(3)
        x = cell["x0"].copy()
        for k in range(4):
            F = np.eye(3) + 0.01 * (k + 1) * np.array([[1, 0.3, 0.1], [0.2, -0.5, 0.1], [0.0, 0.4, 0.2]])
            rcell.rcell_set_deformation(c.h, F[None])
            Q, R = oracle.qr(F)
            x = oracle.remap(inputs.to_f32(x), oracle.delta_R(R, R_prev))
            R_prev = R
            xg, _, _ = rcell.rcell_get_atoms(c.h, 0, len(x))
            assert np.abs(xg - x).max() <= 1e-5 * np.abs(x).max()


def test_degenerate_F_and_thin_box_are_reported_per_cell():
    prm = rcell.params_lj_cu()
    cells = [lj_cell(5, seed=k) for k in range(3)]
    F = np.stack([np.eye(3), np.diag([1.0, 1.0, -1.0]), np.diag([0.6, 1.0, 1.0])])
    with Ctx(prm, cells) as c:
        rcell.rcell_set_deformation(c.h, F)
        st = rcell.rcell_sync(c.h)
        assert rcell.STATUS[st] in ("RC_EDEGEN", "RC_EBOX")
        # cell 0 is untouched and still runs; the context is reusable after clearing
        rcell.rcell_clear_status(c.h)
        rcell.rcell_set_deformation(c.h, np.stack([np.eye(3)] * 3))
        rcell.rcell_run(c.h, 5, 2)
        sig, se, P = rcell.rcell_stress(c.h)
        assert np.all(np.isfinite(sig))
    # a bad F on its own: EDEGEN, and the cell keeps its previous box
    with Ctx(prm, cells[:1]) as c:
        rcell.rcell_set_deformation(c.h, np.diag([1.0, -1.0, 1.0])[None])
        assert rcell.STATUS[rcell.rcell_sync(c.h)] == "RC_EDEGEN"
        H, _, _ = rcell.rcell_get_box(c.h, 0)
        assert np.array_equal(H, inputs.to_f32(cells[0]["H0"]))
        rcell.rcell_clear_status(c.h)
        rcell.rcell_set_deformation(c.h, np.diag([0.6, 1.0, 1.0])[None])
        assert rcell.STATUS[rcell.rcell_sync(c.h)] == "RC_EBOX"


def _guarded(x, H, rlist):
    """True when no pair distance lies within 1e-5 r_list of r_list."""
    lo = oracle.neighbor_pairs(x, H, rlist * (1 - 1e-5))
    hi = oracle.neighbor_pairs(x, H, rlist * (1 + 1e-5))
    return len(lo) == len(hi)


@pytest.mark.parametrize("shear", [False, True])
def test_neighbor_sets_bit_exact(shear):
    prm = rcell.params_lj_cu()
    rlist = prm.rc + prm.skin
    for seed in range(1, 6):
        cell = lj_cell(5, jit=0.2, seed=seed)
        with Ctx(prm, [cell]) as c:
            if shear:
                rcell.rcell_set_deformation(c.h, np.array(GOLD["cases"]["C(t)"]["F"])[None])
            rcell.rcell_eval(c.h)
            x, _, _ = rcell.rcell_get_atoms(c.h, 0, len(cell["x0"]))
            H, _, _ = rcell.rcell_get_box(c.h, 0)
            if not _guarded(x, H, rlist):
                continue
            got = rcell.rcell_get_neighbors(c.h, 0, 500 * 200)
            ref = oracle.neighbor_pairs(x, H, rlist)
            assert len(got) == len(ref)
            assert {tuple(p) for p in got} == {tuple(p) for p in ref}
            return
    pytest.fail("no guarded configuration found")


def _eval_and_compare(prm, cells, bonds_of=None):
    with Ctx(prm, cells) as c:
        rcell.rcell_eval(c.h)
        pe, W = rcell.rcell_get_energy(c.h)
        for k, cell in enumerate(cells):
            n = len(cell["x0"])
            x, _, f = rcell.rcell_get_atoms(c.h, k, n)
            H, _, _ = rcell.rcell_get_box(c.h, k)
            fo, Wo, eo = oracle.forces(oracle_pot(prm), x, H, bonds=cell.get("bonds"))
            assert force_err(f, fo) <= 1e-5, (k, force_err(f, fo))
            assert abs(pe[k] - eo) <= 1e-5 * max(abs(eo), 1.0) * max(1.0, n / 1000)
            wscale = max(np.abs(Wo).max(), 1e-12)
            assert np.abs(W[k] - Wo).max() <= 1e-4 * wscale, (k, np.abs(W[k] - Wo).max() / wscale)


def test_forces_energy_virial_lj_tilted_box():
    prm = rcell.params_lj_cu()
    cells = [lj_cell(5, jit=0.15, seed=7)]
    with Ctx(prm, cells) as c:
        rcell.rcell_set_deformation(c.h, np.array(GOLD["cases"]["B(t)"]["F"])[None])
        rcell.rcell_eval(c.h)
        x, _, f = rcell.rcell_get_atoms(c.h, 0, 500)
        H, _, _ = rcell.rcell_get_box(c.h, 0)
        fo, Wo, eo = oracle.forces(oracle_pot(prm), x, H)
        assert force_err(f, fo) <= 1e-5
        pe, W = rcell.rcell_get_energy(c.h)
        assert np.abs(W[0] - Wo).max() <= 1e-4 * np.abs(Wo).max()
        assert abs(pe[0] - eo) <= 1e-5 * abs(eo)


def test_forces_sutton_chen_4000_atom_cell():
    prm = rcell.params_sc_cu()
    x, H = inputs.fcc(10, 10, 10, 3.615)
    cells = [dict(H0=H, x0=inputs.to_f32(inputs.jitter(x, 0.1, 11)))]
    _eval_and_compare(prm, cells)


def test_forces_kremer_grest_melt():
    prm = rcell.params_kg()
    x, H, bonds = inputs.kg_melt(20, 50, 0.85, seed=4, pushoff_iters=300)
    cells = [dict(H0=H, x0=inputs.to_f32(x), bonds=bonds)]
    _eval_and_compare(prm, cells)


def test_kremer_grest_uneven_batch():
    # uneven bead-spring cells (1000, 1500, 2500 beads) in one batch, each with its
    # own bonds, box and neighbour bins
    prm = rcell.params_kg()
    cells = []
    for k, nch in enumerate((20, 30, 50)):
        x, H, bonds = inputs.kg_melt(nch, 50, 0.85, seed=40 + k, pushoff_iters=300)
        cells.append(dict(H0=H, x0=inputs.to_f32(x), bonds=bonds))
    _eval_and_compare(prm, cells)


def test_ragged_batch_of_uneven_cells():
    # cells of 256, 480, 500 and 864 atoms in one batch: tiles of 128 with ragged tails
    prm = rcell.params_lj_cu()
    cells = []
    for k, dims in enumerate([(4, 4, 4), (4, 5, 6), (5, 5, 5), (6, 6, 6)]):
        x, H = inputs.fcc(*dims, 3.615)
        cells.append(dict(H0=H, x0=inputs.to_f32(inputs.jitter(x, 0.1, 20 + k))))
    _eval_and_compare(prm, cells)


def test_kg_broken_bond_is_reported():
    prm = rcell.params_kg()
    H = np.diag([8.0, 8.0, 8.0])
    x = np.array([[1.0, 1.0, 1.0], [2.7, 1.0, 1.0], [5.0, 5.0, 5.0]])
    with Ctx(prm, [dict(H0=H, x0=x, bonds=np.array([[0, 1]]))]) as c:
        rcell.rcell_eval(c.h)
        assert rcell.STATUS[rcell.rcell_sync(c.h)] == "RC_EBOND"


@pytest.mark.parametrize("tpa", [0, 1, 2, 4, 8])
def test_short_trajectory_matches_oracle(tpa):
    # same seed, same Philox counters: positions, velocities and per-step virial
    # stress of a 10-step Langevin run agree to FP32 accuracy
    prm = rcell.params_lj_cu()
    cell = lj_cell(5, jit=0.05, seed=3)
    n = len(cell["x0"])
    with Ctx(prm, [cell]) as c:
        rcell.rcell_set_tuning(c.h, tpa, 1)
        H, _, _ = rcell.rcell_get_box(c.h, 0)  # the FP32-exact MD box
        rcell.rcell_run(c.h, 10, 10)
        s_g, pe_g, ke_g = rcell.rcell_get_series(c.h, 0, 10)
        x, v, _ = rcell.rcell_get_atoms(c.h, 0, n)
    xo, vo, ev, so, peo, keo = oracle.md_run(oracle_pot(prm), oracle_md(prm), cell["x0"], cell["v0"], H,
                                             cell=0, ev=0, n_steps=10, n_avg=10)
    assert ev == 11
    assert np.abs(min_image_diff(x, xo, H)).max() < 1e-4
    assert np.abs(v - vo).max() < 1e-3 * np.abs(vo).max()
    assert np.abs(s_g - so).max() <= 1e-4 * np.abs(so).max()
    assert np.abs(pe_g - peo).max() <= 1e-5 * np.abs(peo).max()
    assert np.abs(ke_g - keo).max() <= 1e-4 * np.abs(keo).max()


@pytest.mark.parametrize("use_graphs", [0, 1])
def test_time_averaged_stress_plain_method(use_graphs):
    # the plain method at 256 atoms: uniaxial increments F = diag(1 + 0.002k, 1, 1),
    # MD after each, stress averaged over the second half; GPU vs oracle within
    # max(2 %, 3 sigma) per component (sigma from both blocking errors)
    prm = rcell.params_lj_cu()
    cell = lj_cell(4, jit=0.0, seed=1)
    n_steps, n_avg = 300, 150
    x, v = cell["x0"].copy(), cell["v0"].copy()
    R_prev = np.eye(3)
    ev = 0
    with Ctx(prm, [cell]) as c:
        rcell.rcell_set_tuning(c.h, -1, use_graphs)
        for k in range(1, 4):
            F = np.diag([1 + 0.002 * k, 1.0, 1.0])
            rcell.rcell_set_deformation(c.h, F[None])
            rcell.rcell_run(c.h, n_steps, n_avg)
            sig, se, P = rcell.rcell_stress(c.h)
            Q, R = oracle.qr(F)
            x = oracle.remap(x, oracle.delta_R(R, R_prev))
            R_prev = R
            x, v, ev, so, _, _ = oracle.md_run(oracle_pot(prm), oracle_md(prm), x, v, R @ cell["H0"], cell=0, ev=ev,
                                               n_steps=n_steps, n_avg=n_avg)
            so_fem = np.array([oracle.rotate_pk1(Q, F, s)[0] for s in so])
            ref = np.array([oracle.block_stats(so_fem[:, j]) for j in range(6)])
            tol = np.maximum(0.02 * np.abs(ref[:, 0]), 3 * np.sqrt(se[0] ** 2 + ref[:, 1] ** 2))
            assert np.all(np.abs(sig[0] - ref[:, 0]) <= tol), (k, sig[0], ref[:, 0], tol)
            # P = J sigma F^-T of the GPU's own sigma
            _, Po = oracle.rotate_pk1(Q, F, _md_frame(Q, sig[0]))
            assert np.abs(P[0] - Po).max() <= 1e-10 * np.abs(Po).max()


def _md_frame(Q, s_fem):
    s, _ = oracle.rotate_pk1(Q.T, np.eye(3), s_fem)
    return s


def test_series_blocking_error_matches_oracle_statistics():
    prm = rcell.params_lj_cu()
    cell = lj_cell(4, seed=2)
    with Ctx(prm, [cell]) as c:
        rcell.rcell_run(c.h, 400, 256)
        sig, se, _ = rcell.rcell_stress(c.h)
        s_g, _, _ = rcell.rcell_get_series(c.h, 0, 256)
    ref = np.array([oracle.block_stats(s_g[:, j]) for j in range(6)])
    assert np.abs(sig[0] - ref[:, 0]).max() <= 1e-10 * np.abs(ref[:, 0]).max()
    assert np.abs(se[0] - ref[:, 1]).max() <= 1e-8 * np.abs(ref[:, 1]).max()


def test_fe_matches_oracle():
    X, conn = inputs.hex_mesh(3, 2, 2, 3.0, 2.0, 2.0)
    rng = np.random.default_rng(0)
    inner = np.all((X > 1e-9) & (X < np.array([3.0, 2.0, 2.0]) - 1e-9), axis=1)
    X[inner] += rng.uniform(-0.1, 0.1, (inner.sum(), 3))
    mask, val = inputs.uniaxial_bc(X, 3.0)
    args = (X, conn, mask, val, 1.3, 0.05, 0.7, 0.4)
    fe = rcell.fe_create(*args)
    ref = oracle.FEMesh(*args)
    try:
        for step, lam in enumerate([0.01, 0.02, 0.03]):
            rcell.fe_apply_bc(fe, lam)
            ref.apply_bc(lam)
            Fg = np.zeros((conn.shape[0], 3, 3))
            rcell.fe_get_F(fe, Fg)
            assert np.abs(Fg - ref.F()).max() < 1e-13
            P = rng.standard_normal((conn.shape[0], 3, 3))
            rcell.fe_update(fe, P)
            ref.update(P)
            d, v = rcell.fe_get_state(fe, X.shape[0])
            assert np.abs(d - ref.d).max() < 1e-12 * max(1.0, np.abs(ref.d).max())
            assert np.abs(v - ref.v).max() < 1e-12 * max(1.0, np.abs(ref.v).max())
    finally:
        rcell.fe_destroy(fe)


def test_fe_step_single_element_prescribes_uniaxial_F():
    prm = rcell.params_lj_cu()
    cell = lj_cell(4)
    L = cell["H0"][0, 0]
    X, conn = inputs.hex_mesh(1, 1, 1, L, L, L)
    mask, val = inputs.uniaxial_bc(X, L, all_nodes=True)
    fe = rcell.fe_create(X, conn, mask, val, 1.0, 0.01, 0.0, 0.0)
    with Ctx(prm, [cell]) as c:
        try:
            u = np.zeros((8, 3))
            for k in (1, 2):
                rcell.fe_step(fe, c.h, 0.002 * k, 50, 20, u)
                H, Q, R = rcell.rcell_get_box(c.h, 0)
                assert np.abs(R - np.diag([1 + 0.002 * k, 1, 1])).max() < 1e-15
                assert np.abs(Q - np.eye(3)).max() < 1e-15
        finally:
            rcell.fe_destroy(fe)


def test_checkpoint_restore_replays_identically():
    prm = rcell.params_lj_cu()
    cell = lj_cell(5, seed=9)
    n = len(cell["x0"])
    with Ctx(prm, [cell]) as c:
        rcell.rcell_run(c.h, 30, 10)
        blob = rcell.rcell_checkpoint(c.h, 0)
        rcell.rcell_run(c.h, 40, 10)
        x1, v1, _ = rcell.rcell_get_atoms(c.h, 0, n)
        rcell.rcell_restore(c.h, 0, blob)
        rcell.rcell_run(c.h, 40, 10)
        x2, v2, _ = rcell.rcell_get_atoms(c.h, 0, n)
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2)


def test_fe_with_affine_predictor_matches_oracle():
    X, conn = inputs.hex_mesh(3, 2, 2, 3.0, 2.0, 2.0)
    rng = np.random.default_rng(5)
    inner = np.all((X > 1e-9) & (X < np.array([3.0, 2.0, 2.0]) - 1e-9), axis=1)
    X[inner] += rng.uniform(-0.1, 0.1, (inner.sum(), 3))
    mask, val = inputs.uniaxial_bc(X, 3.0)
    g = np.zeros_like(X)
    g[:, 0] = X[:, 0]
    args = (X, conn, mask, val, 1.3, 0.05, 0.7, 0.4)
    fe = rcell.fe_create(*args)
    ref = oracle.FEMesh(*args)
    rcell.fe_set_predictor(fe, g)
    ref.set_predictor(g)
    try:
        for lam in (0.01, 0.02, 0.035):
            rcell.fe_apply_bc(fe, lam)
            ref.apply_bc(lam)
            Fg = np.zeros((conn.shape[0], 3, 3))
            rcell.fe_get_F(fe, Fg)
            assert np.abs(Fg - ref.F()).max() < 1e-13
            P = rng.standard_normal((conn.shape[0], 3, 3))
            rcell.fe_update(fe, P)
            ref.update(P)
            d, v = rcell.fe_get_state(fe, X.shape[0])
            assert np.abs(d - ref.d).max() < 1e-12 * max(1.0, np.abs(ref.d).max())
            assert np.abs(v - ref.v).max() < 1e-12 * max(1.0, np.abs(ref.v).max())
    finally:
        rcell.fe_destroy(fe)


@pytest.mark.parametrize("pot", ["lj", "sc", "kg"])
def test_lean_walk_forces_match_oracle(pot):
    # one lane per atom with the plain (not software-pipelined) list walk
    if pot == "lj":
        prm, cells = rcell.params_lj_cu(), [lj_cell(5, jit=0.15, seed=71)]
    elif pot == "sc":
        prm = rcell.params_sc_cu()
        x, H = inputs.fcc(10, 10, 10, 3.615)
        cells = [dict(H0=H, x0=inputs.to_f32(np.mod(inputs.jitter(x, 0.1, 72), H[0, 0])))]
    else:
        prm = rcell.params_kg()
        x, H, bonds = inputs.kg_melt(20, 50, 0.85, seed=73, pushoff_iters=300)
        cells = [dict(H0=H, x0=inputs.to_f32(x), bonds=bonds)]
    with Ctx(prm, cells) as c:
        rcell.rcell_set_tuning(c.h, 0, 1)
        rcell.rcell_eval(c.h)
        pe, W = rcell.rcell_get_energy(c.h)
        x, _, f = rcell.rcell_get_atoms(c.h, 0, len(cells[0]["x0"]))
        H, _, _ = rcell.rcell_get_box(c.h, 0)
    fo, Wo, eo = oracle.forces(oracle_pot(prm), x, H, bonds=cells[0].get("bonds"))
    assert force_err(f, fo) <= 1e-5
    assert np.abs(W[0] - Wo).max() <= 1e-4 * np.abs(Wo).max()
    assert abs(pe[0] - eo) <= 1e-5 * max(abs(eo), 1.0)
