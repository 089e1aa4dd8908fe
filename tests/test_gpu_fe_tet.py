"""The 4-node tetrahedron FE (the paper's C3D4 element, Sec. 3.2) on the GPU,
through the C ABI: geometry, F, assembly and the explicit update against the
FP64 oracle (FP64 on both sides: 1e-12), and an FE-MD coupled step with one
r-cell per tetrahedron."""
import numpy as np
import pytest

import oracle
from _helpers import lj_cell
from paper_1902_09171_gb300 import inputs, rcell

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


def test_tet_fe_matches_oracle():
    X, conn = inputs.tet_mesh(3, 2, 2, 3.0, 2.0, 2.0)
    rng = np.random.default_rng(5)
    inner = np.all((X > 1e-9) & (X < np.array([3.0, 2.0, 2.0]) - 1e-9), axis=1)
    X[inner] += rng.uniform(-0.1, 0.1, (inner.sum(), 3))
    mask, val = inputs.uniaxial_bc(X, 3.0)
    args = (X, conn, mask, val, 1.3, 0.05, 0.7)
    fe = rcell.fe_create_tet4(*args)
    ref = oracle.FETetMesh(*args)
    try:
        for lam in (0.01, 0.02, 0.03):
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


def test_inverted_tetrahedron_is_rejected():
    X = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    z = np.zeros((4, 3))
    with pytest.raises(rcell.RCellError):
        rcell.fe_create_tet4(X, np.array([[0, 2, 1, 3]]), z.astype(np.int32), z, 1.0, 0.1, 0.0)


def test_fe_step_on_tetrahedra_prescribes_uniaxial_F():
    # six tetrahedra of one cube with every node prescribed: each element, and
    # so each r-cell behind it, sees exactly F = diag(1 + lambda, 1, 1)
    prm = rcell.params_lj_cu()
    L = lj_cell(4)["H0"][0, 0]
    X, conn = inputs.tet_mesh(1, 1, 1, L, L, L)
    mask, val = inputs.uniaxial_bc(X, L, all_nodes=True)
    fe = rcell.fe_create_tet4(X, conn, mask, val, 1.0, 0.01, 0.0)
    cells = [lj_cell(4, seed=20 + k) for k in range(len(conn))]
    ctx = rcell.rcell_create(prm, cells)
    try:
        u = np.zeros((len(X), 3))
        for k in (1, 2):
            rcell.fe_step(fe, ctx, 0.002 * k, 40, 20, u)
            for c in range(len(conn)):
                H, Q, R = rcell.rcell_get_box(ctx, c)
                assert np.abs(R - np.diag([1 + 0.002 * k, 1, 1])).max() < 1e-15
                assert np.abs(Q - np.eye(3)).max() < 1e-15
        P = np.zeros((len(conn), 3, 3))
        rcell.fe_get_P(fe, P)
        assert np.all(np.isfinite(P)) and np.abs(P).max() > 0
    finally:
        rcell.fe_destroy(fe)
        rcell.rcell_destroy(ctx)
