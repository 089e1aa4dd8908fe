"""GPU tests of the surrogate coupling: per-cell activity mask of the r-cell
batch, surrogate input features, and the FE step with surrogate + MD fallback."""
import numpy as np
import pytest

from _helpers import lj_cell
from oracle import mlp
from paper_1902_09171_gb300 import inputs, rcell
from paper_1902_09171_gb300 import surrogate as S

pytestmark = pytest.mark.gpu


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


def test_inactive_cells_are_frozen(torch):
    prm = rcell.params_lj_cu()
    cells = [lj_cell(4, seed=k) for k in range(3)]
    ctx = rcell.rcell_create(prm, cells)
    try:
        rcell.rcell_run(ctx, 10, 5)
        before = [rcell.rcell_get_atoms(ctx, k, 256)[:2] for k in range(3)]
        H_before = rcell.rcell_get_box(ctx, 1)[0]
        rcell.rcell_set_active(ctx, np.array([1, 0, 1], dtype=np.int32))
        rcell.rcell_set_deformation(ctx, np.stack([np.diag([1.01, 1, 1])] * 3))
        rcell.rcell_run(ctx, 10, 5)
        assert rcell.rcell_sync(ctx) == 0
        after = [rcell.rcell_get_atoms(ctx, k, 256)[:2] for k in range(3)]
        assert np.array_equal(before[1][0], after[1][0]) and np.array_equal(before[1][1], after[1][1])
        assert np.array_equal(rcell.rcell_get_box(ctx, 1)[0], H_before)
        assert not np.allclose(before[0][0], after[0][0])
        # re-enabled: the frozen cell takes the whole deformation since its last update in one remap
        rcell.rcell_set_active(ctx, np.array([1, 1, 1], dtype=np.int32))
        rcell.rcell_set_deformation(ctx, np.stack([np.diag([1.02, 1, 1])] * 3))
        H1 = rcell.rcell_get_box(ctx, 1)[0]
        assert abs(H1[0, 0] / H_before[0, 0] - 1.02) < 1e-6
    finally:
        rcell.rcell_destroy(ctx)


def test_features_match_oracle(torch):
    rng = np.random.default_rng(0)
    Fp = np.eye(3) + 0.05 * rng.standard_normal((37, 3, 3))
    F = Fp + 0.01 * rng.standard_normal((37, 3, 3))
    dFp = torch.tensor(Fp, dtype=torch.float64, device="cuda")
    dF = torch.tensor(F, dtype=torch.float64, device="cuda")
    u = torch.zeros((37, 15), dtype=torch.float32, device="cuda")
    S.sur_features(dFp, dF, u)
    torch.cuda.synchronize()
    ref = mlp.features(Fp, F)
    assert np.abs(u.cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()


def _bar(torch, K, seed):
    prm = rcell.params_lj_cu()
    cells = [lj_cell(4, seed=seed + k) for k in range(4)]
    L = cells[0]["H0"][0, 0]
    X, conn = inputs.hex_mesh(4, 1, 1, 4 * L, L, L)
    mask, val = inputs.uniaxial_bc(X, 4 * L)
    st = torch.cuda.current_stream()
    ctx = rcell.rcell_create(prm, cells, stream=st)
    fe = rcell.fe_create(X, conn, mask, val, 0.3, 0.05, 20.0, 0.0, stream=st)
    sur = S.sur_create(K, 4, 1, 3, stream=st)
    return ctx, fe, sur, X


def test_fe_step_surrogate_all_md_equals_fe_step(torch):
    st = torch.cuda.Stream()
    torch.cuda.set_stream(st)
    try:
        a = _bar(torch, 2, 10)
        b = _bar(torch, 2, 10)
        h = torch.zeros((2, 4, 128), dtype=torch.float32, device="cuda")
        Fp = torch.eye(3, dtype=torch.float64, device="cuda").repeat(4, 1, 1).contiguous()
        flag = torch.zeros(4, dtype=torch.int32, device="cuda")
        nn = a[3].shape[0]
        for k, lam in enumerate([0.002, 0.004]):
            rcell.fe_step(a[1], a[0], lam, 20, 10, None)
            n = rcell.fe_step_surrogate(b[1], b[0], b[2], lam, 20, 10, 1e9, 1e9, 0.1, 1, h, Fp, flag)
            assert n == 4 and int(flag.min()) == 2  # forced, not tripped
        da, _ = rcell.fe_get_state(a[1], nn)
        db, _ = rcell.fe_get_state(b[1], nn)
        assert np.array_equal(da, db)
        assert np.abs(Fp.cpu().numpy()[:, 0, 0] - 1.0).max() > 0  # F_prev advanced
    finally:
        for c in (a, b):
            rcell.fe_destroy(c[1])
            rcell.rcell_destroy(c[0])
            S.sur_destroy(c[2])
        torch.cuda.set_stream(torch.cuda.default_stream())


def test_fe_step_surrogate_without_md_uses_the_surrogate_stress(torch):
    st = torch.cuda.Stream()
    torch.cuda.set_stream(st)
    ctx, fe, sur, X = _bar(torch, 2, 20)
    try:
        h = torch.zeros((2, 4, 128), dtype=torch.float32, device="cuda")
        Fp = torch.eye(3, dtype=torch.float64, device="cuda").repeat(4, 1, 1).contiguous()
        flag = torch.zeros(4, dtype=torch.int32, device="cuda")
        h2 = h.clone()
        n = rcell.fe_step_surrogate(fe, ctx, sur, 0.002, 20, 10, 1e9, 1e9, 0.1, 0, h, Fp, flag)
        assert n == 0 and int(flag.sum()) == 0
        P = torch.zeros((4, 3, 3), dtype=torch.float64, device="cuda")
        rcell.fe_get_P(fe, P)
        # the same increment through the surrogate alone
        F = Fp.clone()  # F_prev now holds this step's F
        u = torch.zeros((4, 15), dtype=torch.float32, device="cuda")
        S.sur_features(torch.eye(3, dtype=torch.float64, device="cuda").repeat(4, 1, 1).contiguous(), F, u)
        mean = torch.zeros((4, 6), dtype=torch.float32, device="cuda")
        spread = torch.zeros(4, dtype=torch.float32, device="cuda")
        S.sur_step(sur, u, h2, 0.1, mean, spread)
        torch.cuda.synchronize()
        assert torch.equal(h, h2)
        Fn, m = F.cpu().numpy(), mean.cpu().numpy().astype(np.float64)
        for e in range(4):
            sig = np.array([[m[e, 0], m[e, 3], m[e, 4]], [m[e, 3], m[e, 1], m[e, 5]], [m[e, 4], m[e, 5], m[e, 2]]])
            ref = np.linalg.det(Fn[e]) * sig @ np.linalg.inv(Fn[e]).T
            assert np.abs(P.cpu().numpy()[e] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    finally:
        rcell.fe_destroy(fe)
        rcell.rcell_destroy(ctx)
        S.sur_destroy(sur)
        torch.cuda.set_stream(torch.cuda.default_stream())
