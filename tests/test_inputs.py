"""The seeded host-side generators and helpers of the workloads (no GPU):
uneven cell sizes, deformation-gradient histories, the tensile deformation and
the surrogate's feature scales keep the properties their docstrings state."""
import numpy as np
import pytest

from paper_1902_09171_gb300 import inputs, pipeline


def test_uniform_sizes_are_seeded_bounded_multiples():
    s = inputs.uniform_sizes(64, 5000, 20000, 50, 3)
    assert s.shape == (64,) and np.all(s % 50 == 0)
    assert s.min() >= 5000 and s.max() <= 20000
    assert np.array_equal(s, inputs.uniform_sizes(64, 5000, 20000, 50, 3))
    assert not np.array_equal(s, inputs.uniform_sizes(64, 5000, 20000, 50, 4))
    assert len(np.unique(s)) > 32  # uneven: a spread of sizes, not one size


def test_strain_paths_start_at_identity_and_stay_in_their_bounds():
    n, T, ms, sh, jit, lat = 400, 60, 0.3, 0.08, 0.01, 0.1
    F = inputs.strain_paths(n, T, seed=11, max_strain=ms, max_shear=sh, jitter=jit, max_lateral=lat)
    assert F.shape == (n, T + 1, 3, 3)
    assert np.array_equal(F[:, 0], np.tile(np.eye(3), (n, 1, 1)))
    assert np.all(np.linalg.det(F) > 0)
    exx = F[:, :, 0, 0] - 1.0
    assert exx.max() <= ms + jit + 1e-12 and exx.min() >= -ms - jit - 1e-12
    mono = np.all(np.diff(exx, axis=1) * np.sign(exx[:, -1:]) >= -jit / 60 - 1e-12, axis=1)
    assert exx[mono, -1].min() >= -0.5 * ms - jit - 1e-12  # ramps go at most half as far in compression
    assert np.abs(F[:, :, 0, 1]).max() <= sh + jit + 1e-12
    for d in (1, 2):  # -nu eps_x with nu <= 1/2, plus a drift in [-lat, lat / 4]
        e = F[:, :, d, d] - 1.0
        assert e.max() <= 0.5 * ms + 0.25 * lat + jit + 1e-12
        assert e.min() >= -0.5 * ms - lat - jit - 1e-12
    # both kinds of axial history occur: monotone ramps and cycles (sign changes of the increment)
    inc = np.diff(exx, axis=1)
    cyclic = np.any(inc[:, 1:] * inc[:, :-1] < -1e-12, axis=1)
    assert 0.2 < cyclic.mean() < 0.8
    assert np.array_equal(F, inputs.strain_paths(n, T, seed=11, max_strain=ms, max_shear=sh, jitter=jit,
                                                 max_lateral=lat))


@pytest.mark.parametrize("nu", [0.0, 0.3, 0.5])
def test_tensile_F_is_a_uniaxial_stretch_with_lateral_contraction(nu):
    for eps in (-0.05, 0.0, 0.02, 0.3):
        F = pipeline.tensile_F(eps, nu)
        lam = 1.0 + eps
        assert np.array_equal(F, np.diag(np.diag(F)))
        assert F[0, 0] == lam and F[1, 1] == F[2, 2]
        assert abs(np.linalg.det(F) - lam ** (1.0 - 2.0 * nu)) <= 1e-15 * max(1.0, lam)


def test_feature_scales_floor_each_block_and_share_one_output_scale():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    U = rng.standard_normal((64, 10, 15))
    U[:, :, 3] *= 1e-6  # a barely excited increment component
    U[:, :, 12] *= 1e-6  # a barely excited strain component
    U[:, :, 9:] *= 7.0
    Y = rng.standard_normal((64, 10, 6)) * np.array([1.0, 2.0, 3.0, 0.1, 0.1, 0.1])
    u, y = pipeline.feature_scales(torch.tensor(U, dtype=torch.float32), torch.tensor(Y, dtype=torch.float32))
    assert u.shape == (15,) and y.shape == (6,)
    std = U.reshape(-1, 15).std(0, ddof=1)  # torch's unbiased estimator
    for a, b in ((0, 9), (9, 15)):
        assert np.all(u[a:b] >= 0.1 * std[a:b].max() * (1 - 1e-6))
        big = std[a:b] >= 0.1 * std[a:b].max()
        assert np.allclose(u[a:b][big], std[a:b][big], rtol=1e-5)
    assert np.allclose(u[3], 0.1 * std[0:9].max(), rtol=1e-5) and np.allclose(u[12], 0.1 * std[9:15].max(), rtol=1e-5)
    assert np.all(y == y[0]) and abs(y[0] - np.sqrt((Y ** 2).mean())) <= 1e-5 * y[0]


def test_bar_strain_paths_start_at_identity_and_stay_in_their_bounds():
    n, T, ax, sh, lat, jit = 300, 25, 0.15, 0.12, 0.05, 0.005
    F = inputs.bar_strain_paths(n, T, seed=13, max_axial=ax, max_shear=sh, max_lateral=lat, jitter=jit)
    assert F.shape == (n, T + 1, 3, 3)
    assert np.array_equal(F[:, 0], np.tile(np.eye(3), (n, 1, 1)))
    assert np.all(np.linalg.det(F) > 0)
    exx = F[:, :, 0, 0] - 1.0
    assert exx.max() <= ax + jit + 1e-12 and exx.min() >= -0.2 * ax - jit - 1e-12
    for (i, j) in ((0, 1), (0, 2), (1, 0), (2, 0)):
        assert np.abs(F[:, :, i, j]).max() <= sh + jit + 1e-12
        assert np.abs(F[:, -1, i, j]).max() > 0.5 * sh  # every shear is driven
    assert np.abs(F[:, :, 1, 2]).max() <= jit + 1e-12  # the other shears only jitter
    assert np.array_equal(F, inputs.bar_strain_paths(n, T, seed=13, max_axial=ax, max_shear=sh, max_lateral=lat,
                                                      jitter=jit))


def test_necking_mesh_has_the_imperfection_at_mid_length():
    h = 28.66
    X, conn = inputs.necking_mesh(32, 4, 4, h, 0.05)
    X0, conn0 = inputs.hex_mesh(32, 4, 4, 32 * h, 4 * h, 4 * h)
    assert np.array_equal(conn, conn0) and conn.shape == (512, 8)
    moved = np.any(X != X0, axis=1)
    assert np.allclose(X[moved, 0], 16 * h) and moved.sum() == 5 * 5 - 1  # the mid plane; its centre node stays
    mid = np.abs(X[:, 0] - 16 * h) < 1e-9
    area = (X[mid, 1].max() - X[mid, 1].min()) * (X[mid, 2].max() - X[mid, 2].min())
    assert np.isclose(area, 0.95 * (4 * h) ** 2, rtol=1e-12)
