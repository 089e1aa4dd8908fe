"""Pins of the oracle's finite-element update (Sec. 2.2, Eq. f): hex-8 with one
centroid quadrature point, lumped mass, hourglass control, explicit update."""
import numpy as np

import oracle
from paper_1902_09171_gb300 import inputs


def distorted_mesh(seed=0):
    X, conn = inputs.hex_mesh(3, 2, 2, 3.0, 2.0, 2.0)
    rng = np.random.default_rng(seed)
    interior = np.all((X > 1e-9) & (X < np.array([3.0, 2.0, 2.0]) - 1e-9), axis=1)
    X = X.copy()
    X[interior] += rng.uniform(-0.15, 0.15, (interior.sum(), 3))
    return X, conn


def test_patch_test_affine_field_gives_uniform_F():
    X, conn = distorted_mesh()
    A = np.array([[0.02, 0.01, -0.03], [0.005, -0.01, 0.02], [0.0, 0.015, 0.01]])
    mask = np.zeros((len(X), 3), np.int32)
    fe = oracle.FEMesh(X, conn, mask, np.zeros((len(X), 3)), 1.0, 0.1, 0.0, 0.0)
    fe.d = X @ A.T + np.array([0.3, -0.1, 0.2])
    F = fe.F()
    assert np.abs(F - (np.eye(3) + A)).max() < 1e-14


def test_uniform_P_leaves_interior_nodes_free_of_force():
    X, conn = distorted_mesh(1)
    mask = np.zeros((len(X), 3), np.int32)
    fe = oracle.FEMesh(X, conn, mask, np.zeros((len(X), 3)), 1.0, 0.1, 0.0, 0.5)
    P = np.array([[1.0, 0.2, -0.3], [0.1, 2.0, 0.4], [-0.2, 0.3, 1.5]])
    fint = fe.update(np.tile(P, (fe.ne, 1, 1)))
    interior = np.all((X > 1e-9) & (X < np.array([3.0, 2.0, 2.0]) - 1e-9), axis=1)
    assert np.abs(fint[interior]).max() < 1e-13
    # boundary: total force on the x = L face equals P n A (traction), n = +x
    xL = np.abs(X[:, 0] - 3.0) < 1e-9
    assert np.allclose(fint[xL].sum(0), P[:, 0] * 4.0, atol=1e-12)
    assert np.abs(fint.sum(0)).max() < 1e-12


def test_hourglass_orthogonal_to_linear_fields():
    X, conn = distorted_mesh(2)
    Xe = X[conn[0]]
    g, V = oracle.hex8_geometry(Xe)
    rng = np.random.default_rng(3)
    A = 0.05 * rng.standard_normal((3, 3))
    de = Xe @ A.T + rng.standard_normal(3)
    f_hg = oracle.hex8_fint(Xe, g, V, np.zeros((3, 3)), de, hg_coef=7.0)
    assert np.abs(f_hg).max() < 1e-13
    # an hourglass mode (xi*eta pattern in u_z) is resisted
    nat = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1], [-1, -1, 1], [1, -1, 1], [1, 1, 1],
                    [-1, 1, 1]], float)
    de = np.zeros((8, 3))
    de[:, 2] = 0.01 * nat[:, 0] * nat[:, 1]
    f_hg = oracle.hex8_fint(Xe, g, V, np.zeros((3, 3)), de, hg_coef=7.0)
    assert (f_hg * de).sum() > 0  # restoring: positive work against the mode
    assert np.abs(oracle.hex8_F(g, de) - np.eye(3)).max() < 0.02  # barely seen by the centroid F


def test_geometry_volume_and_mass():
    X, conn = inputs.hex_mesh(2, 2, 1, 2.0, 3.0, 1.5)
    H = np.array([[1.0, 0.2, 0.1], [0.0, 1.1, -0.2], [0.0, 0.0, 0.9]])  # affine map: parallelepipeds
    X = X @ H.T
    fe = oracle.FEMesh(X, conn, np.zeros((len(X), 3), np.int32), np.zeros((len(X), 3)), 2.5, 0.1, 0.0, 0.0)
    assert abs(fe.V0.sum() - 2.0 * 3.0 * 1.5 * np.linalg.det(H)) < 1e-12
    assert abs(fe.mass.sum() - 2.5 * fe.V0.sum()) < 1e-12


def test_single_element_uniaxial_bc_gives_exact_F():
    X, conn = inputs.hex_mesh(1, 1, 1, 14.46, 14.46, 14.46)
    mask, val = inputs.uniaxial_bc(X, 14.46, all_nodes=True)
    fe = oracle.FEMesh(X, conn, mask, val, 1.0, 0.1, 0.0, 0.0)
    for lam in (0.002, 0.01, 0.02):
        fe.apply_bc(lam)
        assert np.abs(fe.F()[0] - np.diag([1 + lam, 1.0, 1.0])).max() < 1e-15


def test_damped_explicit_update_reaches_static_bar_solution():
    # linear material P = E (F - I): with ends pulled apart and lateral faces free
    # the static solution is u_x = lambda X everywhere; the damped explicit update
    # (lumped mass, assembly of Eq. f) must converge to it.
    L = 4.0
    X, conn = inputs.hex_mesh(4, 1, 1, L, 1.0, 1.0)
    mask, val = inputs.uniaxial_bc(X, L)
    Emod, rho0 = 10.0, 1.0
    h = 1.0
    dt = 0.3 * h / np.sqrt(Emod / rho0)
    fe = oracle.FEMesh(X, conn, mask, val, rho0, dt, 2.0, 0.1 * Emod)
    lam = 0.01
    for _ in range(3000):
        fe.apply_bc(lam)
        F = fe.F()
        P = Emod * (F - np.eye(3))
        fe.update(P)
    assert np.abs(fe.d[:, 0] - lam * X[:, 0]).max() < 1e-8
    assert np.abs(fe.d[:, 1:]).max() < 1e-8


def test_affine_predictor_moves_free_nodes_affinely():
    # with g = (X_x, 0, 0) and the end faces prescribed consistently, the predicted
    # displacement of every node is lambda X_x: every element (a distorted mesh
    # included) has F = I + lambda e_x (x) e_x exactly, increment after increment
    X, conn = inputs.hex_mesh(4, 2, 2, 4.0, 2.0, 2.0)
    rng = np.random.default_rng(3)
    inner = np.all((X > 1e-9) & (X < np.array([4.0, 2.0, 2.0]) - 1e-9), axis=1)
    X[inner] += rng.uniform(-0.15, 0.15, (inner.sum(), 3))
    mask, val = inputs.uniaxial_bc(X, 4.0)
    m = oracle.FEMesh(X, conn, mask, val, 1.0, 0.05, 0.5, 0.1)
    g = np.zeros_like(X)
    g[:, 0] = X[:, 0]
    m.set_predictor(g)
    for lam in (0.01, 0.025, 0.03):
        m.apply_bc(lam)
        F = m.F()
        assert np.abs(F - np.diag([1.0 + lam, 1.0, 1.0])).max() < 1e-13
        assert np.abs(m.d[:, 0] - lam * X[:, 0]).max() < 1e-13
    # without the predictor only the prescribed DOFs move
    m2 = oracle.FEMesh(X, conn, mask, val, 1.0, 0.05, 0.5, 0.1)
    m2.apply_bc(0.01)
    assert np.abs(m2.d[mask == 0]).max() == 0.0
