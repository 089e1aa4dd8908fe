"""Pins of the oracle's 4-node tetrahedron FE (the paper's C3D4 element,
Sec. 3.2): closed-form shape-function gradients, linear completeness (patch
tests), traction balance, volume and mass, and convergence of the damped
explicit update to the static bar."""
import numpy as np

import oracle
from paper_1902_09171_gb300 import inputs


def distorted_tet_mesh(seed=0):
    X, conn = inputs.tet_mesh(3, 2, 2, 3.0, 2.0, 2.0)
    rng = np.random.default_rng(seed)
    interior = np.all((X > 1e-9) & (X < np.array([3.0, 2.0, 2.0]) - 1e-9), axis=1)
    X = X.copy()
    X[interior] += rng.uniform(-0.12, 0.12, (interior.sum(), 3))
    return X, conn


def _mesh(X, conn, mask=None, val=None, rho0=1.0, dt=0.1, damping=0.0):
    nn = len(X)
    mask = np.zeros((nn, 3), np.int32) if mask is None else mask
    val = np.zeros((nn, 3)) if val is None else val
    return oracle.FETetMesh(X, conn, mask, val, rho0, dt, damping)


def test_unit_tetrahedron_gradients_and_volume():
    # N = (1 - x - y - z, x, y, z) on the unit right tetrahedron: constant gradients by hand
    X = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    fe = _mesh(X, np.array([[0, 1, 2, 3]]), rho0=6.0)
    assert abs(fe.V0[0] - 1.0 / 6.0) < 1e-15
    ref = np.array([[-1.0, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    assert np.abs(fe.gradN[0] - ref).max() < 1e-15
    assert np.allclose(fe.mass, 0.25)
    # an inverted tetrahedron is rejected
    try:
        _mesh(X, np.array([[0, 2, 1, 3]]))
        raise AssertionError("inverted element accepted")
    except oracle.OracleError as e:
        assert e.code == oracle.OR_EDEGEN


def test_mesh_volume_mass_and_partition_of_unity():
    X, conn = distorted_tet_mesh(2)
    fe = _mesh(X, conn, rho0=2.5)
    assert abs(fe.V0.sum() - 12.0) < 1e-12 and np.all(fe.V0 > 0)
    assert abs(fe.mass.sum() - 2.5 * 12.0) < 1e-11
    assert np.abs(fe.gradN.sum(1)).max() < 1e-13  # sum_a grad N_a = 0


def test_patch_test_affine_and_rotation_fields_give_exact_F():
    X, conn = distorted_tet_mesh(3)
    fe = _mesh(X, conn)
    A = np.array([[0.02, 0.01, -0.03], [0.005, -0.01, 0.02], [0.0, 0.015, 0.01]])
    fe.d = X @ A.T + np.array([0.3, -0.1, 0.2])
    assert np.abs(fe.F() - (np.eye(3) + A)).max() < 1e-14
    th = 0.7
    Q = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    fe.d = X @ (Q - np.eye(3)).T
    assert np.abs(fe.F() - Q).max() < 1e-14


def test_uniform_P_balances_interior_nodes_and_face_traction():
    X, conn = distorted_tet_mesh(4)
    fe = _mesh(X, conn)
    P = np.array([[1.0, 0.2, -0.3], [0.1, 2.0, 0.4], [-0.2, 0.3, 1.5]])
    fint = fe.update(np.tile(P, (fe.ne, 1, 1)))
    interior = np.all((X > 1e-9) & (X < np.array([3.0, 2.0, 2.0]) - 1e-9), axis=1)
    assert np.abs(fint[interior]).max() < 1e-13
    xL = np.abs(X[:, 0] - 3.0) < 1e-9
    assert np.allclose(fint[xL].sum(0), P[:, 0] * 4.0, atol=1e-12)
    assert np.abs(fint.sum(0)).max() < 1e-12


def test_damped_explicit_update_reaches_static_bar_solution():
    # linear material P = E (F - I), ends pulled apart, lateral faces free: the
    # static solution u_x = lambda X, u_y = u_z = 0 (zero Poisson ratio); tets
    # have no hourglass modes, so no stabilisation is needed
    L = 4.0
    X, conn = inputs.tet_mesh(4, 1, 1, L, 1.0, 1.0)
    mask, val = inputs.uniaxial_bc(X, L)
    Emod, rho0 = 10.0, 1.0
    dt = 0.2 / np.sqrt(Emod / rho0)
    fe = _mesh(X, conn, mask, val, rho0, dt, 2.0)
    lam = 0.01
    for _ in range(4000):
        fe.apply_bc(lam)
        fe.update(Emod * (fe.F() - np.eye(3)))
    assert np.abs(fe.d[:, 0] - lam * X[:, 0]).max() < 1e-8
    assert np.abs(fe.d[:, 1:]).max() < 1e-8
