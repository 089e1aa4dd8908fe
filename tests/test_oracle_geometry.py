"""Pins of the oracle's coupling geometry (Sec. 2.1): QR split, Delta R, remap,
stress rotation and the first Piola-Kirchhoff stress (Eq. Pmd)."""
import json
import os

import numpy as np
import pytest

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1.json")))
CASES = list(GOLD["cases"].items())


def voigt(S):
    S = np.asarray(S)
    return np.array([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]])


@pytest.mark.parametrize("name,case", CASES)
def test_qr_reproduces_table1(name, case):
    # Table 1 prints F, Q, R to 3 decimals; the unique positive-diagonal QR of the
    # printed F must round to the printed Q and R (half a unit in the last place,
    # plus the rounding already present in the printed F).
    Q, R = oracle.qr(case["F"])
    assert np.abs(Q - np.array(case["Q"])).max() <= 5e-4 + 1e-12
    assert np.abs(R - np.array(case["R"])).max() <= 5e-4 + 1e-12


@pytest.mark.parametrize("name,case", CASES)
def test_qr_properties(name, case):
    F = np.array(case["F"])
    Q, R = oracle.qr(F)
    assert np.abs(Q.T @ Q - np.eye(3)).max() < 1e-14
    assert np.abs(np.tril(R, -1)).max() == 0.0
    assert np.all(np.diag(R) > 0)
    assert np.abs(Q @ R - F).max() < 1e-14
    assert abs(np.linalg.det(Q) - 1.0) < 1e-14


def test_qr_random_and_degenerate():
    rng = np.random.default_rng(0)
    for _ in range(200):
        F = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
        if np.linalg.det(F) <= 0:
            with pytest.raises(oracle.OracleError):
                oracle.qr(F)
            continue
        Q, R = oracle.qr(F)
        assert np.abs(Q @ R - F).max() < 1e-13
        assert np.all(np.diag(R) > 0)
        # uniqueness: any other QR with positive diagonal equals this one
        q2, r2 = np.linalg.qr(F)
        D = np.diag(np.sign(np.diag(r2)))
        assert np.abs(q2 @ D - Q).max() < 1e-12
    # det F <= 0 has no rotation + positive stretch: reported, not returned
    for F in (np.diag([1.0, 1.0, -1.0]), np.zeros((3, 3)), np.array([[1, 2, 3], [2, 4, 6], [0, 0, 1.0]])):
        with pytest.raises(oracle.OracleError) as e:
            oracle.qr(F)
        assert e.value.code == oracle.OR_EDEGEN


def test_rotation_only_F():
    # a pure rotation gives Q = F, R = I
    th = 0.3
    F = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    Q, R = oracle.qr(F)
    assert np.abs(R - np.eye(3)).max() < 1e-15
    assert np.abs(Q - F).max() < 1e-15


@pytest.mark.parametrize("name,case", CASES)
def test_rotation_reproduces_table1(name, case):
    # sigma_FEM = Q sigma_MD Q^T (Sec. 2.1); Table 1 prints both sides to 3 decimals.
    Q, R = oracle.qr(case["F"])
    s_fem, P = oracle.rotate_pk1(Q, case["F"], voigt(case["sigma_MD"]))
    assert np.abs(s_fem - voigt(case["sigma_FEM"])).max() <= 1.5e-3


@pytest.mark.parametrize("name,case", CASES)
def test_table1_symmetry_of_pattern_C(name, case):
    # a symmetric [111] load on a cubic crystal: equal diagonal and equal
    # off-diagonal FEM-frame stress components (Table 1, C(t)/C(c)); the oracle's
    # rotation of the printed sigma_MD keeps that symmetry to print precision.
    if not name.startswith("C"):
        return
    Q, _ = oracle.qr(case["F"])
    s_fem, _ = oracle.rotate_pk1(Q, case["F"], voigt(case["sigma_MD"]))
    assert np.ptp(s_fem[:3]) < 4e-3 and np.ptp(s_fem[3:]) < 4e-3


def test_pk1_balance_and_uniaxial():
    rng = np.random.default_rng(1)
    for _ in range(50):
        F = np.eye(3) + 0.2 * rng.standard_normal((3, 3))
        if np.linalg.det(F) <= 0:
            continue
        Q, R = oracle.qr(F)
        s = rng.standard_normal(6)
        s_fem, P = oracle.rotate_pk1(Q, F, s)
        J = np.linalg.det(F)
        S = np.array([[s_fem[0], s_fem[3], s_fem[4]], [s_fem[3], s_fem[1], s_fem[5]], [s_fem[4], s_fem[5], s_fem[2]]])
        # P F^T = J sigma (symmetric): angular momentum balance of Eq. Pmd
        assert np.abs(P @ F.T - J * S).max() < 1e-12
    # uniaxial stretch: P_xx = sigma_xx, P_yy = lambda sigma_yy
    lam = 1.05
    F = np.diag([lam, 1.0, 1.0])
    Q, R = oracle.qr(F)
    s_fem, P = oracle.rotate_pk1(Q, F, [2.0, 1.0, 1.0, 0, 0, 0])
    assert abs(P[0, 0] - 2.0) < 1e-14 and abs(P[1, 1] - lam) < 1e-14


def test_delta_R_and_remap_compose():
    # Eq. LAMMPS2: after remaps by successive Delta R the atoms sit at R(t) H0 S,
    # exactly the positions Eq. LAMMPS1 gives for the box H_MD = R H0.
    rng = np.random.default_rng(2)
    H0 = np.diag([10.0, 11.0, 12.0])
    S = rng.uniform(0, 1, (50, 3))
    x = S @ H0.T
    R_prev = np.eye(3)
    for k in range(5):
        F = np.eye(3) + 0.05 * (k + 1) * rng.standard_normal((3, 3)) * 0.3
        Q, R = oracle.qr(F)
        dR = oracle.delta_R(R, R_prev)
        assert np.abs(np.tril(dR, -1)).max() < 1e-15  # product of upper-triangular factors
        x = oracle.remap(x, dR)
        R_prev = R
    assert np.abs(x - S @ (R @ H0).T).max() < 1e-12


def test_box_widths():
    H = np.array([[10.0, 3.0, 1.0], [0, 8.0, 2.0], [0, 0, 9.0]])
    w = oracle.box_widths(H)
    a, b, c = H[:, 0], H[:, 1], H[:, 2]
    V = np.linalg.det(H)
    assert abs(w[0] - V / np.linalg.norm(np.cross(b, c))) < 1e-12
    assert abs(w[1] - V / np.linalg.norm(np.cross(c, a))) < 1e-12
    assert abs(w[2] - V / np.linalg.norm(np.cross(a, b))) < 1e-12
