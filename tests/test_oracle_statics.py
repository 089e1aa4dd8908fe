"""Pins of the molecular-statics part of the FP64 oracle (Sec. 2.2):
Eq. PK1 (first Piola-Kirchhoff stress from the pair sum with reference
separations) and the FIRE energy minimiser behind Eq. CGPR1."""
import numpy as np
import pytest

import oracle
from paper_1902_09171_gb300 import inputs
from test_oracle_forces import LJ_CU, _fcc_lattice_sums, lj_cu, sc_cu


def _affine_case(kind):
    """Reference box H0 (orthogonal), reference positions X, potential, bonds, units."""
    if kind == "lj":
        X, H0 = inputs.fcc(4, 4, 4, 3.615)
        return inputs.jitter(X, 0.08, 21), H0, lj_cu(), None, 0
    if kind == "sc":
        X, H0 = inputs.fcc(5, 5, 5, 3.615)
        return inputs.jitter(X, 0.08, 22), H0, sc_cu(), None, 0
    X, H0, bonds = inputs.kg_melt(8, 20, 0.85, seed=23, pushoff_iters=200)
    return X, H0, oracle.pot_kg(), bonds, 1


@pytest.mark.parametrize("kind", ["lj", "sc", "kg"])
def test_pk1_is_the_energy_derivative_with_respect_to_F(kind):
    # P = (1 / Omega_0) dE/dF for the affine family x = F X, H = F H0 (the
    # definition Eq. PK1 restates); a general, non-symmetric F
    X, H0, pot, bonds, units = _affine_case(kind)
    rng = np.random.default_rng(5)
    F = np.eye(3) + 0.03 * rng.standard_normal((3, 3))
    P = oracle.pk1_pairs(pot, X @ F.T, F @ H0, H0, bonds=bonds, units=units)
    pconv = oracle.lib().or_pconv(units)
    omega0 = np.linalg.det(H0)
    h = 1e-6
    for a in range(3):
        for b in range(3):
            dF = np.zeros((3, 3))
            dF[a, b] = h
            ep = oracle.forces(pot, X @ (F + dF).T, (F + dF) @ H0, bonds=bonds)[2]
            em = oracle.forces(pot, X @ (F - dF).T, (F - dF) @ H0, bonds=bonds)[2]
            fd = pconv * (ep - em) / (2 * h) / omega0
            assert abs(P[a, b] - fd) <= 1e-6 * max(1.0, np.abs(P).max()), (a, b, P[a, b], fd)


@pytest.mark.parametrize("kind", ["lj", "sc", "kg"])
def test_pk1_times_R_transpose_is_the_virial_stress(kind):
    # in the MD box H = R H0: P R^T / J = -W / V (potential part of the virial
    # stress, tension-positive), for the same configuration
    X, H0, pot, bonds, units = _affine_case(kind)
    R = np.array([[1.04, 0.03, -0.02], [0.0, 0.98, 0.05], [0.0, 0.0, 1.01]])
    x, H = X @ R.T, R @ H0
    P = oracle.pk1_pairs(pot, x, H, H0, bonds=bonds, units=units)
    _, W, _ = oracle.forces(pot, x, H, bonds=bonds)
    sigma = -oracle.lib().or_pconv(units) * W / np.linalg.det(H)
    lhs = P @ R.T / np.linalg.det(R)
    assert np.abs(lhs - sigma).max() <= 1e-10 * max(1.0, np.abs(sigma).max())
    assert np.abs(lhs - lhs.T).max() <= 1e-10 * max(1.0, np.abs(sigma).max())


def test_fire_relaxes_a_jittered_crystal_to_the_lattice():
    # Eq. CGPR1 on a perfect FCC crystal: the minimum is the lattice itself (up
    # to a rigid translation), with the closed-form lattice energy
    a = 3.615
    X, H0 = inputs.fcc(4, 4, 4, a)
    x0 = inputs.jitter(X, 0.05, 31)
    pot = lj_cu()
    x, iters = oracle.fire_minimize(pot, x0, H0, 63.546, 1e-8, 2e-3, 2e-2, 5000)
    assert 0 < iters < 5000
    f, _, e = oracle.forces(pot, x, H0)
    assert np.sqrt((f ** 2).sum(1)).max() < 1e-8
    eps, sig, rc = LJ_CU["eps"], LJ_CU["sigma"], LJ_CU["rc"]
    ref = _fcc_lattice_sums(a, rc, lambda r: 0.5 * np.sum(4 * eps * ((sig / r) ** 12 - (sig / r) ** 6)))
    assert abs(e / len(x) - ref) <= 1e-10 * abs(ref)
    shift = (x - X).mean(0)
    assert np.abs(x - X - shift).max() < 1e-6
    # (the jittered start can sit lower in energy: with plain truncation, jitter
    # pulls some pairs of the fifth shell, 0.02 A outside rc, inside it; the
    # forces do not see that step, so the minimiser returns to the lattice)


def test_fire_stops_at_once_when_already_relaxed_and_reports_non_convergence():
    X, H0 = inputs.fcc(4, 4, 4, 3.615)
    x, iters = oracle.fire_minimize(lj_cu(), X, H0, 63.546, 1e-6, 2e-3, 2e-2, 100)
    assert iters == 0 and np.array_equal(x, X)
    x0 = inputs.jitter(X, 0.05, 32)
    _, it2 = oracle.fire_minimize(lj_cu(), x0, H0, 63.546, 1e-12, 2e-3, 2e-2, 3)
    assert it2 == -1


def test_fire_move_cap_limits_every_atom_displacement():
    # a melt straight from the generator has overlaps and large forces: one
    # iteration with the cap moves no atom by more than dmax, and the cap is
    # only active where the uncapped move would be larger
    x0, H, bonds = inputs.kg_melt(6, 20, 0.85, seed=33, pushoff_iters=20)
    pot = oracle.pot_kg()
    x1, _ = oracle.fire_minimize(pot, x0, H, 1.0, 1e-12, 0.005, 0.05, 1, bonds=bonds, units=1, dmax=0.01)
    d = np.linalg.norm(x1 - x0, axis=1)
    assert d.max() <= 0.01 * (1 + 1e-12)
    x2, _ = oracle.fire_minimize(pot, x0, H, 1.0, 1e-12, 0.005, 0.05, 1, bonds=bonds, units=1)
    d2 = np.linalg.norm(x2 - x0, axis=1)
    capped = d2 > 0.01
    assert capped.any() and np.allclose(d[~capped], d2[~capped], rtol=0, atol=1e-15)
    # a capped relaxation of the melt ends at a minimum without breaking bonds
    xm, it = oracle.fire_minimize(pot, x0, H, 1.0, 1e-6, 0.005, 0.05, 20000, bonds=bonds, units=1, dmax=0.05)
    assert it > 0
    f, _, _ = oracle.forces(pot, xm, H, bonds=bonds)
    assert np.sqrt((f ** 2).sum(1)).max() < 1e-6
