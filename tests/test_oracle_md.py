"""Pins of the oracle's fixed-box MD (velocity Verlet + Langevin), its random
numbers, its stress estimator and its sampling statistics."""
import numpy as np
import pytest

import oracle
from paper_1902_09171_gb300 import inputs

M_CU = 63.546
KB = inputs.KB_EV


def test_philox_statistics():
    # uniform 32-bit words: byte histogram flat, bits balanced, no repeats
    words = np.array([oracle.philox([i, 7, 3, 0], [12345, 678]) for i in range(20000)]).ravel()
    assert len(np.unique(words)) == len(words)
    bits = np.unpackbits(words.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.002
    hist = np.bincount((words >> 24).astype(np.int64), minlength=256)
    chi2 = ((hist - len(words) / 256) ** 2 / (len(words) / 256)).sum()
    assert chi2 < 256 + 6 * np.sqrt(2 * 256)
    # a one-bit change in counter or key changes about half the output bits
    base = oracle.philox([1, 2, 3, 4], [5, 6])
    for ctr, key in (([1, 2, 3, 5], [5, 6]), ([1, 2, 3, 4], [5, 7]), ([0x80000001, 2, 3, 4], [5, 6])):
        o = oracle.philox(ctr, key)
        flips = np.unpackbits((o ^ base).view(np.uint8)).sum()
        assert 40 < flips < 88


def test_normals_statistics():
    z = np.array([oracle.normals3(t, 1, e, 99) for t in range(300) for e in range(40)]).ravel()
    n = len(z)
    assert abs(z.mean()) < 4 / np.sqrt(n)
    assert abs(z.var() - 1) < 4 * np.sqrt(2 / n)
    assert abs((z ** 4).mean() - 3) < 0.15
    # the three components of one draw are uncorrelated
    Z = z.reshape(-1, 3)
    c = np.corrcoef(Z.T)
    assert np.abs(c - np.eye(3)).max() < 4 / np.sqrt(len(Z))


def test_maxwell_sampling():
    n, kT = 4000, 300 * KB
    v = inputs.maxwell(n, M_CU, kT, 0, 3)
    assert np.abs(v.sum(0)).max() < 1e-9
    T = (M_CU * (v ** 2).sum() / inputs.vel_unit_sq(0)) / (3 * n * KB)
    assert abs(T - 300) < 300 * 4 * np.sqrt(2 / (3 * n))


def test_block_stats():
    rng = np.random.default_rng(0)
    # iid: SE ~= std / sqrt(n)
    y = rng.standard_normal(4096)
    m, se = oracle.block_stats(y)
    assert abs(m - y.mean()) < 1e-14
    assert 0.8 < se / (y.std(ddof=1) / np.sqrt(len(y))) < 1.4
    # AR(1) with phi = 0.9: SE of the mean -> sqrt((1+phi)/(1-phi)) * std / sqrt(n)
    phi, n = 0.9, 1 << 15
    e = rng.standard_normal(n)
    y = np.zeros(n)
    for t in range(1, n):
        y[t] = phi * y[t - 1] + e[t]
    m, se = oracle.block_stats(y)
    ref = np.sqrt((1 + phi) / (1 - phi)) * np.sqrt(1 / (1 - phi * phi)) / np.sqrt(n)
    assert 0.75 < se / ref < 1.5
    # tiny series
    assert oracle.block_stats(np.array([1.0]))[1] == 0.0


def test_nve_energy_conservation():
    # Langevin off, dt = 1 fs.  The cutoff is placed inside the gap between the
    # 4th (5.11 A) and 5th (5.72 A) FCC shells so that no pair crosses it during
    # the run; unshifted truncation otherwise adds a jump of U(rc) per crossing.
    x, H = inputs.fcc(4, 4, 4, 3.615)
    n = len(x)
    pot = oracle.pot_lj(0.415, 2.277, 5.41)
    md = oracle.MD(0, M_CU, 300 * KB, 0.0, 0.001, 1)
    v = inputs.maxwell(n, M_CU, 300 * KB, 0, 1)
    _, _, ev, ss, pe, ke = oracle.md_run(pot, md, x, v, H, n_steps=2000, n_avg=2000)
    E = (pe + ke) / n
    assert np.abs(E - E[0]).max() < 1e-4 * 0.415
    slope = np.polyfit(np.arange(len(E)), E, 1)[0] * len(E)
    assert abs(slope) < 2e-5 * 0.415
    assert ev == 2001


def test_langevin_temperature_and_ideal_gas_stress():
    # non-interacting particles (epsilon = 0) under the thermostat: <T> = target
    # and the tension-positive stress is -rho kT on the diagonal
    x, H = inputs.fcc(3, 3, 3, 3.615)
    n = len(x)
    pot = oracle.pot_lj(0.0, 2.277, 0.5)
    kT = 300 * KB
    md = oracle.MD(0, M_CU, kT, 0.1, 0.002, 11)
    _, _, _, ss, pe, ke = oracle.md_run(pot, md, x, np.zeros_like(x), H, n_steps=3000, n_avg=2500)
    T = ke.mean() / (1.5 * n * KB)
    assert abs(T - 300) < 300 * 0.05
    p_ideal = n * kT / np.linalg.det(H) * oracle.pconv(0)
    mean_diag = ss[:, :3].mean()
    assert abs(mean_diag + p_ideal * T / 300) < 0.05 * p_ideal
    assert np.abs(ss[:, 3:].mean(0)).max() < 0.1 * p_ideal


def test_langevin_thermalises_interacting_crystal():
    x, H = inputs.fcc(3, 3, 3, 3.615)
    n = len(x)
    kT = 300 * KB
    md = oracle.MD(0, M_CU, kT, 0.1, 0.002, 5)
    _, _, _, ss, pe, ke = oracle.md_run(oracle.pot_lj(0.415, 2.277, 5.41), md, x, np.zeros_like(x), H,
                                         n_steps=2500, n_avg=1500)
    assert abs(ke.mean() / (1.5 * n * KB) - 300) < 300 * 0.06


def test_md_run_semantics():
    x, H = inputs.fcc(3, 3, 3, 3.615)
    n = len(x)
    pot = oracle.pot_lj(0.415, 2.277, 5.41)
    md = oracle.MD(0, M_CU, 300 * KB, 0.1, 0.002, 1)
    v = inputs.maxwell(n, M_CU, 300 * KB, 0, 2)
    # zero steps: nothing happens, no random numbers consumed
    x0, v0, ev0, *_ = oracle.md_run(pot, md, x, v, H, n_steps=0)
    assert ev0 == 0 and np.array_equal(x0, x) and np.array_equal(v0, v)
    # a run consumes n_steps + 1 force evaluations; reruns are deterministic
    a = oracle.md_run(pot, md, x, v, H, ev=5, n_steps=10, n_avg=4)
    b = oracle.md_run(pot, md, x, v, H, ev=5, n_steps=10, n_avg=4)
    assert a[2] == 16 and np.array_equal(a[0], b[0]) and np.array_equal(a[3], b[3])
    # another seed or another cell id gives another trajectory
    md2 = oracle.MD(0, M_CU, 300 * KB, 0.1, 0.002, 2)
    c = oracle.md_run(pot, md2, x, v, H, ev=5, n_steps=10, n_avg=4)
    d = oracle.md_run(pot, md, x, v, H, cell=3, ev=5, n_steps=10, n_avg=4)
    assert not np.allclose(a[0], c[0]) and not np.allclose(a[0], d[0])
    # splitting a run in two (state carried over) equals one run when the
    # second part's setup force matches: with the thermostat off that holds exactly
    md0 = oracle.MD(0, M_CU, 300 * KB, 0.0, 0.002, 1)
    one = oracle.md_run(pot, md0, x, v, H, n_steps=20)
    half = oracle.md_run(pot, md0, x, v, H, n_steps=10)
    two = oracle.md_run(pot, md0, half[0], half[1], H, ev=half[2], n_steps=10)
    assert np.abs(one[0] - two[0]).max() < 1e-12 and np.abs(one[1] - two[1]).max() < 1e-12


def test_kinetic_stress_term():
    # one moving particle, no interactions: sigma = -m v (x) v / V (tension-positive)
    H = np.diag([20.0, 20.0, 20.0])
    v = np.array([[1.0, 2.0, 3.0]])
    s = oracle.stress_inst(0, M_CU, v, np.zeros((3, 3)), H)
    K = M_CU * np.outer(v[0], v[0]) / inputs.vel_unit_sq(0)
    ref = -K / 8000.0 * oracle.pconv(0)
    assert np.allclose(s, [ref[0, 0], ref[1, 1], ref[2, 2], ref[0, 1], ref[0, 2], ref[1, 2]], rtol=1e-14)
