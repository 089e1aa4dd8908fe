"""Pins of the oracle's MD-fallback decision (oracle/fallback.py): ensemble
statistics against closed forms, the trip / hysteresis / forced rules on
hand-built histories, and the merged first Piola-Kirchhoff stress against the
uniaxial closed form of Eq. Pmd."""
import numpy as np

from oracle import fallback as fb


def test_ensemble_stats_closed_forms():
    # two members at m +- d: sample variance per component 2 d^2, so the spread is
    # sqrt(2) |d| / |m|
    m = np.array([1.0, -2.0, 0.5, 0.0, 0.3, 0.0])
    d = np.array([0.1, 0.0, 0.0, 0.2, 0.0, 0.0])
    mean, spread = fb.ensemble_stats(np.stack([m + d, m - d])[:, None, :], 1e-9)
    assert np.allclose(mean[0], m, atol=1e-15)
    assert np.isclose(spread[0], np.sqrt(2.0) * np.linalg.norm(d) / np.linalg.norm(m), rtol=1e-14)
    # K = 4 members: unbiased (K - 1) normalisation
    S = np.array([[1.0] * 6, [2.0] * 6, [3.0] * 6, [4.0] * 6])[:, None, :]
    _, sp = fb.ensemble_stats(S, 1e-9)
    var = np.var([1.0, 2.0, 3.0, 4.0], ddof=1)
    assert np.isclose(sp[0], np.sqrt(6 * var) / np.sqrt(6 * 2.5 ** 2), rtol=1e-14)
    # identical members: zero spread; a single member: zero spread
    assert fb.ensemble_stats(np.ones((3, 2, 6)), 0.1)[1].max() == 0.0
    assert fb.ensemble_stats(np.ones((1, 2, 6)), 0.1)[1].max() == 0.0
    # the floor replaces a small mean norm
    S = np.stack([np.full(6, 1e-3), np.full(6, -1e-3)])[:, None, :]
    _, sp = fb.ensemble_stats(S, 0.5)
    assert np.isclose(sp[0], np.sqrt(6 * 2e-6) / 0.5, rtol=1e-14)


def test_decision_rules_on_a_scripted_history():
    on, off = 0.02, 0.01
    # spread history of one point and the flags the rules give, step by step
    hist = [(0.005, 1, 2), (0.030, 1, 1),   # forced increments; a trip wins over forcing
            (0.015, 0, 1),                  # above off while tripped: stays on MD
            (0.010, 0, 0),                  # at off (not above): released
            (0.015, 0, 0),                  # above off but not tripped before: surrogate
            (0.020, 0, 0),                  # at on (not above): surrogate
            (0.021, 0, 1), (0.011, 0, 1), (0.009, 0, 0),
            (float("nan"), 0, 1)]           # an undefined indicator falls back to MD
    flag = np.array([0])
    for s, force, want in hist:
        flag = fb.decide(np.array([s]), flag, on, off, force)
        assert flag[0] == want, (s, force, want, flag[0])
    # a forced point (flag 2) is not held by the hysteresis
    assert fb.decide(np.array([0.015]), np.array([2]), on, off, 0)[0] == 0
    # points are independent
    got = fb.decide(np.array([0.03, 0.015, 0.015, 0.0]), np.array([0, 1, 0, 1]), on, off, 0)
    assert got.tolist() == [1, 1, 0, 0]


def test_merged_stress_uniaxial_closed_form():
    # uniaxial stretch lambda with a uniaxial Cauchy stress s: P_xx = s / lambda * J = s
    # for J = lambda (no lateral contraction); the MD stress passes through unchanged
    lam, s = 1.05, 2.0
    F = np.stack([np.diag([lam, 1.0, 1.0])] * 2)
    s_mean = np.array([[s, 0, 0, 0, 0, 0]] * 2, dtype=np.float64)
    P_md = np.stack([np.full((3, 3), 7.0)] * 2)
    P = fb.merge_P(np.array([0, 1]), s_mean, F, P_md)
    assert np.isclose(P[0, 0, 0], s * lam / lam) and np.abs(P[0] - np.diag([s, 0, 0])).max() < 1e-15
    assert np.array_equal(P[1], P_md[1])
    # simple shear F = I + g e_x e_y with sigma_xy = t: P F^T = J sigma (symmetric)
    g, t = 0.1, 0.7
    F = np.eye(3)
    F[0, 1] = g
    P = fb.cauchy_to_pk1(F, [0, 0, 0, t, 0, 0])
    assert np.abs(P @ F.T - np.array([[0, t, 0], [t, 0, 0], [0, 0, 0]])).max() < 1e-15
