"""Pins of the oracle's force / energy / virial evaluation (the MD engine of Sec. 2.1
and the polymer model of Sec. 3.2: LJ, Sutton-Chen EAM, Kremer-Grest FENE+WCA)."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1902_09171_gb300 import inputs

LJ_CU = dict(eps=0.415, sigma=2.277, rc=2.5 * 2.277)
SC_CU = dict(eps=1.2382e-2, a=3.61, rc=7.22, n=9.0, m=6.0, c=39.432)


def lj_cu():
    return oracle.pot_lj(LJ_CU["eps"], LJ_CU["sigma"], LJ_CU["rc"])


def sc_cu():
    return oracle.pot_sc(SC_CU["eps"], SC_CU["a"], SC_CU["rc"], SC_CU["n"], SC_CU["m"], SC_CU["c"])


def random_cell(n, H, dmin, seed):
    rng = np.random.default_rng(seed)
    pts = []
    Hi = np.linalg.inv(H)
    while len(pts) < n:
        p = H @ rng.uniform(0, 1, 3)
        ok = True
        for q in pts:
            d = Hi @ (p - q)
            d -= np.round(d)
            if np.linalg.norm(H @ d) < dmin:
                ok = False
                break
        if ok:
            pts.append(p)
    return np.array(pts)


def tiny_cells():
    # 4..32 atoms in reduced LJ units, rc = 2.5; boxes with 2 and 3 bins per axis,
    # orthogonal and tilted (every perpendicular width >= 2 rc)
    out = []
    for k, (n, H) in enumerate([
        (4, np.diag([5.2, 5.3, 5.4])),
        (12, np.diag([5.1, 5.1, 7.6])),
        (32, np.diag([7.6, 7.7, 7.8])),
        (20, np.array([[6.0, 1.0, 0.5], [0, 6.2, -0.8], [0, 0, 6.4]])),
        (27, np.array([[8.0, 2.0, 1.5], [0, 7.5, 1.0], [0, 0, 7.9]])),
    ]):
        out.append((random_cell(n, H, 0.9, 10 + k), H))
    return out


@pytest.mark.parametrize("kind", ["lj", "sc"])
def test_brute_force_equals_cell_list_tiny(kind):
    for x, H in tiny_cells():
        pot = oracle.pot_lj(1.0, 1.0, 2.5) if kind == "lj" else oracle.pot_sc(0.1, 1.0, 2.5, 9, 6, 30.0)
        f1, W1, e1 = oracle.forces(pot, x, H, use_cells=False)
        f2, W2, e2 = oracle.forces(pot, x, H, use_cells=True)
        scale = np.abs(f1).max() + 1e-300
        assert np.abs(f1 - f2).max() <= 1e-12 * scale
        assert abs(e1 - e2) <= 1e-12 * abs(e1)
        assert np.abs(W1 - W2).max() <= 1e-12 * np.abs(W1).max()
        # the neighbour sets agree as sets
        p1 = {tuple(p) for p in oracle.neighbor_pairs(x, H, 2.5, use_cells=False)}
        p2 = {tuple(p) for p in oracle.neighbor_pairs(x, H, 2.5, use_cells=True)}
        assert p1 == p2


def test_pair_set_by_explicit_images():
    # brute force over a much larger image range (+-2) finds the same ordered pairs
    for x, H in tiny_cells():
        rc = 2.5
        ref = set()
        n = len(x)
        for i in range(n):
            for j in range(n):
                for t in itertools.product(range(-2, 3), repeat=3):
                    if i == j and t == (0, 0, 0):
                        continue
                    d = x[j] + H @ np.array(t, float) - x[i]
                    if d @ d < rc * rc:
                        ref.add((i, j))
        got = {tuple(p) for p in oracle.neighbor_pairs(x, H, rc, use_cells=True)}
        assert got == ref


@pytest.mark.parametrize("kind", ["lj", "sc", "kg"])
def test_newton_third_law_and_force_fd(kind):
    if kind == "lj":
        x, H = inputs.fcc(4, 4, 4, 3.615)
        x = inputs.jitter(x, 0.15, 3)
        pot, bonds = lj_cu(), None
    elif kind == "sc":
        x, H = inputs.fcc(5, 5, 5, 3.615)
        x = inputs.jitter(x, 0.15, 4)
        pot, bonds = sc_cu(), None
    else:
        x, H, bonds = inputs.kg_melt(8, 20, 0.85, seed=5, pushoff_iters=200)
        pot = oracle.pot_kg()
    f, W, e = oracle.forces(pot, x, H, bonds=bonds)
    assert np.abs(f.sum(0)).max() < 1e-12 * np.abs(f).sum()
    # f_i = -dE/dx_i by central differences
    h = 1e-5 if kind != "kg" else 1e-6
    rng = np.random.default_rng(6)
    for i in rng.choice(len(x), 6, replace=False):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            fd = -(oracle.forces(pot, xp, H, bonds=bonds)[2] - oracle.forces(pot, xm, H, bonds=bonds)[2]) / (2 * h)
            assert abs(fd - f[i, a]) <= 2e-6 * max(1.0, np.abs(f).max())


@pytest.mark.parametrize("kind", ["lj", "sc", "kg"])
def test_virial_matches_strain_derivative(kind):
    # 0 K: V sigma_ab = dE/d eps_ab under x -> (I+eps) x, H -> (I+eps) H with
    # symmetric eps; with sigma = -W/V this is dE/dh = -W_ab.
    if kind == "lj":
        x, H = inputs.fcc(4, 4, 4, 3.615)
        x = inputs.jitter(x, 0.1, 7)
        pot, bonds = lj_cu(), None
    elif kind == "sc":
        x, H = inputs.fcc(5, 5, 5, 3.615)
        x = inputs.jitter(x, 0.1, 8)
        pot, bonds = sc_cu(), None
    else:
        x, H, bonds = inputs.kg_melt(8, 20, 0.85, seed=9, pushoff_iters=200)
        pot = oracle.pot_kg()
    f, W, e = oracle.forces(pot, x, H, bonds=bonds)
    h = 1e-6
    for a, b in [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]:
        E = np.zeros((3, 3))
        if a == b:
            E[a, a] = 1.0
        else:
            E[a, b] = E[b, a] = 0.5
        Mp, Mm = np.eye(3) + h * E, np.eye(3) - h * E
        ep = oracle.forces(pot, x @ Mp.T, Mp @ H, bonds=bonds)[2]
        em = oracle.forces(pot, x @ Mm.T, Mm @ H, bonds=bonds)[2]
        fd = (ep - em) / (2 * h)
        assert abs(fd + W[a, b]) <= 1e-6 * max(1.0, np.abs(W).max())


def _fcc_lattice_sums(a, rc, fn):
    # enumerate FCC lattice vectors n1 a1 + n2 a2 + n3 a3 (primitive vectors) in FP64
    a1, a2, a3 = np.array([0, 0.5, 0.5]) * a, np.array([0.5, 0, 0.5]) * a, np.array([0.5, 0.5, 0]) * a
    K = int(np.ceil(2 * rc / a)) + 2
    rs = []
    for n1, n2, n3 in itertools.product(range(-K, K + 1), repeat=3):
        if n1 == n2 == n3 == 0:
            continue
        r = np.linalg.norm(n1 * a1 + n2 * a2 + n3 * a3)
        if r < rc:
            rs.append(r)
    rs = np.array(rs)
    return fn(rs)


def test_lj_fcc_lattice_energy_closed_form():
    a = 3.615
    eps, sig, rc = LJ_CU["eps"], LJ_CU["sigma"], LJ_CU["rc"]
    ref = _fcc_lattice_sums(a, rc, lambda r: 0.5 * np.sum(4 * eps * ((sig / r) ** 12 - (sig / r) ** 6)))
    x, H = inputs.fcc(4, 4, 4, a)
    f, W, e = oracle.forces(lj_cu(), x, H, use_cells=False)
    assert abs(e / len(x) - ref) <= 1e-12 * abs(ref)
    assert np.abs(f).max() < 1e-12
    # shells counted: 12, 6, 24, 12 inside rc (the 5th shell at a sqrt(5/2) is just outside)
    cnt = _fcc_lattice_sums(a, rc, lambda r: len(r))
    assert cnt == 12 + 6 + 24 + 12


def test_sc_fcc_lattice_energy_closed_form():
    a = 3.615
    p = SC_CU

    def e_of(r):
        return p["eps"] * (0.5 * np.sum((p["a"] / r) ** p["n"]) - p["c"] * np.sqrt(np.sum((p["a"] / r) ** p["m"])))

    ref = _fcc_lattice_sums(a, p["rc"], e_of)
    x, H = inputs.fcc(5, 5, 5, a)
    f, W, e = oracle.forces(sc_cu(), x, H, use_cells=True)
    assert abs(e / len(x) - ref) <= 1e-12 * abs(ref)
    assert np.abs(f).max() < 1e-12


def test_sc_shell_exactly_at_cutoff_is_excluded():
    # When the lattice parameter equals the potential's a and rc = 2a, the 8th FCC
    # shell (6 atoms at distance 2a) lies exactly at the cutoff.  With binary-exact
    # numbers (a = 4) the squared distance is exactly rc^2, and the strict r < rc
    # test must leave that shell out.
    a = 4.0
    pot = oracle.pot_sc(SC_CU["eps"], a, 2 * a, SC_CU["n"], SC_CU["m"], SC_CU["c"])
    x, H = inputs.fcc(5, 5, 5, a)
    for cells in (False, True):
        f, W, e = oracle.forces(pot, x, H, use_cells=cells)

        def e_of(r):
            r = r[r < 2 * a * (1 - 1e-12)]
            return SC_CU["eps"] * (0.5 * np.sum((a / r) ** 9) - SC_CU["c"] * np.sqrt(np.sum((a / r) ** 6)))

        ref = _fcc_lattice_sums(a, 2 * a * (1 + 1e-9), e_of)
        assert abs(e / len(x) - ref) <= 1e-12 * abs(ref)
        n_in = len(oracle.neighbor_pairs(x, H, 2 * a, use_cells=cells)) // len(x)
        assert n_in == 12 + 6 + 24 + 12 + 24 + 8 + 48  # shells 1..7; the 8th (6 atoms) is out


@pytest.mark.parametrize("kind", ["lj", "sc"])
@pytest.mark.parametrize("case", ["B(t)", "B(c)", "C(t)", "C(c)"])
def test_frame_indifference_table1(kind, case):
    # Sec. 2.1 / Table 1 analogue: the stress of the general box F H0 (positions
    # F H0 S) equals Q sigma(R H0) Q^T, where the MD sees only the triangular box.
    import json
    import os
    F = np.array(json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1.json")))
                 ["cases"][case]["F"])
    nc = 4 if kind == "lj" else 6
    x0, H0 = inputs.fcc(nc, nc, nc, 3.615)
    pot = lj_cu() if kind == "lj" else sc_cu()
    Q, R = oracle.qr(F)
    zero_v = np.zeros_like(x0)
    # route 1: general (non-triangular) box, brute force
    xg, Hg = x0 @ F.T, F @ H0
    _, Wg, _ = oracle.forces(pot, xg, Hg, use_cells=False)
    sg = oracle.stress_inst(0, 63.546, zero_v, Wg, Hg)
    # route 2: triangular MD box R H0, then rotate back
    xm, Hm = x0 @ R.T, R @ H0
    _, Wm, _ = oracle.forces(pot, xm, Hm, use_cells=True)
    sm = oracle.stress_inst(0, 63.546, zero_v, Wm, Hm)
    s_fem, _ = oracle.rotate_pk1(Q, F, sm)
    assert np.abs(s_fem - sg).max() <= 1e-10 * np.abs(sg).max()


def test_kg_bond_terms_and_errors():
    # a single bonded dimer far from everything else: FENE + WCA energy by hand
    H = np.diag([10.0, 10.0, 10.0])
    x = np.array([[1.0, 1.0, 1.0], [1.95, 1.0, 1.0]])
    bonds = np.array([[0, 1]])
    pot = oracle.pot_kg()
    f, W, e = oracle.forces(pot, x, H, bonds=bonds)
    r = 0.95
    ref = -0.5 * 30 * 1.5 ** 2 * np.log(1 - (r / 1.5) ** 2) + 4 * (r ** -12 - r ** -6) + 1.0
    assert abs(e - ref) < 1e-12
    # bonded pairs are excluded from the non-bonded LJ: the same dimer unbonded is LJ only
    f2, W2, e2 = oracle.forces(pot, x, H, bonds=np.zeros((0, 2), np.int32))
    assert abs(e2 - 4 * (r ** -12 - r ** -6)) < 1e-12
    # bond across the periodic boundary uses the minimum image
    xb = np.array([[0.2, 5.0, 5.0], [9.4, 5.0, 5.0]])
    _, _, eb = oracle.forces(pot, xb, H, bonds=bonds)
    r = 0.8
    assert abs(eb - (-0.5 * 30 * 2.25 * np.log(1 - r * r / 2.25) + 4 * (r ** -12 - r ** -6) + 1.0)) < 1e-10
    # overstretched bond (r >= R0): reported as an error
    xs = np.array([[1.0, 1.0, 1.0], [2.6, 1.0, 1.0]])
    with pytest.raises(oracle.OracleError) as ei:
        oracle.forces(pot, xs, H, bonds=bonds)
    assert ei.value.code == oracle.OR_EBOND
