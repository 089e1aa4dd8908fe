"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds input GENERATORS only -- lattices, velocities, melts, meshes,
deformation paths -- and none of the method's arithmetic (no forces, no
integrator, no QR, no stress).  Both the CUDA path and the FP64 oracle are fed
from here, so neither depends on the other.

Workload recipes (the paper's own data are not available; these stand in):
  * Cu-like FCC crystals (Sec. 3.1 uses a 10x10x10 FCC Cu cell, 4000 atoms,
    edge 36.15 A): ``fcc(nx, ny, nz, a)`` with a = 3.615 A.
  * Kremer-Grest melts (Sec. 3.2: linear bead-spring chains at melt density):
    ``kg_melt(n_chains, chain_len, density, seed)`` -- seeded random walks with
    bond length 0.97 sigma, then a displacement-capped soft push-off.
  * Maxwell velocities with zero centre-of-mass momentum.
"""
from __future__ import annotations

import numpy as np

# CODATA 2018 exact / recommended values, used only to turn kT/m into a
# velocity scale in metal units (Angstrom/ps).
_EV = 1.602176634e-19
_AMU = 1.66053906660e-27
KB_EV = 8.617333262e-5  # Boltzmann constant, eV/K


def vel_unit_sq(units: int) -> float:
    """(energy / mass) expressed in (velocity unit)^2: metal eV/amu -> (A/ps)^2."""
    return _EV / _AMU / 1e4 if units == 0 else 1.0


def fcc(nx: int, ny: int, nz: int, a: float):
    """FCC lattice of nx*ny*nz conventional cells; returns x (4 nx ny nz, 3) and H0 = diag(L)."""
    base = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 1, 3)
    x = ((g + base[None]) * a).reshape(-1, 3)
    H0 = np.diag([nx * a, ny * a, nz * a]).astype(np.float64)
    return np.ascontiguousarray(x), H0


def maxwell(n: int, mass: float, kT: float, units: int, seed: int):
    """Seeded Maxwell-Boltzmann velocities at temperature kT with zero total momentum."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 3)) * np.sqrt(kT * vel_unit_sq(units) / mass)
    v -= v.mean(axis=0, keepdims=True)
    return v


def jitter(x: np.ndarray, amp: float, seed: int):
    """Uniform random displacement of every coordinate in [-amp, amp]."""
    rng = np.random.default_rng(seed)
    return x + rng.uniform(-amp, amp, size=x.shape)


def to_f32(a: np.ndarray) -> np.ndarray:
    """Round to the FP32 grid (what the GPU stores), returned as float64."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def hex_mesh(nx: int, ny: int, nz: int, Lx: float, Ly: float, Lz: float):
    """Structured 8-node hex mesh of a box [0,Lx]x[0,Ly]x[0,Lz]; node order per element
    (-,-,-) (+,-,-) (+,+,-) (-,+,-) (-,-,+) (+,-,+) (+,+,+) (-,+,+)."""
    xs, ys, zs = np.linspace(0, Lx, nx + 1), np.linspace(0, Ly, ny + 1), np.linspace(0, Lz, nz + 1)
    X = np.stack(np.meshgrid(xs, ys, zs, indexing="ij"), -1).reshape(-1, 3)

    def nid(i, j, k):
        return (i * (ny + 1) + j) * (nz + 1) + k

    conn = []
    for i in range(nx):
        for j in range(ny):
            for k in range(nz):
                conn.append([nid(i, j, k), nid(i + 1, j, k), nid(i + 1, j + 1, k), nid(i, j + 1, k),
                             nid(i, j, k + 1), nid(i + 1, j, k + 1), nid(i + 1, j + 1, k + 1),
                             nid(i, j + 1, k + 1)])
    return np.ascontiguousarray(X), np.asarray(conn, dtype=np.int32)


def tet_mesh(nx: int, ny: int, nz: int, Lx: float, Ly: float, Lz: float):
    """The structured hex mesh of hex_mesh split into 4-node tetrahedra: six per
    hexahedron around its (-,-,-)-(+,+,+) diagonal, the same diagonal direction
    in every hexahedron so that neighbouring faces match; every tetrahedron has
    positive orientation.  Returns X (nn, 3) and conn (6 nx ny nz, 4)."""
    X, hexes = hex_mesh(nx, ny, nz, Lx, Ly, Lz)
    split = [(0, 1, 2, 6), (0, 2, 3, 6), (0, 3, 7, 6), (0, 7, 4, 6), (0, 4, 5, 6), (0, 5, 1, 6)]
    conn = []
    for h in hexes:
        for t in split:
            q = [int(h[a]) for a in t]
            e1, e2, e3 = X[q[1]] - X[q[0]], X[q[2]] - X[q[0]], X[q[3]] - X[q[0]]
            if np.dot(np.cross(e1, e2), e3) < 0:
                q[1], q[2] = q[2], q[1]
            conn.append(q)
    return X, np.asarray(conn, dtype=np.int32)


def necking_mesh(nx: int, ny: int, nz: int, h: float, imperfection: float = 0.05):
    """Hex-8 bar of nx x ny x nz cubic elements of edge h along x, with a cross-section
    imperfection at mid-length: the nodes of the plane x = (nx // 2) h are moved
    towards the bar axis by the factor sqrt(1 - imperfection) in y and z, so that
    the section there has (1 - imperfection) of the nominal area.  Returns X, conn."""
    X, conn = hex_mesh(nx, ny, nz, nx * h, ny * h, nz * h)
    mid = np.abs(X[:, 0] - (nx // 2) * h) < 1e-9 * h
    c = np.array([0.5 * ny * h, 0.5 * nz * h])
    X[mid, 1:] = c + np.sqrt(1.0 - imperfection) * (X[mid, 1:] - c)
    return X, conn


def uniaxial_bc(X: np.ndarray, L: float, all_nodes: bool = False):
    """Boundary conditions for uniaxial extension along x (load factor = engineering strain).

    all_nodes=True prescribes u = (lambda X_x, 0, 0) on every node (a single-element
    uniaxial-strain test).  Otherwise: x=0 face u_x = 0, x=L face u_x = lambda L,
    the node at the origin fully pinned, and the origin's x-edge neighbour on the
    x=L face pinned in y and z (rigid-body modes); lateral faces free.
    Returns (mask, val), each (nn, 3); prescribed d = lambda * val.
    """
    nn = X.shape[0]
    mask = np.zeros((nn, 3), dtype=np.int32)
    val = np.zeros((nn, 3))
    if all_nodes:
        mask[:] = 1
        val[:, 0] = X[:, 0]
        return mask, val
    tol = 1e-9 * max(L, 1.0)
    x0 = np.abs(X[:, 0]) < tol
    xL = np.abs(X[:, 0] - L) < tol
    mask[x0, 0] = 1
    mask[xL, 0] = 1
    val[xL, 0] = L
    origin = np.where(x0 & (np.abs(X[:, 1]) < tol) & (np.abs(X[:, 2]) < tol))[0]
    mask[origin, :] = 1
    far = np.where(xL & (np.abs(X[:, 1]) < tol) & (np.abs(X[:, 2]) < tol))[0]
    mask[far, 1] = 1
    mask[far, 2] = 1
    return mask, val


def uniform_sizes(n_cells: int, lo: int, hi: int, multiple: int, seed: int):
    """Uneven r-cell sizes: U[lo, hi] rounded down to a multiple of `multiple`."""
    rng = np.random.default_rng(seed)
    s = rng.integers(lo, hi + 1, size=n_cells)
    return (s // multiple) * multiple


def kg_melt(n_chains: int, chain_len: int, density: float, seed: int, bond: float = 0.97,
            pushoff_iters: int = 300):
    """Kremer-Grest style melt: seeded random-walk chains in a cubic box at the given
    number density, followed by a displacement-capped push-off of overlapping
    non-bonded beads (soft harmonic repulsion inside 1 sigma) that keeps bond
    lengths near `bond`.  Returns x (N,3), H0, bonds (n_bonds, 2) int32.

    This is input preparation, not the method: its only purpose is a start state
    without overlaps, from which both the CUDA path and the oracle equilibrate.
    """
    rng = np.random.default_rng(seed)
    n = n_chains * chain_len
    L = (n / density) ** (1.0 / 3.0)
    x = np.zeros((n, 3))
    for c in range(n_chains):
        p = rng.uniform(0, L, 3)
        base = c * chain_len
        x[base] = p
        for k in range(1, chain_len):
            while True:
                u = rng.standard_normal(3)
                u /= np.linalg.norm(u)
                q = x[base + k - 1] + bond * u
                if k < 2 or np.linalg.norm(q - x[base + k - 2]) > 1.02:
                    break
            x[base + k] = q
    bonds = np.array([[c * chain_len + k, c * chain_len + k + 1]
                      for c in range(n_chains) for k in range(chain_len - 1)], dtype=np.int32)
    x = _pushoff(x, L, bonds, chain_len, pushoff_iters)
    return np.ascontiguousarray(x), np.diag([L, L, L]), bonds


def _pushoff(x, L, bonds, chain_len, iters, rcut=0.95, cap=0.05):
    """Capped gradient steps on sum over non-bonded pairs of (rcut - r)^2 (r < rcut) plus
    (r - bond)^2 springs on bonds; the close pairs come from a periodic k-d tree."""
    from scipy.spatial import cKDTree

    n = x.shape[0]
    bi, bj = bonds[:, 0], bonds[:, 1]
    for _ in range(iters):
        x = np.mod(x, L)
        x[x >= L] -= L  # np.mod can round up to L
        pairs = cKDTree(x, boxsize=L).query_pairs(rcut, output_type="ndarray")
        disp = np.zeros_like(x)
        worst = 0.0
        if len(pairs):
            ii, jj = pairs[:, 0], pairs[:, 1]
            adjacent = (ii // chain_len == jj // chain_len) & (np.abs(ii - jj) == 1)
            ii, jj = ii[~adjacent], jj[~adjacent]
            d = x[ii] - x[jj]
            d -= L * np.round(d / L)
            r = np.linalg.norm(d, axis=1)
            m = (r < rcut) & (r > 1e-12)
            if np.any(m):
                worst = float((rcut - r[m]).max())
                push = (0.5 * (rcut - r[m]) / r[m])[:, None] * d[m]
                np.add.at(disp, ii[m], push)
                np.add.at(disp, jj[m], -push)
        d = x[bj] - x[bi]
        d -= L * np.round(d / L)
        r = np.linalg.norm(d, axis=1)
        corr = (0.5 * (r - 0.97) / np.maximum(r, 1e-12))[:, None] * d
        np.add.at(disp, bi, corr)
        np.add.at(disp, bj, -corr)
        nrm = np.linalg.norm(disp, axis=1, keepdims=True)
        disp *= np.minimum(1.0, cap / np.maximum(nrm, 1e-300))
        x = x + disp
        if worst < 0.12:
            break
    return np.mod(x, L)


def strain_paths(n_paths: int, n_inc: int, seed: int, max_strain: float = 0.3, max_shear: float = 0.08,
                 jitter: float = 0.01, max_lateral: float = 0.1):
    """Seeded deformation-gradient histories F[p, t] (t = 0..n_inc, F[:, 0] = I).

    Axial stretch along x: a monotone ramp to an amplitude drawn from
    [-max_strain / 2, max_strain], or one to three sine cycles of that amplitude
    growing as sqrt(t), which swing to minus the amplitude as well (so cyclic
    paths reach max_strain in compression too).  Each lateral stretch (y, z) is
    -nu * eps_x (nu in [0, 0.5]) plus its own drift that saturates on a random
    time scale (from a few increments to the whole path), between -max_lateral
    and +max_lateral / 4 -- so paths include lateral contraction at zero axial
    load, as a free surface under residual tension produces.  A monotone simple
    shear F_xy up to max_shear and a small random ramp (amplitude `jitter`) in
    all nine components complete the path.  Returns (n_paths, n_inc + 1, 3, 3)."""
    rng = np.random.default_rng(seed)
    t = np.arange(n_inc + 1) / n_inc
    F = np.tile(np.eye(3), (n_paths, n_inc + 1, 1, 1))
    for p in range(n_paths):
        amp = rng.uniform(-0.5 * max_strain, max_strain)
        if rng.uniform() < 0.5:
            ex = amp * t
        else:
            cycles = rng.integers(1, 4)
            ex = amp * np.sin(np.pi * cycles * t) * t ** 0.5
        nu = rng.uniform(0.0, 0.5)
        gam = rng.uniform(-max_shear, max_shear) * t
        F[p, :, 0, 0] = 1.0 + ex
        for d in (1, 2):
            drift = rng.uniform(-max_lateral, 0.25 * max_lateral)
            tau = np.exp(rng.uniform(np.log(2.0 / n_inc), 0.0))
            F[p, :, d, d] = 1.0 - nu * ex + drift * (1.0 - np.exp(-t / tau)) / (1.0 - np.exp(-1.0 / tau))
        F[p, :, 0, 1] = gam
        F[p] += jitter * rng.uniform(-1, 1, (3, 3))[None] * t[:, None, None]
    return F


def bar_strain_paths(n_paths: int, n_inc: int, seed: int, max_axial: float = 0.15, max_shear: float = 0.12,
                     max_lateral: float = 0.05, jitter: float = 0.005):
    """Seeded deformation-gradient histories F[p, t] (t = 0..n_inc, F[:, 0] = I) of the
    kind the elements of a bar in uniaxial tension go through: a monotone axial
    stretch to an amplitude in [-max_axial / 5, max_axial] along a ramp t^q
    (q in [0.5, 2]); lateral stretches -nu eps_x (nu in [0, 0.5]) plus their own
    drift in [-max_lateral, max_lateral / 2] that saturates on a random time scale
    (a few increments to the whole path: a thermal expansion that settles while the
    Poisson contraction grows makes a lateral path that turns back); the four
    shears F_xy, F_xz, F_yx, F_zx
    each ramped to an amplitude in [-max_shear, max_shear]; a random ramp of
    amplitude `jitter` in all nine components.  Returns (n_paths, n_inc + 1, 3, 3)."""
    rng = np.random.default_rng(seed)
    t = np.arange(n_inc + 1) / n_inc
    F = np.tile(np.eye(3), (n_paths, n_inc + 1, 1, 1))
    for p in range(n_paths):
        ex = rng.uniform(-0.2 * max_axial, max_axial) * t ** rng.uniform(0.5, 2.0)
        nu = rng.uniform(0.0, 0.5)
        F[p, :, 0, 0] = 1.0 + ex
        for d in (1, 2):
            drift = rng.uniform(-max_lateral, 0.5 * max_lateral)
            tau = np.exp(rng.uniform(np.log(2.0 / n_inc), 0.0))
            F[p, :, d, d] = 1.0 - nu * ex + drift * (1.0 - np.exp(-t / tau)) / (1.0 - np.exp(-1.0 / tau))
        for (i, j) in ((0, 1), (0, 2), (1, 0), (2, 0)):
            F[p, :, i, j] = rng.uniform(-max_shear, max_shear) * t ** rng.uniform(0.5, 2.0)
        F[p] += jitter * rng.uniform(-1, 1, (3, 3))[None] * t[:, None, None]
    return F


def kg_cells(n_cells: int, n_chains: int, chain_len: int, density: float, seed: int, n_distinct: int = 4,
             starmap=None):
    """n_cells Kremer-Grest r-cells built from n_distinct seeded melts, each copy
    shifted by a seeded random periodic translation (positions wrapped).  Returns
    a list of dicts (H0, x0, bonds).  starmap (e.g. a process pool's) generates
    the melts in parallel; the result does not depend on it."""
    rng = np.random.default_rng(seed)
    jobs = [(n_chains, chain_len, density, seed * 1000 + k) for k in range(n_distinct)]
    if starmap is None:
        melts = [kg_melt(*j) for j in jobs]
    else:
        melts = list(starmap(kg_melt, jobs))
    cells = []
    for c in range(n_cells):
        x, H, b = melts[c % n_distinct]
        L = H[0, 0]
        xs = np.mod(x + rng.uniform(0, L, 3), L)
        cells.append(dict(H0=H.copy(), x0=to_f32(xs), bonds=b))
    return cells
