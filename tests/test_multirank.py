"""Multi-rank host logic on CPU (gloo, world size 2): the cell partition, the
stress gather, the max-over-ranks timing reduction, and the sharded FE load
increment (each rank runs its own cells, the stresses are all-gathered, every
rank advances the same FE mesh)."""
import os
import socket

import numpy as np
import pytest

from paper_1902_09171_gb300 import dist as rdist


def test_shard_by_atoms_balanced_and_complete():
    rng = np.random.default_rng(0)
    n = rng.integers(5000, 20001, size=64) // 50 * 50
    for world in (1, 2, 3, 4, 8):
        b = rdist.shard_by_atoms(n, world)
        assert b[0][0] == 0 and b[-1][1] == 64
        assert all(b[k][1] == b[k + 1][0] for k in range(world - 1))
        loads = [int(n[a:c].sum()) for a, c in b]
        assert max(loads) - min(loads) <= 2 * int(n.max())
    assert rdist.shard_by_atoms([10, 10], 4)[-1] == (2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = [4000] * 5 + [8000] * 3
        bounds = rdist.shard_by_atoms(n, world)
        a, b = bounds[rank]
        local = torch.arange(a, b, dtype=torch.float64).repeat(6, 1).T.contiguous() * 10 + rank
        full = rdist.gather_cells(local, bounds)
        t = rdist.max_over_ranks(1.0 + rank)
        out.put((rank, full.numpy().tolist(), t, bounds))
    finally:
        dist.destroy_process_group()


def test_two_rank_gather_and_timing():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, full, t, bounds in res:
        full = np.array(full)
        assert full.shape == (8, 6)
        owner = [0 if c < bounds[0][1] else 1 for c in range(8)]
        assert np.array_equal(full[:, 0], np.arange(8) * 10 + np.array(owner))
        assert t == 2.0


class _OracleFE:
    """The oracle's FP64 hex-8 FE (test side) behind the fe interface of fe_step_sharded."""

    def __init__(self, *args):
        import oracle
        self.m = oracle.FEMesh(*args)

    def apply_bc(self, lam):
        self.m.apply_bc(lam)

    def F(self):
        import torch
        return torch.tensor(self.m.F())

    def update(self, P):
        self.m.update(P.numpy())


def _bar_args():
    from paper_1902_09171_gb300 import inputs
    X, conn = inputs.hex_mesh(6, 2, 1, 6.0, 2.0, 1.0)
    X[7] += [0.05, -0.03, 0.0]  # an interior node off the grid: elements differ
    mask, val = inputs.uniaxial_bc(X, 6.0)
    return X, conn, mask, val, 1.3, 0.05, 0.7, 0.4


def _stub_cells(F):
    """Stand-in for the r-cells: a linear elastic P(F) per cell, evaluated only from
    this rank's F (the engine sees nothing but its own cells)."""
    import torch
    E = F - torch.eye(3, dtype=F.dtype)
    eps = 0.5 * (E + E.transpose(1, 2))
    tr = eps.diagonal(dim1=1, dim2=2).sum(-1)
    return 2.0 * eps + 0.7 * tr[:, None, None] * torch.eye(3, dtype=F.dtype) + 0.1 * E


def _sharded_history(world, rank, n_inc=5):
    X, conn, mask, val, *rest = _bar_args()
    fe = _OracleFE(X, conn, mask, val, *rest)
    bounds = rdist.shard_by_atoms(np.arange(1, len(conn) + 1) * 100, world)
    hist = []
    for k in range(n_inc):
        rdist.fe_step_sharded(fe, _stub_cells, 0.01 * (k + 1), bounds, rank)
        hist.append(fe.m.d.copy())
    return np.array(hist), bounds


def _fe_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        hist, bounds = _sharded_history(world, rank)
        out.put((rank, hist.tolist(), bounds))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharded_fe_step_equals_one_rank():
    torch = pytest.importorskip("torch")
    ref, _ = _sharded_history(1, 0)
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_fe_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, hist, bounds in res:
        assert bounds[0][1] > 0 and bounds[1][0] == bounds[0][1] and bounds[1][1] == 12  # both ranks own cells
        assert np.array_equal(np.array(hist), ref), rank  # bit for bit
    assert np.abs(ref[-1]).max() > 0
