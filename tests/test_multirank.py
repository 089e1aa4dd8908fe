"""Multi-rank host logic on CPU (gloo, world size 2): the cell partition, the
stress gather and the max-over-ranks timing reduction."""
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
