"""Multi-GPU layout of the r-cell batch (one process per GPU).

The r-cells of a load step are independent at the MD level (Sec. 2.3: the
paper gives each r-cell its own communicator split), so the cells are split
into contiguous, atom-balanced shards, one per rank, with no collective on the
MD data path.  The only exchange is the FE-level one of Sec. 2.3 (scatter F,
gather the stress): each rank contributes the stresses of its own cells and
`gather_cells` assembles the full per-cell array on every rank.
"""
from __future__ import annotations

import numpy as np


def shard_by_atoms(n_atoms_per_cell, world: int):
    """Contiguous split of the cells into `world` shards with nearly equal atom
    counts (greedy prefix cut).  Returns a list of (first, last+1) per rank."""
    n = np.asarray(n_atoms_per_cell, dtype=np.int64)
    total = int(n.sum())
    cuts = [0]
    acc = 0
    r = 1
    for i, a in enumerate(n):
        acc += int(a)
        while r < world and acc >= r * total / world and len(cuts) == r:
            cuts.append(i + 1)
            r += 1
    while len(cuts) < world:
        cuts.append(len(n))
    cuts.append(len(n))
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def gather_cells(local, bounds, group=None):
    """All-gather per-cell rows (torch tensor, local cells x k) into the full array
    ordered by cell, on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    counts = [b - a for a, b in bounds]
    width = local.shape[1:]
    pad = max(counts)
    buf = torch.zeros((pad,) + tuple(width), dtype=local.dtype, device=local.device)
    buf[:local.shape[0]] = local
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([p[:c] for p, c in zip(parts, counts)], dim=0)


def max_over_ranks(value: float, group=None) -> float:
    """Largest value over all ranks (the timing rule: the slowest rank sets the time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def fe_step_sharded(fe, run_cells, lam: float, bounds, rank: int, group=None):
    """One FE load increment with the r-cells split over ranks: the FEM <-> r-cell
    scatter / gather of Sec. 2.3 in GPU form.  Every rank holds the whole (small)
    FE mesh and advances it identically; rank `rank` runs only its own cells
    bounds[rank] = (a, b):
      1. fe.apply_bc(lam); F = fe.F()          all elements, on every rank
      2. P_local = run_cells(F[a:b])           this rank's r-cells (QR, remap, MD, stress)
      3. P = all-gather of P_local             the only exchange: 9 doubles per cell
      4. fe.update(P)                          on every rank, from the same P
    fe: object with apply_bc(lam), F() -> tensor (ne, 3, 3) and update(P);
    run_cells(F_local) -> tensor (b - a, 3, 3).  Without an initialised process
    group (one rank) step 3 is the identity.  Returns the full P."""
    import torch.distributed as dist
    fe.apply_bc(lam)
    F = fe.F()
    a, b = bounds[rank]
    P_local = run_cells(F[a:b].contiguous())
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        P = gather_cells(P_local, bounds, group)
    else:
        P = P_local
    fe.update(P)
    return P
