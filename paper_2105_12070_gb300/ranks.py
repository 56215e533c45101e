"""Multi-rank helpers (one process per GPU, torch.distributed).

Cells are independent (Sec. 2.2), so the forward solve shards with no data exchange: a rank
integrates its own cells, in equal-count blocks (shard_range) or in blocks of equal predicted
cost (shard_by_cost, the GPU counterpart of the paper's dynamic load balancing).  The only exchanges are host-side bookkeeping (the slowest rank's time)
and, for the adjoint, the sum over ranks of the per-mechanism ln A gradients.
"""
from __future__ import annotations


def shard_range(ncells: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block of cells [first, last) of `rank` when ncells are split over `world`
    ranks as evenly as possible (the first ncells % world ranks get one more)."""
    if world < 1 or not (0 <= rank < world) or ncells < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(ncells, world)
    first = rank * base + min(rank, extra)
    return first, first + base + (1 if rank < extra else 0)


def shard_by_cost(cost, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block of cells [first, last) of `rank` such that the ranks' summed cost is as
    even as contiguous blocks allow: boundary k is the first cell at which the running cost
    reaches k/world of the total, so every rank's load is at most total/world plus the cost of one
    cell.  This is the load balancing of Sec. 2.2 (DLBFoam redistributes cells by the chemistry
    time each took in the previous flow step) for one process per GPU.  The natural cost is the
    step attempts of each cell in the previous call (chem_last_cell_counters: steps + rejects).
    With no cost at all the split is shard_range's."""
    import numpy as np
    c = np.asarray(cost, dtype=np.float64).ravel()
    if world < 1 or not (0 <= rank < world) or np.any(c < 0) or not np.all(np.isfinite(c)):
        raise ValueError("bad shard arguments")
    n = c.shape[0]
    total = float(c.sum())
    if total <= 0.0:
        return shard_range(n, rank, world)
    prefix = np.concatenate([[0.0], np.cumsum(c)])

    def boundary(k):
        if k <= 0:
            return 0
        if k >= world:
            return n
        return int(np.searchsorted(prefix, k * total / world, side="left"))

    return boundary(rank), boundary(rank + 1)


def max_over_ranks(values, device=None):
    """Element-wise max of a list of floats over all ranks (identity on one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def sum_lnA_grad(g_lnA):
    """In place: g_lnA (R,) summed over ranks, each rank holding the gradient of its own cells
    (the adjoint's one exchange step).  Identity on one process."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(g_lnA, op=dist.ReduceOp.SUM)
    return g_lnA
