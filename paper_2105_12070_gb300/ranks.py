"""Multi-rank helpers (one process per GPU, torch.distributed).

Cells are independent (Sec. 2.2), so the forward solve shards with no data exchange: a rank
integrates its own cells.  The only exchanges are host-side bookkeeping (the slowest rank's time)
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
