"""Slice sharding across ranks (one process per GPU).

Slices are independent problems (Sec. II.C.2), so N GPUs split a stack of
slices into contiguous shards and solve them with no data-path collective;
the only collectives are the timing barrier and a max-over-ranks reduction.
"""

from __future__ import annotations


def slice_shard(n_slices: int, rank: int, world: int) -> tuple[int, int]:
    """[start, stop) of rank's contiguous shard; sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or n_slices < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_slices, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Max of a float over all ranks of the default process group (value itself if none)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
