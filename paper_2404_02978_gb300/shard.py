"""Realisation sharding across ranks (one process per GPU, weak scaling).

Realisation r of Eq. 3 draws its terms from stream points (r N_f + k) of one
continuing sequence (Sec. 3.2), so a rank that synthesises realisations
[offset, offset + count) through `real_offset` produces exactly the values a
single process would produce for them: the ranks need no exchange on the data
path.  The only collective is the reduction of the step time (max over ranks).
"""
from __future__ import annotations


def realisation_slice(rank: int, world: int, per_rank: int, base: int = 0) -> tuple[int, int]:
    """(real_offset, count) of `rank` when each of `world` ranks takes `per_rank`
    consecutive realisations starting at `base`."""
    if world < 1 or not 0 <= rank < world or per_rank < 0 or base < 0:
        raise ValueError("need 0 <= rank < world, per_rank >= 0, base >= 0")
    return base + rank * per_rank, per_rank


def max_over_ranks(value: float, world: int, device="cpu") -> float:
    """The largest `value` over all ranks (the whole job's time); identity at world 1."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
