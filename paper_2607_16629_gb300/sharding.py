"""Channel sharding across ranks (one process per GPU).

Channels are independent decompositions, so N ranks split them with no
exchange on the data path (weak scaling: every rank keeps the same number
of channels).  The only collective is the timing reduction: the slowest
rank's time is the job's time."""
from __future__ import annotations

from typing import List


def channels_for_rank(per_rank: int, world: int, rank: int) -> List[int]:
    """Global channel ids owned by `rank` when each of `world` ranks takes
    `per_rank` consecutive channels."""
    if per_rank < 1 or world < 1 or not 0 <= rank < world:
        raise ValueError("bad sharding arguments")
    return list(range(rank * per_rank, (rank + 1) * per_rank))


def max_over_ranks(value: float, device=None) -> float:
    """Largest `value` over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
