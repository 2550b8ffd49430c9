"""Query sharding over ranks (one process per GPU, graph replicated).

Walk queries are independent (FlowWalker Section 5), so N GPUs each take a
contiguous slice of the query range with the query ids of the full range in
the random-number counter: the union of the shards' paths is bit-identical to
one GPU running every query.  No data-path collective exists; the only
cross-rank operations are a start barrier and a max/sum of host scalars for
reporting, over whatever torch.distributed group the caller set up.
"""

from __future__ import annotations

import os
from typing import Tuple


def env_rank() -> Tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def shard_range(total: int, rank: int, world: int) -> Tuple[int, int]:
    """[begin, end) of the queries owned by `rank`: contiguous, sizes differ by
    at most one, the first total % world ranks one larger."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(total, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def reduce_scalar(value: float, op: str = "max", device="cpu") -> float:
    """max or sum of a host scalar over the default process group (identity
    without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())
