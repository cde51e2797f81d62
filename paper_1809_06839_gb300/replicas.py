"""Host-side logic of running the augmentation path on several GPUs.

Images are independent, so the path has no exchange step: several GPUs run
independent replicas (one process per GPU), each on its own share of a
ragged batch.  This module holds the two pieces of host logic that involves:
the partition of a ragged batch into contiguous per-rank slices of about
equal pixel count, and the max-over-ranks reduction of a timing.  Neither
touches pixel data; no collective is on the data path.
"""
from __future__ import annotations

from typing import Sequence, Tuple

import torch


def shard_by_pixels(sizes: Sequence[Tuple[int, int]], world: int, rank: int) -> Tuple[int, int]:
    """Contiguous slice [start, end) of the batch for `rank` out of `world`:
    slice boundaries are placed where the running pixel count first reaches
    k/world of the total, so every rank's pixel load is within one image of
    the mean.  Empty slices are possible when there are fewer images than
    ranks."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    n = len(sizes)
    total = sum(int(h) * int(w) for h, w in sizes)

    def boundary(k: int) -> int:
        # first index whose prefix pixel count reaches k * total / world (exact integers)
        if k <= 0:
            return 0
        if k >= world:
            return n
        acc = 0
        for i, (h, w) in enumerate(sizes):
            if acc * world >= k * total:
                return i
            acc += int(h) * int(w)
        return n

    return boundary(rank), boundary(rank + 1)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over all ranks (the slowest rank's time); `value`
    itself without a process group."""
    if dist is None:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
