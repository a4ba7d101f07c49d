"""Partition independent frames across ranks (one process per GPU).

FNR frames are independent problems, so multi-GPU runs split the frames and
exchange nothing on the data path. ``shard`` balances by pixel count with
the longest-first greedy rule (each frame, largest first, goes to the rank
with the least work so far; ties to the lower rank), which is deterministic,
so every rank computes the same assignment without communicating.
"""
from __future__ import annotations

from typing import List, Sequence


def assignment(work: Sequence[int], world: int) -> List[int]:
    """Rank of every item (same length as ``work``)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(work)), key=lambda i: (-int(work[i]), i))
    load = [0] * world
    owner = [0] * len(work)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += int(work[i])
    return owner


def shard(work: Sequence[int], world: int, rank: int) -> List[int]:
    """Indices of the items owned by ``rank``, in ascending order."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return [i for i, r in enumerate(assignment(work, world)) if r == rank]
