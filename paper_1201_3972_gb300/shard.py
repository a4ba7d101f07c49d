"""Partition independent frames across ranks (one process per GPU).

FNR frames are independent problems, so multi-GPU runs split the frames and
exchange nothing on the data path. ``shard`` balances by pixel count with
the longest-first greedy rule (each frame, largest first, goes to the rank
with the least work so far; ties to the lower rank), which is deterministic,
so every rank computes the same assignment without communicating.

A single frame too large for one device splits into row bands instead
(``row_bands``): a band of output rows [y0, y1) reads the input rows
[y0 - r, y1 + r) clipped to the frame, r = (k - 1) / 2, since every window of
its pixels lies there (Sec. 3.3: the k x k window S_xy). Filtering that
halo-extended sub-frame as a frame of its own gives exactly the whole-frame
result on the band's rows: a window only meets the sub-frame's top or bottom
edge where that edge is the frame's own, so the border rule acts on the same
rows. The halo rows of the sub-frame's output are discarded.
"""
from __future__ import annotations

from typing import List, NamedTuple, Sequence


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


class Band(NamedTuple):
    y0: int  # first output row of the band
    y1: int  # one past its last output row
    h0: int  # first input row it reads (y0 - r, clipped)
    h1: int  # one past the last input row it reads (y1 + r, clipped)


def row_bands(H: int, k: int, parts: int) -> List[Band]:
    """Split the H rows of a frame into ``parts`` contiguous bands whose heights
    differ by at most one (the first H mod parts bands take the extra row);
    bands of height 0 appear when parts > H. Each band carries its halo rows
    for a window of size k (odd, >= 3)."""
    if H < 1 or parts < 1:
        raise ValueError("H and parts must be >= 1")
    if k < 3 or k % 2 == 0:
        raise ValueError("k must be odd and >= 3")
    r = (k - 1) // 2
    base, extra = divmod(H, parts)
    bands = []
    y = 0
    for b in range(parts):
        h = base + (1 if b < extra else 0)
        y0, y1 = y, y + h
        bands.append(Band(y0, y1, max(0, y0 - r), min(H, y1 + r)) if h else Band(y0, y1, y0, y0))
        y = y1
    return bands
