"""Host-side sharding of independent tiles across ranks (one GPU per rank).

Tiles are independent reconstructions (the paper processes 4K x 4K tiles of a
slide concurrently, Sec. V, and hands them to workers on demand, Sec. IV), so
a multi-GPU run needs no collective on the data path: each rank takes a share
of the tiles. Shares are balanced by longest-processing-time-first on a cost
per tile (predicted by the cost model, or the pixel count).
"""
from __future__ import annotations

import heapq
from typing import List, Sequence


def lpt_shards(costs: Sequence[float], world: int) -> List[List[int]]:
    """Assigns tile indices to `world` shards, most expensive first, each to the
    currently lightest shard (ties: lowest rank). Deterministic."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    shards: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return shards


def my_tiles(costs: Sequence[float], rank: int, world: int) -> List[int]:
    return lpt_shards(costs, world)[rank]
