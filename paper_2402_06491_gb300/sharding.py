"""Host-side sharding of a point solve over ranks (one process per GPU).

Points are independent problems (Sec. 3: the probabilistic part splits into
independent sets of points), so rank r solves a contiguous slice of them with
point_base equal to the slice's first global index.  Every point keeps its own
random stream, so the union of the slices reproduces the single-rank solve
exactly and no data-path collective is needed.
"""
from __future__ import annotations


def shard_range(n: int, world: int, rank: int) -> tuple:
    """[start, stop) of the points owned by `rank` out of `world` (balanced, contiguous)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need world >= 1 and 0 <= rank < world")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    stop = start + base + (1 if rank < extra else 0)
    return start, stop
