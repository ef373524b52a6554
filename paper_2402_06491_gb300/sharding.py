"""Host-side sharding of a point solve and of the PDD subdomains over ranks (one process per GPU).

Points are independent problems (Sec. 3: the probabilistic part splits into
independent sets of points), so rank r solves a contiguous slice of them with
point_base equal to the slice's first global index.  Every point keeps its own
random stream, so the union of the slices reproduces the single-rank solve
exactly and no data-path collective is needed.

For the PDD, every rank needs all interface values (one all-gather of the
nodal values, the single exchange of the method) and then solves its own
contiguous range of the decoupled subdomains (grt_pdd_solve_range).
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


def pdd_subdomain_range(grid: dict, world: int, rank: int) -> tuple:
    """[begin, end) of the row-major subdomains of a PDD grid owned by `rank` (balanced, contiguous)."""
    nsub = 1
    for a in range(int(grid["dim"])):
        nsub *= int(grid["sub"][a])
    return shard_range(nsub, world, rank)
