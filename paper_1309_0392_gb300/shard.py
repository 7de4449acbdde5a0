"""Sharding a combination scheme over ranks (one GPU each).

The grids of a scheme are independent (Sec. 2: the coarse parallelism of the
combination technique), so ranks split them with no exchange until the
gather: every rank hierarchizes its own grids, gathers them into a partial
fp64 sparse vector (the coefficients of other ranks' grids set to 0), and one
sum all-reduce of the sparse vector completes the combination.  The way back
needs no exchange: every rank holds the whole sparse vector after the
all-reduce and scatters it onto its own grids (then dehierarchizes them).
On the GPU a rank's plan holds only its grids: Plan.scheme(d, n, owned=...).
"""
from __future__ import annotations

import heapq

import numpy as np


def partition_grids(points, world: int):
    """Greedy largest-first split of grids (by point count) over `world`
    ranks; returns a list of sorted grid-index lists, one per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0, r) for r in range(world)]
    owned = [[] for _ in range(world)]
    for g in sorted(range(len(points)), key=lambda i: (-int(points[i]), i)):
        load, r = heapq.heappop(heap)
        owned[r].append(g)
        heapq.heappush(heap, (load + int(points[g]), r))
    return [sorted(o) for o in owned]


def owned_coeffs(coeffs, owned):
    """Coefficient vector of one rank: its grids keep theirs, the rest get 0."""
    c = np.zeros(len(coeffs), dtype=np.float64)
    c[list(owned)] = np.asarray(coeffs, dtype=np.float64)[list(owned)]
    return c


def allreduce_sparse(partial, group=None):
    """Sum the ranks' partial sparse vectors in place (torch.distributed)."""
    import torch.distributed as dist
    dist.all_reduce(partial, op=dist.ReduceOp.SUM, group=group)
    return partial
