"""Sharding of a periodic lattice's Fourier blocks over ranks (one GPU each).

Thm. 3.3 makes the |L| Fourier blocks independent: rank r of W solves the
contiguous range of linear Fourier indices jbar returned by j_range (its own
per-axis factors are recomputed locally; they are small), the sorted parts
are gathered, and merge() reproduces the single-GPU ordering (ascending
value, ties by Fourier index).  The only exchange is the gather of the
eigenvalues (|L| m0 doubles and ints).
"""
from __future__ import annotations

import heapq

import numpy as np


def j_range(ncell, rank, world):
    """Contiguous [j0, j1) of rank `rank` among `world` (sizes differ by <= 1)."""
    base, extra = divmod(int(ncell), int(world))
    j0 = rank * base + min(rank, extra)
    return j0, j0 + base + (1 if rank < extra else 0)


def merge(parts):
    """Merge per-rank (evals, block_of) lists, each sorted by (value, block),
    into one ascending (value, block) order."""
    items = heapq.merge(*[zip(np.asarray(e).tolist(), np.asarray(b).tolist()) for e, b in parts])
    out = list(items)
    if not out:
        return np.zeros(0), np.zeros(0, np.int32)
    ev, blk = zip(*out)
    return np.asarray(ev, float), np.asarray(blk, np.int32)


def solve_sharded(solve_range, ncell, group=None):
    """solve_range(j0, j1) -> (evals, block_of) sorted for this rank's range;
    all_gather over `group` (torch.distributed) and merge.  Without an
    initialised process group, one rank solves everything."""
    import torch.distributed as dist
    if group is None and not (dist.is_available() and dist.is_initialized()):
        return merge([solve_range(0, ncell)])
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    j0, j1 = j_range(ncell, rank, world)
    mine = solve_range(j0, j1)
    parts = [None] * world
    dist.all_gather_object(parts, (np.asarray(mine[0]), np.asarray(mine[1])), group=group)
    return merge(parts)
