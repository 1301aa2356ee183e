"""Query sharding across ranks (one process per GPU).

Queries are independent, so a grid is split into contiguous z-slabs, one per
rank, with no data-path collective; every rank keeps a full copy of the
geometry.  With ``weak=True`` the global grid grows with the world size so
each rank keeps the single-GPU number of queries.
"""
from __future__ import annotations


def slab(dims, rank: int, world: int):
    """[k0, k1) range of the last grid axis owned by `rank`."""
    nz = int(dims[-1])
    base, extra = divmod(nz, world)
    k0 = rank * base + min(rank, extra)
    k1 = k0 + base + (1 if rank < extra else 0)
    return k0, k1


def shard_grid(lo, hi, dims, rank: int, world: int, weak: bool = True):
    """The sub-grid (lo, hi, dims) of `rank`.  Weak: the global grid has
    dims[-1] * world samples on the last axis, so every rank gets dims[-1]."""
    lo, hi, dims = list(lo), list(hi), list(dims)
    nz = dims[-1] * world if weak else dims[-1]
    if nz < world:
        raise ValueError("fewer grid planes than ranks")
    k0, k1 = slab(dims[:-1] + [nz], rank, world)
    step = (hi[-1] - lo[-1]) / (nz - 1) if nz > 1 else 0.0
    z0 = lo[-1] + k0 * step
    z1 = lo[-1] + (k1 - 1) * step
    return tuple(lo[:-1] + [z0]), tuple(hi[:-1] + [z1]), tuple(dims[:-1] + [k1 - k0]), (k0, k1, nz)
