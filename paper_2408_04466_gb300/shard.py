"""Query sharding across ranks (one process per GPU).

Queries are independent, so a grid is split into contiguous z-slabs (a point
list into contiguous ranges), one per rank, with no collective on the
forward path; every rank keeps a full copy of the geometry.  With
``weak=True`` the global grid grows with the world size so each rank keeps
the single-GPU number of queries.

The backward pass has one exchange step: dw/dV is a sum over queries, so each
rank's gradient over its own queries is summed across ranks
(``allreduce_grad_vertices``); dw/dp stays with the rank that owns the query.
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


def shard_range(n: int, rank: int, world: int):
    """[i0, i1) of a list of n queries owned by `rank` (contiguous, sizes
    differ by at most one)."""
    base, extra = divmod(int(n), world)
    i0 = rank * base + min(rank, extra)
    return i0, i0 + base + (1 if rank < extra else 0)


def allreduce_grad_vertices(grad_v):
    """Sum dw/dV (a tensor, in place) over the ranks of the default process
    group; a no-op without one or with a single rank."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(grad_v, op=dist.ReduceOp.SUM)
    return grad_v
