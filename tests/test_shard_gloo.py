"""Multi-rank query sharding, exercised with world_size-2 gloo ranks on the
CPU: each rank takes its z-slab of the weak-scaled grid, the slabs tile the
global grid exactly, and the max-over-ranks timing reduction is correct."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2408_04466_gb300.shard import shard_grid, slab


def test_slab_partition():
    for nz in (1, 2, 7, 256, 513):
        for world in (1, 2, 3, 4, 8):
            if nz < world:
                continue
            spans = [slab((4, 4, nz), r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == nz
            for a, b in zip(spans, spans[1:]):
                assert a[1] == b[0]
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi, dims, (k0, k1, nz) = shard_grid((-1.2, -1.2, -1.2), (1.2, 1.2, 1.2), (8, 8, 8), rank, world, weak=True)
    # each rank's planes, as global plane indices, gathered on every rank
    mine = torch.tensor([k0, k1, nz, dims[2]], dtype=torch.int64)
    allv = [torch.zeros(4, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(allv, mine)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    if rank == 0:
        q.put(([v.tolist() for v in allv], float(t.item()), lo, hi, dims))
    dist.destroy_process_group()


def test_weak_sharding_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    spans, tmax, lo, hi, dims = res
    assert tmax == 2.0
    assert spans[0][0] == 0 and spans[0][1] == spans[1][0] and spans[1][1] == 16
    assert all(s[3] == 8 for s in spans)          # weak: every rank keeps 8 planes
    assert np.isclose(lo[2], -1.2)


def _grad_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import gen
    import oracle
    from paper_2408_04466_gb300.shard import allreduce_grad_vertices, shard_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = gen.icosphere_cap(subdiv=2, seed=4)
    P = np.random.default_rng(0).uniform(-1.3, 1.3, (96, 3)).astype(np.float32)
    gw = np.linspace(-1.0, 2.0, len(P))
    i0, i1 = shard_range(len(P), rank, world)
    gp, gv = oracle.grad3d_vos(m.V, m.F, P[i0:i1], gw=gw[i0:i1])
    gv = torch.as_tensor(gv)
    allreduce_grad_vertices(gv)
    dist.barrier()
    if rank == 0:
        q.put((gv.numpy(), i0, i1))
    dist.destroy_process_group()


def test_backward_allreduce_two_gloo_ranks():
    """dw/dV summed over two ranks' query shards equals dw/dV over all
    queries (the one exchange step of the sharded backward)."""
    import gen
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 30500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_grad_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gv, i0, i1 = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert (i0, i1) == (0, 48)
    m = gen.icosphere_cap(subdiv=2, seed=4)
    P = np.random.default_rng(0).uniform(-1.3, 1.3, (96, 3)).astype(np.float32)
    gw = np.linspace(-1.0, 2.0, len(P))
    _, full = oracle.grad3d_vos(m.V, m.F, P, gw=gw)
    assert np.allclose(gv, full, rtol=1e-12, atol=1e-14)
