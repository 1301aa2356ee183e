"""Batched evaluation of many meshes of uneven sizes (gwn_eval_meshes): one
persistent launch over (mesh, query-tile) work items, replayed from a CUDA
graph, must give every query the same bits as gwn_eval on its own mesh."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gwn(cuda_available):
    import paper_2408_04466_gb300 as pkg
    from paper_2408_04466_gb300 import build
    build.build()
    return pkg


@pytest.fixture(scope="module")
def ctx(gwn):
    return gwn.Context(0)


def _meshes():
    """Nine meshes from 1e3 to 1e6 triangles, with a grid or a point list each."""
    out = []
    for s in (3, 4, 5, 6):
        m = gen.icosphere_cap(subdiv=s, grid_n=24 + 8 * s, seed=s)
        out.append((m.V, m.F, gen.Grid((-1.2, -1.15, -1.25), (1.2, 1.3, 1.1), (24 + 8 * s, 20 + 8 * s, 28)), None))
    for nu, nv, nq in ((96, 64, 20000), (512, 512, 300000), (720, 720, 1 << 20)):
        m = gen.slit_torus(n_u=nu, n_v=nv, n_queries=nq, seed=nu)
        out.append((m.V, m.F, None, m.points))
    for n, holes in ((128, 6), (256, 10)):
        m = gen.holey_heightfield(n=n, n_holes=holes, grid_n=40, seed=n)
        out.append((m.V, m.F, gen.Grid(m.grid.lo, m.grid.hi, (48, 40, 36)), None))
    return out


def test_meshes_batched_bit_identical(gwn, ctx):
    import torch
    d = gen.random_direction(31)
    meshes, queries, refs = [], [], []
    specs = _meshes()
    assert len(specs) >= 8
    for k, (V, F, g, P) in enumerate(specs):
        mesh = gwn.Mesh(ctx, V, F)
        if k in (1, 5):
            mesh.set_index("tree")                       # the LBVH path in the batch as well
        mesh.prepare(d)
        q = gwn.Grid(g.lo, g.hi, g.dims) if g is not None else gwn.Points(torch.as_tensor(P).cuda())
        # two evaluations: the second has the bins where the first built them
        mesh.eval(q, d)
        refs.append(mesh.eval(q, d).clone())
        meshes.append(mesh)
        queries.append(q)
    tri = [len(F) for V, F, g, P in specs]
    assert min(tri) < 2000 and max(tri) > 1_000_000
    assert sum(m.info()["n_bins"] > 0 for m in meshes) >= 3   # both crossing paths take part
    outs = [torch.full_like(r, float("nan")) for r in refs]
    gwn.eval_meshes(ctx, meshes, queries, d, outs=outs)     # plan, autotune, capture
    torch.cuda.synchronize()
    ctx.check()
    for k, (o, r) in enumerate(zip(outs, refs)):
        assert torch.equal(o, r), (k, int((o != r).sum()))
    for o in outs:
        o.fill_(float("nan"))
    _, st = gwn.eval_meshes(ctx, meshes, queries, d, outs=outs, stats=True)   # graph replay
    torch.cuda.synchronize()
    ctx.check()
    for k, (o, r) in enumerate(zip(outs, refs)):
        assert torch.equal(o, r), (k, int((o != r).sum()))
    assert st["n_queries"] == sum(q.n for q in queries)
    tiles, blocks = gwn.meshes_plan(ctx)
    assert tiles in (1, 4, 16) and blocks in (1, 2)
    # a forced shape without the graph gives the same bits
    outs2 = gwn.eval_meshes(ctx, meshes, queries, d, tiles_per_item=4, blocks_per_sm=1, use_graph=False)
    torch.cuda.synchronize()
    for k, (o, r) in enumerate(zip(outs2, refs)):
        assert torch.equal(o, r), k
    # spot check against the oracle on the smallest mesh
    V, F, g, _ = specs[0]
    Pq = gen.grid_points(g)
    sub = np.arange(0, len(Pq), 97)
    wo, _, _ = oracle.w3d_oneshot(V, F, Pq[sub], d)
    keep = oracle.dist3d(V, F, Pq[sub]) > 1e-4 * float(np.linalg.norm(V.max(0) - V.min(0)))
    assert np.abs(outs[0].cpu().numpy()[sub] - wo)[keep].max() <= 1e-6


def test_meshes_batch_errors(gwn, ctx):
    import torch
    m = gen.icosphere_cap(subdiv=3, seed=2)
    mesh = gwn.Mesh(ctx, m.V, m.F)
    g = gwn.Grid((-1, -1, -1), (1, 1, 1), (8, 8, 8))
    with pytest.raises(gwn.GwnError):                  # not prepared for d
        gwn.eval_meshes(ctx, [mesh], [g], m.d)
    mesh.prepare(m.d)
    with pytest.raises(gwn.GwnError):                  # host points
        gwn.eval_meshes(ctx, [mesh], [gwn.Points(torch.zeros((4, 3)))], m.d)
    w = gwn.eval_meshes(ctx, [mesh], [g], m.d)[0]
    torch.cuda.synchronize()
    assert torch.equal(w, mesh.eval(g, m.d))
    ctx.check()
