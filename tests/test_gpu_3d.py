"""GPU parity of the 3D one-shot path against the FP64 oracle, through the
C ABI.  Bar: crossing counts bit-exact on every query; |dw| <= 1e-6 (float32
path) at queries farther than 1e-4 x bbox diagonal from the surface."""
import math

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu
TOL = 1e-6


@pytest.fixture(scope="module")
def gwn(cuda_available):
    import paper_2408_04466_gb300 as pkg
    from paper_2408_04466_gb300 import build
    build.build()
    return pkg


@pytest.fixture(scope="module")
def ctx(gwn):
    return gwn.Context(0)


def _diag(V):
    V = np.asarray(V, np.float64)
    return float(np.linalg.norm(V.max(0) - V.min(0)))


def _run(gwn, ctx, V, F, P, d, **kw):
    mesh = gwn.Mesh(ctx, V, F)
    import torch
    Pt = torch.as_tensor(np.ascontiguousarray(P, np.float32)).cuda()
    r = mesh.eval(gwn.Points(Pt), d, want_chi=True, want_b=True, **kw)
    torch.cuda.synchronize()
    ctx.check()
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in r.items()}


def _check(V, F, P, d, r, tol=TOL, near=1e-4):
    wo, chio, Bo = oracle.w3d_oneshot(V, F, P, d)
    assert np.array_equal(r["chi"], chio), f"chi mismatch on {(r['chi'] != chio).sum()} queries"
    dist = oracle.dist3d(V, F, P)
    keep = dist > near * _diag(V)
    if keep.any():
        errB = np.where(keep, np.abs(r["b"].astype(np.float64) - Bo), 0.0)
        errw = np.where(keep, np.abs(r["w"].astype(np.float64) - wo), 0.0)
        i = int(np.argmax(errw))
        assert errB.max() <= tol and errw.max() <= tol, (
            f"max |dB| {errB.max():.3e}, max |dw| {errw.max():.3e} at query {i} p={P[i].tolist()} "
            f"dist={dist[i]:.3e} w_gpu={r['w'][i]!r} w_oracle={wo[i]!r} chi={r['chi'][i]}")
    return keep


def test_octant_and_closed_cube(gwn, ctx):
    V = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float32)
    F = np.array([[0, 1, 2]], np.int32)
    for s in range(4):
        d = gen.random_direction(100 + s)
        r = _run(gwn, ctx, V, F, np.zeros((1, 3)), d)
        assert abs(r["w"][0] - 0.125) < TOL
    Vc = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], np.float32)
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    Fc = np.array([t for a, b, c, dd in quads for t in ((a, b, c), (a, c, dd))], np.int32)
    n = np.cross(Vc[Fc[:, 1]] - Vc[Fc[:, 0]], Vc[Fc[:, 2]] - Vc[Fc[:, 0]])
    flip = np.einsum("ij,ij->i", n, Vc[Fc].mean(1)) < 0
    Fc[flip] = Fc[flip][:, [0, 2, 1]]
    rng = np.random.default_rng(0)
    P = rng.uniform(-2, 2, (4000, 3)).astype(np.float32)
    P = P[np.abs(np.abs(P).max(1) - 1) > 1e-3]
    r = _run(gwn, ctx, Vc, Fc, P, gen.random_direction(7))
    inside = np.abs(P).max(1) < 1
    assert np.array_equal(r["chi"], inside.astype(np.int32))
    assert np.all(r["b"] == 0) and np.abs(r["w"] - inside).max() == 0


def test_small_cap_full_grid(gwn, ctx):
    m = gen.icosphere_cap(subdiv=4, grid_n=32, seed=3)
    P = gen.grid_points(m.grid)
    mesh = gwn.Mesh(ctx, m.V, m.F)
    r = mesh.eval(gwn.Grid(m.grid.lo, m.grid.hi, m.grid.dims), m.d, want_chi=True, want_b=True, stats=True)
    import torch
    torch.cuda.synchronize()
    rr = {k: v.cpu().numpy() for k, v in r.items() if k != "stats"}
    _check(m.V, m.F, P, m.d, rr)
    st = r["stats"]
    assert st["n_queries"] == len(P) and st["n_stack_overflow"] == 0
    assert st["n_pairs"] == len(P) * mesh.info()["n_boundary_edges"]


def test_queries_beside_long_edges(gwn, ctx):
    """A 2 x 2 square (two triangles, four boundary edges of length 2) seen
    from queries 3e-4 .. 1e-2 from the interior of its boundary edges, on
    their outer side in every direction about the edge: a and b nearly
    opposite, the float32 boundary term's worst conditioning.  |dw| <= 1e-6 on every query."""
    V = np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0]], np.float32)
    F = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    rng = np.random.default_rng(21)
    n = 4000
    e = rng.integers(0, 4, n)
    t = rng.uniform(-0.9, 0.9, n)
    h = 10 ** rng.uniform(np.log10(3e-4), -2, n)
    # edge k runs along axis (k % 2) at the fixed other coordinate +-1
    along = np.where(e % 2 == 0, 0, 1)
    other = np.where((e == 0) | (e == 3), -1.0, 1.0)
    ang = rng.uniform(-np.pi / 2, np.pi / 2, n)       # on the outer side of the edge: distance h from M
    P = np.zeros((n, 3))
    P[np.arange(n), along] = t
    P[np.arange(n), 1 - along] = other * (1.0 + h * np.cos(ang))
    P[:, 2] = h * np.sin(ang)
    P = P.astype(np.float32)
    for s in range(3):
        d = gen.random_direction(300 + s)
        r = _run(gwn, ctx, V, F, P, d)
        keep = _check(V, F, P, d, r)
        assert keep.mean() > 0.95


def test_soups_with_multiplicities(gwn, ctx):
    """Random soups (non-manifold, repeated faces): long edges (up to ~5
    units) pass close to queries, the case where a float32 boundary term is
    ill-conditioned (a and b nearly opposite); the library recomputes those
    pairs in float64, so the bar is the workload bar, 1e-6, on every query
    beyond 1e-4 x diagonal, against both the one-shot oracle and the
    definition."""
    rng = np.random.default_rng(11)
    for trial in range(3):
        V = rng.standard_normal((40, 3)).astype(np.float32)
        F = rng.integers(0, 40, (70, 3)).astype(np.int32)
        F = F[(F[:, 0] != F[:, 1]) & (F[:, 1] != F[:, 2]) & (F[:, 0] != F[:, 2])]
        F = np.concatenate([F, F[:6]])
        P = (2.5 * rng.standard_normal((3000, 3))).astype(np.float32)
        d = gen.random_direction(200 + trial)
        r = _run(gwn, ctx, V, F, P, d)
        keep = _check(V, F, P, d, r)
        wv = oracle.w3d_vos(V, F, P)
        errv = np.abs(r["w"].astype(np.float64) - wv)[keep]
        assert errv.max() <= TOL, errv.max()


def test_near_cut_and_axis_directions(gwn, ctx):
    """Rays grazing boundary edges, and axis-aligned directions on a grid
    (exact zero determinants: the symbolic perturbation decides)."""
    m = gen.icosphere_cap(subdiv=3, seed=5)
    src, dst, _ = oracle.boundary_edges(m.F)
    V = m.V.astype(np.float64)
    d = m.d.astype(np.float64)
    pts = []
    rng = np.random.default_rng(2)
    for e in range(len(src)):
        A, B = V[src[e]], V[dst[e]]
        for t in rng.uniform(0.05, 0.95, 3):
            x = A + t * (B - A)
            side = np.cross(B - A, d)
            side /= np.linalg.norm(side)
            for off in (-1e-5, -1e-7, 0.0, 1e-7, 1e-5):
                pts.append(x - rng.uniform(0.3, 1.5) * d + off * side)
    P = np.array(pts, np.float32)
    r = _run(gwn, ctx, m.V, m.F, P, m.d)
    _check(m.V, m.F, P, m.d, r)
    # axis-aligned directions with grid-aligned vertices and queries
    Vg = np.array([[x, y, 0.0] for x in range(4) for y in range(4)], np.float32)
    Fg = []
    for i in range(3):
        for j in range(3):
            a, b, c, dd = 4 * i + j, 4 * (i + 1) + j, 4 * (i + 1) + j + 1, 4 * i + j + 1
            Fg += [(a, b, c), (a, c, dd)]
    Fg = np.array(Fg, np.int32)
    g = np.arange(-1, 5, 0.5, dtype=np.float32)
    P = np.array([[x, y, z] for x in g for y in g for z in (-1.0, -0.5, 0.5, 1.0)], np.float32)
    for d in ([0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1, 1]):
        d = np.array(d, np.float32)
        r = _run(gwn, ctx, Vg, Fg, P, d)
        _check(Vg, Fg, P, d, r)


def test_edge_cases(gwn, ctx):
    import torch
    d = gen.random_direction(1)
    # empty mesh: w = 0
    r = _run(gwn, ctx, np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), np.ones((5, 3)), d)
    assert np.all(r["w"] == 0) and np.all(r["chi"] == 0)
    # one triangle, non-unit direction
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    F = np.array([[0, 1, 2]], np.int32)
    P = np.array([[0.2, 0.2, -1], [0.2, 0.2, 1], [2, 2, -1]], np.float32)
    r = _run(gwn, ctx, V, F, P, np.array([0.01, 0.02, 5.0], np.float32))
    _check(V, F, P, np.array([0.01, 0.02, 5.0], np.float32), r)
    # zero queries
    mesh = gwn.Mesh(ctx, V, F)
    w = mesh.eval(gwn.Points(torch.zeros((0, 3), device="cuda")), d)
    assert w.numel() == 0
    # host queries and the end-to-end entry point
    Pq = np.random.default_rng(0).uniform(-1, 1, (100, 3)).astype(np.float32)
    wd = mesh.eval(gwn.Points(torch.as_tensor(Pq).cuda()), d).cpu().numpy()
    wh = mesh.eval(gwn.Points(torch.as_tensor(Pq)), d).cpu().numpy()
    we = mesh.eval_host(Pq, d)
    assert np.array_equal(wd, wh) and np.array_equal(wd, we)


def test_eval_host_pinned_output(gwn, ctx):
    """A page-locked host output is written by the kernels directly; the
    values are the device path's, bit for bit (grid and point queries)."""
    import torch
    m = gen.icosphere_cap(subdiv=3, grid_n=24, seed=2)
    mesh = gwn.Mesh(ctx, m.V, m.F)
    g = gwn.Grid(m.grid.lo, m.grid.hi, m.grid.dims)
    wd = mesh.eval(g, m.d).cpu().numpy()
    wp = torch.full((g.n,), float("nan")).pin_memory()
    mesh.eval_host(g, m.d, out=wp)
    assert np.array_equal(wp.numpy(), wd)
    assert np.array_equal(mesh.eval_host(g, m.d), wd)        # pageable: device buffer + copy
    P = gen.grid_points(m.grid)[::7].astype(np.float32)
    wq = mesh.eval(gwn.Points(torch.as_tensor(P).cuda()), m.d).cpu().numpy()
    wpp = torch.empty(len(P)).pin_memory()
    mesh.eval_host(P, m.d, out=wpp)
    assert np.array_equal(wpp.numpy(), wq)
    ctx.check()


def test_invalid_inputs_are_errors(gwn, ctx):
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    with pytest.raises(gwn.GwnError):
        gwn.Mesh(ctx, V, np.array([[0, 1, 3]], np.int32))
    Vn = V.copy()
    Vn[1, 1] = np.nan
    with pytest.raises(gwn.GwnError):
        gwn.Mesh(ctx, Vn, np.array([[0, 1, 2]], np.int32))
    mesh = gwn.Mesh(ctx, V, np.array([[0, 1, 2]], np.int32))
    import torch
    with pytest.raises(gwn.GwnError):
        mesh.eval(gwn.Points(torch.zeros((3, 3), device="cuda")), [0, 0, 0])
    # the context stays usable after errors
    w = mesh.eval(gwn.Points(torch.zeros((3, 3), device="cuda")), [0, 0, 1])
    torch.cuda.synchronize()
    ctx.check()


def _unit_edges_of_loops(off, vid):
    out = []
    for j in range(len(off) - 1):
        lo, hi = int(off[j]), int(off[j + 1])
        for i in range(lo, hi):
            out.append((int(vid[i]), int(vid[i + 1] if i + 1 < hi else vid[lo])))
    return sorted(out)


def _oracle_unit_edge_list(F):
    src, dst, m = oracle.boundary_edges(F)
    out = []
    for s, t, k in zip(src, dst, m):
        out += [(int(s), int(t))] * int(k)
    return sorted(out)


@pytest.mark.parametrize("name", ["cap", "torus", "heightfield", "closed", "soup", "wide_ids", "one_vertex", "empty"])
def test_device_boundary_extraction(gwn, ctx, name):
    """The mesh's boundary loops come from the device intake (half-edge keys,
    radix sort over the key bytes that vertex ids of this size occupy, net
    multiplicities): the unit edges equal the oracle's, and the loops equal the
    host extraction's exactly."""
    rng = np.random.default_rng(11)
    if name == "cap":
        m = gen.icosphere_cap(subdiv=4)
        V, F = m.V, m.F
    elif name == "torus":
        m = gen.slit_torus(n_u=48, n_v=40, n_queries=16)
        V, F = m.V, m.F
    elif name == "heightfield":
        m = gen.holey_heightfield(n=96, n_holes=3)
        V, F = m.V, m.F
    elif name == "closed":
        V, F = gen.icosphere(3)
    elif name == "soup":          # multiplicities 2 and 0, degenerate faces; ids < 256
        V = rng.standard_normal((200, 3)).astype(np.float32)
        F = rng.integers(0, 200, (600, 3)).astype(np.int32)
        F = np.concatenate([F, F[:40], F[:9, [0, 2, 1]], np.array([[5, 5, 7], [9, 9, 9]], np.int32)])
    elif name == "wide_ids":      # ids up to 70,000: three bytes of each id vary
        V = rng.standard_normal((70000, 3)).astype(np.float32)
        F = rng.integers(0, 70000, (5000, 3)).astype(np.int32)
        F = np.concatenate([F, F[:500, [1, 0, 2]], F[500:800]])
    elif name == "one_vertex":
        V = np.zeros((1, 3), np.float32)
        F = np.zeros((3, 3), np.int32)
    else:
        V = rng.standard_normal((4, 3)).astype(np.float32)
        F = np.zeros((0, 3), np.int32)
    V = np.ascontiguousarray(V, np.float32)
    F = np.ascontiguousarray(F, np.int32)
    mesh = gwn.Mesh(ctx, V, F)
    off, vid = mesh.boundary()
    hoff, hvid = gwn.boundary_extract_host(F, len(V))
    assert np.array_equal(np.asarray(off), np.asarray(hoff)) and np.array_equal(np.asarray(vid), np.asarray(hvid))
    assert _unit_edges_of_loops(off, vid) == _oracle_unit_edge_list(F)
    info = mesh.info()
    assert info["n_boundary_edges"] == len(vid) and info["n_loops"] == len(off) - 1
    # device-resident input takes the same path
    import torch
    md = gwn.Mesh(ctx, torch.as_tensor(V).cuda(), torch.as_tensor(F).cuda())
    doff, dvid = md.boundary()
    assert np.array_equal(np.asarray(doff), np.asarray(off)) and np.array_equal(np.asarray(dvid), np.asarray(vid))
    ctx.check()


@pytest.mark.parametrize("case", ["cap_grid", "cap_points", "lattice_soup", "torus_points", "heightfield_grid",
                                  "far_points"])
def test_bins_equal_tree(gwn, ctx, case):
    """The 2D bin index (built once the evaluations reach 4 queries per
    triangle) and the LBVH traversal test the same (query, triangle)
    pairs: crossing counts and w are identical, grid and point queries,
    including a lattice soup whose rays pass through vertices and edges and
    whose query boxes straddle bin boundaries."""
    import torch
    rng = np.random.default_rng(5)
    d = gen.random_direction(9)
    if case.startswith("cap"):
        m = gen.icosphere_cap(subdiv=5, grid_n=72, seed=3)
        V, F, d = m.V, m.F, m.d
        q = gwn.Grid(m.grid.lo, m.grid.hi, m.grid.dims) if case == "cap_grid" else \
            gwn.Points(torch.as_tensor(gen.grid_points(m.grid)[::3].copy()).cuda())
    elif case == "lattice_soup":
        # triangles inside the cells of an 11^3 lattice; d = (1, 2, 3) maps
        # lattice points to lattice points, so rays from the lattice queries
        # pass through vertices
        L = np.stack(np.meshgrid(*(np.arange(11.0),) * 3, indexing="ij"), -1).reshape(-1, 3)
        V = (L / 10.0).astype(np.float32)
        c = rng.integers(0, 10, (900, 3))
        steps = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [1, 0, 1], [0, 1, 1], [1, 1, 1]])
        a, b = steps[rng.integers(0, 7, 900)], steps[rng.integers(0, 7, 900)]
        cid = lambda x: (x[:, 0] * 11 + x[:, 1]) * 11 + x[:, 2]
        F = np.stack([cid(c), cid(c + a), cid(c + b)], 1).astype(np.int32)
        F = np.concatenate([F, F[:50], F[:20, [0, 2, 1]]])
        d = np.array([1.0, 2.0, 3.0], np.float32)
        P = np.concatenate([V, (rng.integers(0, 21, (6000, 3)) / 20.0).astype(np.float32)])
        q = gwn.Points(torch.as_tensor(P).cuda())
    elif case == "far_points":
        # points 1e4 along -d and +d from points of the mesh's box: their rays
        # cross the whole surface (or nothing), and their padded boxes (pad
        # grows with |p|) span several bins, so a pair must be counted in one
        # bin only
        m = gen.icosphere_cap(subdiv=3, grid_n=8, seed=12)
        V, F, d = m.V, m.F, m.d
        dh = d.astype(np.float64) / np.linalg.norm(d.astype(np.float64))
        c = rng.random((6000, 3)) * 2.0 - 1.0
        s_ = np.where(rng.random(6000) < 0.5, -1e4, 1e4)[:, None]
        P = (c + s_ * dh).astype(np.float32)
        q = gwn.Points(torch.as_tensor(P).cuda())
    elif case == "torus_points":
        m = gen.slit_torus(n_u=96, n_v=64, n_queries=60000, seed=2)
        V, F, d = m.V, m.F, m.d
        q = gwn.Points(torch.as_tensor(m.points).cuda())
    else:
        m = gen.holey_heightfield(n=160, n_holes=5, grid_n=64, seed=4)
        V, F, d = m.V, m.F, m.d
        q = gwn.Grid(m.grid.lo, m.grid.hi, m.grid.dims)
    mesh = gwn.Mesh(ctx, V, F)
    r_auto = mesh.eval(q, d, want_chi=True)
    info = mesh.info()
    mesh.set_index("tree")
    r_tree = mesh.eval(q, d, want_chi=True)
    torch.cuda.synchronize()
    ctx.check()
    assert info["n_bins"] > 0 and info["n_bin_entries"] >= len(F) - 100 and info["bin_maxlen"] > 0
    assert torch.equal(r_auto["chi"], r_tree["chi"])
    assert torch.equal(r_auto["w"], r_tree["w"])


def test_inside_voxelization(gwn, ctx):
    """The inside test (w >= 1/2) fused into the boundary term: bit-exact
    against the float32 w of the same path, and equal to the FP64 oracle's
    decision wherever the oracle's w is more than 1e-5 from the threshold."""
    import torch
    m = gen.icosphere_cap(subdiv=3, grid_n=20, seed=6)
    mesh = gwn.Mesh(ctx, m.V, m.F)
    g = gwn.Grid(m.grid.lo, m.grid.hi, m.grid.dims)
    w = mesh.eval(g, m.d)
    ins = mesh.inside(g, m.d)
    torch.cuda.synchronize()
    ctx.check()
    assert ins.dtype == torch.uint8
    assert torch.equal(ins, (w >= 0.5).to(torch.uint8))
    P = gen.grid_points(m.grid)
    wo, _, _ = oracle.w3d_oneshot(m.V, m.F, P, m.d)
    far = np.abs(wo - 0.5) > 1e-5
    assert np.array_equal(ins.cpu().numpy()[far], (wo[far] >= 0.5).astype(np.uint8))
    assert 0 < int(ins.sum()) < g.n
    # closed surface: inside exactly where w = 1
    V, F = gen.icosphere(3)
    closed = gwn.Mesh(ctx, V.astype(np.float32), F.astype(np.int32))
    Pq = (np.random.default_rng(1).random((5000, 3)) * 2.6 - 1.3).astype(np.float32)
    r = np.linalg.norm(Pq.astype(np.float64), axis=1)
    keep = np.abs(r - 1.0) > 0.05
    ci = closed.inside(gwn.Points(torch.as_tensor(Pq).cuda()), m.d).cpu().numpy()
    assert np.array_equal(ci[keep], (r[keep] < 1.0).astype(np.uint8))
    # patch surfaces take the same epilogue; 2D chains are not supported
    pc = gen.patch_spheroid(n=2, amp=0.08, seed=1)
    ps = gwn.Patches(ctx, pc.ctrl, segments=16)
    gp = gwn.Grid((-1.3,) * 3, (1.3,) * 3, (12, 12, 12))
    assert torch.equal(ps.inside(gp, pc.d), (ps.eval(gp, pc.d) >= 0.5).to(torch.uint8))
    ch = gen.bezier_circle_chain(n_seg=8, grid_n=8)
    geo = gwn.Bezier2D(ctx, ch.ctrl, ch.offsets)
    with pytest.raises(gwn.GwnError):
        gwn.Mesh.inside(geo, gwn.Grid(ch.grids[0].lo, ch.grids[0].hi, ch.grids[0].dims), [1, 0, 0])
    ctx.check()


def test_bins_built_once_enough_queries(gwn, ctx):
    """The bins are built by the evaluation at which the queries evaluated on
    a (mesh, d) reach 4 per triangle; a new direction starts the count again;
    the crossing counts do not change when they appear."""
    import torch
    m = gen.icosphere_cap(subdiv=4, grid_n=8, seed=8)
    nf = len(m.F)
    P = torch.as_tensor((np.random.default_rng(2).random((3 * nf, 3)) * 2.4 - 1.2).astype(np.float32)).cuda()
    mesh = gwn.Mesh(ctx, m.V, m.F)
    q = gwn.Points(P)
    c1 = mesh.eval(q, m.d, want_chi=True)["chi"].clone()
    assert mesh.info()["n_bins"] == 0                         # 3 queries per triangle so far
    c2 = mesh.eval(q, m.d, want_chi=True)["chi"].clone()
    assert mesh.info()["n_bins"] > 0                          # 6: built by this call
    assert torch.equal(c1, c2)
    d2 = gen.random_direction(77)
    mesh.eval(q, d2)
    assert mesh.info()["n_bins"] == 0                         # a new direction: a new count
    ctx.check()


def test_bruteforce_comparator(gwn, ctx):
    m = gen.icosphere_cap(subdiv=3, grid_n=16, seed=1)
    mesh = gwn.Mesh(ctx, m.V, m.F)
    g = gwn.Grid(m.grid.lo, m.grid.hi, m.grid.dims)
    wb = mesh.bruteforce(g).cpu().numpy()
    P = gen.grid_points(m.grid)
    wv = oracle.w3d_vos(m.V, m.F, P)
    keep = oracle.dist3d(m.V, m.F, P) > 1e-2
    assert np.abs(wb - wv)[keep].max() < 1e-4


def test_icosphere_cap_full_size_sampled(gwn, ctx):
    """The bench workload: 73,724 triangles, 256^3 grid, evaluated whole in
    the bench's launch configuration; sampled queries checked one by one."""
    import torch
    m = gen.icosphere_cap()
    mesh = gwn.Mesh(ctx, m.V, m.F)
    assert mesh.info()["n_boundary_edges"] == 252 and mesh.info()["n_loops"] == 1
    g = gwn.Grid(m.grid.lo, m.grid.hi, m.grid.dims)
    r = mesh.eval(g, m.d, want_chi=True, want_b=True, stats=True)
    torch.cuda.synchronize()
    ctx.check()
    assert r["stats"]["n_stack_overflow"] == 0
    n = m.grid.n
    rng = np.random.default_rng(123)
    idx = np.sort(rng.choice(n, 3000, replace=False))
    # plus queries whose ray passes near the boundary loop (the hard cases)
    chi_all = r["chi"]
    idx_t = torch.as_tensor(idx).cuda()
    P = gen.grid_points(m.grid, index=idx)
    rr = {"w": r["w"][idx_t].cpu().numpy(), "chi": chi_all[idx_t].cpu().numpy(), "b": r["b"][idx_t].cpu().numpy()}
    _check(m.V, m.F, P, m.d, rr)
    # global invariants over all 16.8M queries: w in a sane range, chi in {-1, 0, 1, 2}
    w = r["w"]
    assert torch.isfinite(w).all()
    vals = torch.unique(chi_all).cpu().numpy()
    assert set(vals.tolist()) <= {-2, -1, 0, 1, 2}


def test_degenerate_rays_overflow_pair_list(gwn, ctx):
    """Every ray through a mesh vertex exactly (axis-aligned flat grid mesh,
    queries under its vertices, d = +z): every triangle test is left
    unsettled by the float32 filter, far more pairs than the deferred-pair
    list holds, so queries are recounted whole as well.  Grid queries (packet
    traversal) and point queries (per-thread traversal) must both match the
    oracle's symbolically perturbed counts exactly."""
    import torch
    nv = 97
    Vg = np.array([[x, y, 0.0] for x in range(nv) for y in range(nv)], np.float32)
    Fg = []
    for i in range(nv - 1):
        for j in range(nv - 1):
            a, b, c, dd = nv * i + j, nv * (i + 1) + j, nv * (i + 1) + j + 1, nv * i + j + 1
            Fg += [(a, b, c), (a, c, dd)]
    Fg = np.array(Fg, np.int32)
    d = np.array([0, 0, 1], np.float32)
    mesh = gwn.Mesh(ctx, Vg, Fg)
    grid = gwn.Grid((-1.0, -1.0, -1.0), (nv, nv, -0.25), (nv + 2, nv + 2, 4))
    r = mesh.eval(grid, d, want_chi=True, stats=True)
    torch.cuda.synchronize()
    ctx.check()
    st = r["stats"]
    assert st["n_deferred_traverse"] > 65536            # the pair list overflowed
    P = gen.grid_points(gen.Grid(grid.lo, grid.hi, grid.dims))
    rng = np.random.default_rng(3)
    sub = np.sort(rng.choice(len(P), 3000, replace=False))
    chio = oracle.chi3d(Vg, Fg, P[sub], d)
    assert np.array_equal(r["chi"].cpu().numpy()[sub], chio)
    # the same queries as a point list
    Pt = torch.as_tensor(P).cuda()
    rp = mesh.eval(gwn.Points(Pt), d, want_chi=True)
    torch.cuda.synchronize()
    ctx.check()
    assert np.array_equal(rp["chi"].cpu().numpy(), r["chi"].cpu().numpy())


def test_axis_direction_line_reuse(gwn, ctx):
    """d parallel to a grid axis: one traversal per grid line serves all its
    queries.  Crossing counts on every query and w on a sample must match the
    oracle for each axis and both senses."""
    import torch
    m = gen.icosphere_cap(subdiv=3, seed=5)
    mesh = gwn.Mesh(ctx, m.V, m.F)
    g = gen.Grid((-1.2, -1.1, -1.3), (1.2, 1.25, 1.15), (40, 36, 32))
    grid = gwn.Grid(g.lo, g.hi, g.dims)
    P = gen.grid_points(g)
    rng = np.random.default_rng(11)
    sub = np.sort(rng.choice(len(P), 1500, replace=False))
    for d in ([0, 0, 1], [0, 0, -1], [1, 0, 0], [0, -1, 0]):
        d = np.array(d, np.float32)
        r = mesh.eval(grid, d, want_chi=True, want_b=True)
        torch.cuda.synchronize()
        ctx.check()
        chio = oracle.chi3d(m.V, m.F, P, d)
        assert np.array_equal(r["chi"].cpu().numpy(), chio), (d, int((r["chi"].cpu().numpy() != chio).sum()))
        rr = {k: r[k].cpu().numpy()[sub] for k in ("w", "chi", "b")}
        _check(m.V, m.F, P[sub], d, rr)


def _rim_distance(P, d, A, B, chunk=256):
    """Distance, in the plane normal to d, from each query's ray p + t d to the
    nearest boundary segment AB whose nearest point lies in front of p
    (float64; a selection heuristic for near-rim rays, not a parity input)."""
    d = np.asarray(d, np.float64)
    d = d / np.linalg.norm(d)
    e1 = np.cross(d, [1.0, 0.0, 0.0] if abs(d[0]) < 0.9 else [0.0, 1.0, 0.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    M = np.stack([e1, e2, d], 1)
    A2, B2 = A @ M, B @ M
    out = np.full(len(P), np.inf)
    for s in range(0, len(P), chunk):
        p2 = P[s:s + chunk].astype(np.float64) @ M
        a = A2[None] - p2[:, None]
        e = (B2 - A2)[None]
        ee = np.maximum((e[..., :2] ** 2).sum(-1), 1e-300)
        t = np.clip(-(a[..., :2] * e[..., :2]).sum(-1) / ee, 0.0, 1.0)
        c = a + t[..., None] * e
        r = np.hypot(c[..., 0], c[..., 1])
        r = np.where(c[..., 2] > 0, r, np.inf)
        out[s:s + chunk] = r.min(1)
    return out


def test_holey_heightfield_full_size_sampled(gwn, ctx):
    """The large-mesh workload at full size: heightfield disk of 8,102,716
    triangles with 32 holes (33 boundary loops, 17,478 edges), the whole
    512^3 grid (134,217,728 queries) evaluated in the bench's configuration.
    Crossing counts are compared exactly and w to 1e-6 with the FP64 oracle on
    512 seeded grid queries plus up to 512 grid queries whose ray passes
    within 1e-3 of a hole's rim (or the outer rim); the LBVH path (fixed
    traversal stack) must agree with the bins on every query and overflow
    nowhere."""
    import torch
    m = gen.holey_heightfield()
    mesh = gwn.Mesh(ctx, m.V, m.F)
    info = mesh.info()
    assert info["n_loops"] == 33 and info["n_boundary_edges"] == 17478
    g = gwn.Grid(m.grid.lo, m.grid.hi, m.grid.dims)
    r = mesh.eval(g, m.d, want_chi=True, want_b=True, stats=True)
    torch.cuda.synchronize()
    ctx.check()
    assert mesh.info()["n_bins"] > 0                      # 16.6 queries per triangle: the bins serve
    assert r["stats"]["n_stack_overflow"] == 0
    w_all, chi_all, b_all = r["w"], r["chi"], r["b"]
    assert torch.isfinite(w_all).all()
    assert set(torch.unique(chi_all).cpu().numpy().tolist()) <= {-2, -1, 0, 1, 2}

    n = m.grid.n
    rng = np.random.default_rng(2024)
    idx_u = rng.choice(n, 512, replace=False)
    # grid queries whose ray passes close to a rim: step back from a boundary
    # vertex along -d, snap to the nearest grid point, keep rays within 1e-3
    src, dst, _ = oracle.boundary_edges(m.F)
    A = m.V[src].astype(np.float64)
    B = m.V[dst].astype(np.float64)
    dh = m.d.astype(np.float64) / np.linalg.norm(m.d.astype(np.float64))
    lo = np.array(m.grid.lo, np.float64)
    hi = np.array(m.grid.hi, np.float64)
    nd = np.array(m.grid.dims)
    step = (hi - lo) / (nd - 1)
    pick = rng.integers(0, len(A), 6000)
    cand = A[pick] - rng.uniform(0.02, 1.0, (6000, 1)) * dh[None]
    ijk = np.rint((cand - lo) / step).astype(np.int64)
    ok = np.all((ijk >= 0) & (ijk < nd), 1)
    flat = np.unique(ijk[ok, 0] + nd[0] * (ijk[ok, 1] + nd[1] * ijk[ok, 2]))
    Pc = gen.grid_points(m.grid, index=flat)
    near = _rim_distance(Pc, m.d, A, B) < 1e-3
    idx_r = flat[near][:512]
    assert len(idx_r) >= 128, len(idx_r)
    idx = np.unique(np.concatenate([idx_u, idx_r]))
    ti = torch.as_tensor(idx).cuda()
    P = gen.grid_points(m.grid, index=idx)
    rr = {"w": w_all[ti].cpu().numpy(), "chi": chi_all[ti].cpu().numpy(), "b": b_all[ti].cpu().numpy()}
    keep = _check(m.V, m.F, P, m.d, rr)
    assert keep.sum() >= 0.9 * len(idx_u)

    # the LBVH traversal (64-entry stack per warp packet) on the full grid
    del b_all
    mesh.set_index("tree")
    rt = mesh.eval(g, m.d, want_chi=True, stats=True)
    torch.cuda.synchronize()
    ctx.check()
    assert rt["stats"]["n_stack_overflow"] == 0
    assert torch.equal(rt["chi"], chi_all)
    assert torch.equal(rt["w"], w_all)
