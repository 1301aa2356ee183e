"""GPU parity of the 2D one-shot path (one +x ray per grid row) against the
FP64 oracle: crossing counts bit-exact on every query the oracle certifies
(all but queries on the curve at float64 resolution; none on these inputs
unless a test places one there); |dw| <= 1e-12 (float64 chains) or 1e-6
(float32 chains) at queries farther than 1e-4 x bbox diagonal from the
curve; batched evaluation identical to per-chain evaluation."""
import math

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


def _grid(gwn, g):
    return gwn.Grid(g.lo, g.hi, g.dims)


def _compare_chain(ctrl64, grid, w, chi, tol, n_unc=0):
    P = gen.grid_points(grid, np.float64 if w.dtype == np.float64 else np.float32).astype(np.float64)
    wq = oracle.w2d_quad(ctrl64, P)
    wc, chic, unc = oracle.w2d_closed_x(ctrl64, P, want_unc=True)
    assert unc.sum() == n_unc, np.nonzero(unc)[0][:10]
    # crossing counts on every certified query, near the curve included
    bad = np.nonzero((chi != chic) & ~unc)[0]
    assert len(bad) == 0, (len(bad), P[bad[:5]].tolist(), chi[bad[:5]].tolist(), chic[bad[:5]].tolist())
    diag = math.hypot(grid.hi[0] - grid.lo[0], grid.hi[1] - grid.lo[1])
    keep = oracle.dist2d(ctrl64, P) > 1e-4 * diag
    err = np.abs(w.astype(np.float64) - wq)[keep].max()
    assert err <= tol, err
    return keep


def test_circle_chain_fp64_full_grid(gwn, ctx):
    c = gen.bezier_circle_chain()
    ch = gwn.Bezier2D(ctx, c.ctrl, c.offsets)
    r = ch.eval(_grid(gwn, c.grids[0]), want_chi=True, want_b=True)
    w = r["w"].cpu().numpy()
    chi = r["chi"].cpu().numpy()
    assert w.dtype == np.float64
    _compare_chain(c.ctrl, c.grids[0], w, chi, 1e-12)
    # the chord term is the boundary part: w - chi
    assert np.array_equal(w - chi, r["b"].cpu().numpy()) or np.abs(w - chi - r["b"].cpu().numpy()).max() < 1e-15


def test_straight_and_closed_chains(gwn, ctx):
    # a closed chain gives integers; a straight segment gives the subtended angle
    m = 3 * 16
    th = 2 * np.pi * np.arange(m + 1) / m
    ctrl = np.stack([np.cos(th), np.sin(th)], 1)
    ctrl[-1] = ctrl[0]
    ch = gwn.Bezier2D(ctx, ctrl, [0, m + 1])
    g = gen.Grid((-1.5, -1.5), (1.5, 1.5), (64, 48))
    w = ch.eval(_grid(gwn, g)).cpu().numpy()
    P = gen.grid_points(g, np.float64)
    keep = oracle.dist2d(ctrl, P) > 1e-3
    assert np.all((np.abs(w - 1) < 1e-12) | (np.abs(w) < 1e-12) | ~keep)
    _compare_chain(ctrl, g, w, ch.eval(_grid(gwn, g), want_chi=True)["chi"].cpu().numpy(), 1e-12)


def test_star_chains_fp32_and_batch(gwn, ctx):
    import torch
    cs = gen.star_chains(n_chains=12, seg_hi=300, grid_n=48, seed=4)
    ch = gwn.Bezier2D(ctx, cs.ctrl, cs.offsets)
    grids = [_grid(gwn, g) for g in cs.grids]
    wb, offs = ch.eval_batch(grids)
    wb2, _ = ch.eval_batch(grids)      # graph replay
    torch.cuda.synchronize()
    assert torch.equal(wb, wb2)
    wb = wb.cpu().numpy()
    for c in range(cs.meta["n_chains"]):
        ctrl = cs.ctrl[cs.offsets[c]:cs.offsets[c + 1]]
        single = gwn.Bezier2D(ctx, ctrl, [0, len(ctrl)])
        r = single.eval(grids[c], want_chi=True)
        ws = r["w"].cpu().numpy()
        n = grids[c].n
        assert np.array_equal(ws, wb[offs[c]:offs[c] + n]), c
        _compare_chain(ctrl.astype(np.float64), cs.grids[c], ws, r["chi"].cpu().numpy(), 1e-6)
    t, rows = ch.batch_plan()
    assert t in (128, 256) and rows in (4, 8, 16, 32, 64)
    # a forced plan gives the same numbers
    wf, _ = ch.eval_batch(grids, threads=256, rows=1, use_graph=False)
    assert np.array_equal(wf.cpu().numpy(), wb)


def test_multi_chain_union(gwn, ctx):
    """gwn_eval on a geometry with several chains sums their winding numbers."""
    cs = gen.star_chains(n_chains=3, seg_hi=40, grid_n=20, seed=9, dtype=np.float64)
    ch = gwn.Bezier2D(ctx, cs.ctrl, cs.offsets)
    g = gen.Grid((-1.6, -1.6), (1.6, 1.6), (40, 36))
    w = ch.eval(_grid(gwn, g)).cpu().numpy()
    P = gen.grid_points(g, np.float64)
    tot = np.zeros(len(P))
    keep = np.ones(len(P), bool)
    for c in range(3):
        ctrl = cs.ctrl[cs.offsets[c]:cs.offsets[c + 1]]
        tot += oracle.w2d_quad(ctrl, P)
        keep &= oracle.dist2d(ctrl, P) > 1e-3
    assert np.abs(w - tot)[keep].max() < 1e-11


def test_bruteforce_2d(gwn, ctx):
    c = gen.bezier_circle_chain(grid_n=24)
    ch = gwn.Bezier2D(ctx, c.ctrl, c.offsets)
    wb = ch.bruteforce(_grid(gwn, c.grids[0])).cpu().numpy()
    P = gen.grid_points(c.grids[0], np.float64)
    keep = oracle.dist2d(c.ctrl, P) > 0.05
    assert np.abs(wb - oracle.w2d_quad(c.ctrl, P))[keep].max() < 1e-9


def test_errors_2d(gwn, ctx):
    with pytest.raises(gwn.GwnError):
        gwn.Bezier2D(ctx, np.zeros((5, 2)), [0, 5])       # not 3k+1
    c = gen.bezier_circle_chain(grid_n=8)
    ch = gwn.Bezier2D(ctx, c.ctrl, c.offsets)
    import torch
    with pytest.raises(gwn.GwnError):       # float32 points for a float64 chain
        q = gwn.Points(torch.zeros((4, 2), dtype=torch.float32, device="cuda"))
        w = torch.empty(4, dtype=torch.float64, device="cuda")
        import ctypes as C
        gwn._capi.check(ch.lib.gwn_eval(ch.h, C.byref(q.to_c()), None, w.data_ptr(), None, None, None), "eval")


def test_star_chains_full_size_sampled(gwn, ctx):
    """The batched workload at full size: 1024 chains, 256^2 grid each, one
    persistent graph launch; a sample of chains is checked query by query."""
    import torch
    cs = gen.star_chains()
    ch = gwn.Bezier2D(ctx, cs.ctrl, cs.offsets)
    grids = [_grid(gwn, g) for g in cs.grids]
    w, offs = ch.eval_batch(grids)
    torch.cuda.synchronize()
    ctx.check()
    rng = np.random.default_rng(5)
    nseg = (np.diff(cs.offsets) - 1) // 3
    pick = list(rng.choice(len(grids), 6, replace=False)) + [int(np.argmax(nseg))]
    for c in pick:
        ctrl = cs.ctrl[cs.offsets[c]:cs.offsets[c + 1]].astype(np.float64)
        n = grids[c].n
        sub = np.sort(rng.choice(n, 1500, replace=False))
        wc = w[int(offs[c]):int(offs[c]) + n].cpu().numpy()[sub]
        P = gen.grid_points(cs.grids[c], np.float32, index=sub).astype(np.float64)
        wq = oracle.w2d_quad(ctrl, P)
        g = cs.grids[c]
        keep = oracle.dist2d(ctrl, P) > 1e-4 * math.hypot(g.hi[0] - g.lo[0], g.hi[1] - g.lo[1])
        assert np.abs(wc.astype(np.float64) - wq)[keep].max() <= 1e-6, c


def _zigzag(n):
    xk = np.arange(n + 1, dtype=np.float64)
    yk = np.where(np.arange(n + 1) % 2 == 0, -1.0, 1.0)
    ctrl = np.zeros((3 * n + 1, 2))
    for k in range(n):
        for j in range(3):
            t = j / 3.0
            ctrl[3 * k + j] = ((1 - t) * xk[k] + t * xk[k + 1], (1 - t) * yk[k] + t * yk[k + 1])
    ctrl[-1] = (xk[-1], yk[-1])
    return ctrl


@pytest.mark.parametrize("n, dims, dtype", [(600, (64, 256), np.float64), (8500, (24, 12), np.float64),
                                            (33000, (40, 8), np.float32)])
def test_many_crossings_per_row(gwn, ctx, n, dims, dtype):
    """A zig-zag chain crossing every row n times (up to 33000 crossings on a
    row, 264k in one work item).  64 rows per work item and 4 rows per work
    item agree exactly, and with the oracle's closed form; the float32 case
    takes the fast row path with the two separate lane scans (more than 32766
    pieces in an item), which must give the generic path's w bit for bit."""
    ctrl = _zigzag(n).astype(dtype)
    ch = gwn.Bezier2D(ctx, ctrl, [0, len(ctrl)])
    g = gen.Grid((-1.0, -1.37), (n + 1.0, 1.41), dims)
    grid = gwn.Grid(g.lo, g.hi, g.dims)
    w_big, _ = ch.eval_batch([grid], threads=128, rows=64, use_graph=False)
    w_bin, _ = ch.eval_batch([grid], threads=128, rows=4, use_graph=False)
    w_big = w_big.cpu().numpy()
    w_bin = w_bin.cpu().numpy()
    assert np.array_equal(w_big, w_bin)
    P = gen.grid_points(g, dtype).astype(np.float64)
    wc, chic, unc = oracle.w2d_closed_x(ctrl.astype(np.float64), P, want_unc=True)
    assert not unc.any()
    if dtype == np.float64:
        keep = oracle.dist2d(ctrl, P) > 1e-6
        assert np.abs(w_bin - wc)[keep].max() < 1e-11
    r = ch.eval(grid, want_chi=True)
    assert np.array_equal(r["chi"].cpu().numpy(), chic)
    assert np.array_equal(r["w"].cpu().numpy(), w_bin)


def test_point_queries_bucket_order(gwn, ctx):
    """From 65,536 points on, the point path evaluates the queries in the
    order of their y-buckets: w and chi equal, bit for bit, those of the
    same points evaluated in chunks below that size (the given order), float32
    and float64; chi matches the oracle on a sample."""
    import torch
    rng = np.random.default_rng(33)
    cs = gen.star_chains(n_chains=1, seg_lo=600, seg_hi=600, grid_n=16, seed=4)
    circ = gen.bezier_circle_chain()
    for ctrl, g, dt in ((cs.ctrl, cs.grids[0], np.float32), (circ.ctrl, circ.grids[0], np.float64)):
        ch = gwn.Bezier2D(ctx, np.ascontiguousarray(ctrl, dt), [0, len(ctrl)])
        n = 150000
        P = np.stack([rng.uniform(g.lo[0], g.hi[0], n), rng.uniform(g.lo[1], g.hi[1], n)], 1).astype(dt)
        Pt = torch.as_tensor(P).cuda()
        r = ch.eval(gwn.Points(Pt), want_chi=True)
        w, chi = r["w"].cpu().numpy(), r["chi"].cpu().numpy()
        parts = [ch.eval(gwn.Points(Pt[a:a + 50000]), want_chi=True) for a in range(0, n, 50000)]
        assert np.array_equal(w, np.concatenate([q["w"].cpu().numpy() for q in parts]))
        assert np.array_equal(chi, np.concatenate([q["chi"].cpu().numpy() for q in parts]))
        sub = rng.choice(n, 3000, replace=False)
        _, chic, unc = oracle.w2d_closed_x(np.asarray(ctrl, np.float64), P[sub].astype(np.float64), want_unc=True)
        assert np.array_equal(chi[sub][~unc], chic[~unc])


def test_point_queries(gwn, ctx):
    """One +x ray per query point (no ray reuse): crossing counts exact and
    w against the oracle's closed form, float64 and float32 chains; grid
    points given as points agree with the grid path away from the curve."""
    import torch
    c = gen.bezier_circle_chain()
    ch = gwn.Bezier2D(ctx, c.ctrl, c.offsets)
    rng = np.random.default_rng(21)
    P = rng.uniform(-1.5, 1.5, (6000, 2))
    # points on rows through control points and through piece end values
    P[:200, 1] = c.ctrl[rng.integers(0, len(c.ctrl), 200), 1]
    r = ch.eval(gwn.Points(torch.as_tensor(P).cuda()), want_chi=True)
    w = r["w"].cpu().numpy()
    chi = r["chi"].cpu().numpy()
    wc, chic, unc = oracle.w2d_closed_x(c.ctrl, P, want_unc=True)
    assert not unc.any()
    assert np.array_equal(chi, chic)
    keep = oracle.dist2d(c.ctrl, P) > 1e-9
    assert np.abs(w - wc)[keep].max() < 1e-12
    # host points
    wh = ch.eval(gwn.Points(torch.as_tensor(P))).cpu().numpy()
    assert np.array_equal(wh, w)
    # grid points as points vs the grid path
    g = c.grids[0]
    Pg = gen.grid_points(g, np.float64)
    wg = ch.eval(_grid(gwn, g)).cpu().numpy()
    wp = ch.eval(gwn.Points(torch.as_tensor(Pg).cuda())).cpu().numpy()
    far = oracle.dist2d(c.ctrl, Pg) > 1e-6
    assert np.abs(wg - wp)[far].max() < 1e-13
    # float32, several chains (w sums over the chains)
    cs = gen.star_chains(n_chains=3, seg_hi=300, grid_n=20, seed=9)
    st = gwn.Bezier2D(ctx, cs.ctrl, cs.offsets)
    Q = rng.uniform(-1.6, 1.6, (8000, 2)).astype(np.float32)
    r = st.eval(gwn.Points(torch.as_tensor(Q).cuda()), want_chi=True)
    w32 = r["w"].cpu().numpy().astype(np.float64)
    tot = np.zeros(len(Q))
    tchi = np.zeros(len(Q), np.int64)
    keep = np.ones(len(Q), bool)
    for k in range(3):
        ctrl = cs.ctrl[cs.offsets[k]:cs.offsets[k + 1]].astype(np.float64)
        wk, ck, uk = oracle.w2d_closed_x(ctrl, Q.astype(np.float64), want_unc=True)
        assert not uk.any()
        tot += wk
        tchi += ck
        keep &= oracle.dist2d(ctrl, Q.astype(np.float64)) > 1e-4 * math.hypot(3.2, 3.2)
    assert np.array_equal(r["chi"].cpu().numpy(), tchi)
    assert np.abs(w32 - tot)[keep].max() <= 1e-6
    # no points
    assert st.eval(gwn.Points(torch.zeros((0, 2), device="cuda"))).numel() == 0


def _near_curve_grids(dtype):
    """Grids whose queries sit within float rounding of crossings: the
    parabola y = x - x^2/3 on [0, 3] (apex (3/2, 3/4); rows 3/4 + k h for
    |k| <= 8, columns through both crossings of each row) and the tent
    (0,0)-(3,3)-(6,0) (rows 3/2 + k h, columns 3/2 + j h).  h is a few float32
    ulps for float32 chains; for float64 chains 2^-40, far below float32 but
    above the oracle's float64 resolution."""
    h = 4 * 2.0 ** -23 if dtype == np.float32 else 2.0 ** -40
    para = np.array([[0, 0], [1, 1], [2, 1], [3, 0]], dtype)
    tent = np.array([[0, 0], [1, 1], [2, 2], [3, 3], [4, 2], [5, 1], [6, 0]], dtype)
    return [(para, gen.Grid((1.5 - 0.004, 0.75 - 8 * h), (1.5 + 0.004, 0.75 + 8 * h), (801, 17))),
            (para, gen.Grid((1.5 - 64 * h, 0.75 - 8 * h), (1.5 + 64 * h, 0.75 + 8 * h), (129, 17))),
            (tent, gen.Grid((1.5 - 32 * h, 1.5 - 8 * h), (1.5 + 32 * h, 1.5 + 8 * h), (65, 17)))]


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_crossings_certified_near_the_curve(gwn, ctx, dtype):
    """Queries within float rounding of the curve: rows through (and a few
    ulps around) the apex of a parabola, where Newton's root is least
    accurate and the apex value is rounded, and columns a few ulps from the
    crossings of a straight segment.  The float path lists these crossings
    for the float64 certification; the counts must equal the oracle's on
    every query it certifies (it leaves out the queries on the curve at
    float64 resolution: the apex, the tent's line), through the row path, the
    batched path and the point path."""
    import torch
    n_cert = 0
    for ctrl, g in _near_curve_grids(dtype):
        ch = gwn.Bezier2D(ctx, ctrl, [0, len(ctrl)])
        grid = _grid(gwn, g)
        r = ch.eval(grid, want_chi=True, stats=True)
        chi = r["chi"].cpu().numpy()
        n_cert += r["stats"]["n_cert"]
        P = gen.grid_points(g, dtype).astype(np.float64)
        wc, chic, unc = oracle.w2d_closed_x(ctrl.astype(np.float64), P, want_unc=True)
        # on the curve at float64 resolution: the tent's line (17 queries) or
        # the apex row's queries within ~1e-20 (in y) of the parabola
        assert unc.sum() <= max(17, g.dims[0]), (g, int(unc.sum()))
        bad = np.nonzero((chi != chic) & ~unc)[0]
        assert len(bad) == 0, (g, len(bad), P[bad[:4]].tolist(), chi[bad[:4]].tolist(), chic[bad[:4]].tolist())
        wb, _ = ch.eval_batch([grid], use_graph=False)
        assert np.array_equal(wb.cpu().numpy(), r["w"].cpu().numpy())
        rp = ch.eval(gwn.Points(torch.as_tensor(P.astype(dtype)).cuda()), want_chi=True)
        chip = rp["chi"].cpu().numpy()
        assert np.array_equal(chip[~unc], chic[~unc])
    assert n_cert > 0                                      # the certification pass had work
    ctx.check()
