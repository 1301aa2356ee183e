"""GPU backward (dw/dp, dw/dV) against the FP64 oracle gradient of the
per-triangle solid-angle sum and against Richardson-extrapolated central
differences of the oracle's w.  Every comparison is per query (dw/dp) or per
vertex (dw/dV), never through an array norm:

    |g - g_ref| <= RTOL * |g_ref| + ATOL      (Euclidean norm of one row)

with RTOL = 1e-4."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu
RTOL = 1e-4
# dw/dp: where the gradient nearly vanishes the float32 sum over boundary
# edges cancels and relative error loses meaning; ATOL is far below the
# gradient magnitudes of these workloads (1e-2 .. 1): a float32 sum of ~2000
# edge terms of size ~1e-3 .. 1 cancels to ~1e-7.
ATOL = 1e-7


def _rows_close(g, ref, atol):
    """Per-row check; returns the indices of rows that fail."""
    g = np.asarray(g, np.float64).reshape(len(ref), -1)
    ref = np.asarray(ref, np.float64).reshape(len(ref), -1)
    err = np.linalg.norm(g - ref, axis=1)
    bar = RTOL * np.linalg.norm(ref, axis=1) + atol
    return np.nonzero(err > bar)[0], err, bar


def _assert_rows(g, ref, atol, what):
    bad, err, bar = _rows_close(g, ref, atol)
    assert len(bad) == 0, (f"{what}: {len(bad)} of {len(ref)} rows off; worst row {bad[np.argmax(err[bad] / bar[bad])]}"
                           f" err/bar {np.max(err[bad] / bar[bad]):.3g}")


def _vertex_atol(ogV, vid):
    """dw/dV rows are sums over queries of terms of both signs, accumulated in
    float32: the absolute part of the bar is 1e-6 of the largest boundary row."""
    return 1e-6 * float(np.linalg.norm(ogV[vid], axis=1).max())


def _check_vertex_grad(gV, ogV, vid, what):
    gV = np.asarray(gV, np.float64)
    _assert_rows(gV[vid], ogV[vid], _vertex_atol(ogV, vid), what)
    interior = np.setdiff1d(np.arange(len(gV)), vid)
    # interior vertices carry no gradient: exactly 0 from the library (the
    # oracle's chain rule over all triangles cancels there; pinned on the CPU)
    assert np.all(gV[interior] == 0), what


def _richardson_grad(V, F, P, h=2.0 ** -8):
    """Central differences of the oracle's w at steps h and h/2 along each
    axis, combined by Richardson extrapolation (error O(h^4)).  The points are
    snapped to multiples of 2^-12 first so that p +- h and p +- h/2 are exact
    in float32 (the oracle reads float32 queries); returns (snapped P, grad)."""
    P0 = (np.round(np.asarray(P, np.float64) * 4096.0) / 4096.0).astype(np.float32)
    pts = []
    for s in (h, h / 2):
        for k in range(3):
            for sg in (1.0, -1.0):
                Q = P0.astype(np.float64).copy()
                Q[:, k] += sg * s
                assert np.array_equal(Q.astype(np.float32).astype(np.float64), Q)
                pts.append(Q.astype(np.float32))
    w = oracle.w3d_vos(V, F, np.concatenate(pts)).reshape(2, 3, 2, len(P0))
    D = (w[:, :, 0] - w[:, :, 1]) / (2 * np.array([h, h / 2]))[:, None, None]     # [step, axis, query]
    R = (4.0 * D[1] - D[0]) / 3.0
    return P0, R.T


@pytest.fixture(scope="module")
def gwn(cuda_available):
    import paper_2408_04466_gb300 as pkg
    from paper_2408_04466_gb300 import build
    build.build()
    return pkg


@pytest.fixture(scope="module")
def ctx(gwn):
    return gwn.Context(0)


def test_small_torus_gradients(gwn, ctx):
    import torch
    m = gen.slit_torus(n_u=48, n_v=32, n_queries=256, seed=2)
    mesh = gwn.Mesh(ctx, m.V, m.F)
    off, vid = mesh.boundary()
    P = m.points[:64]
    gw = np.random.default_rng(1).standard_normal(len(P)).astype(np.float32)
    gp, gV = mesh.backward(torch.as_tensor(P).cuda(), torch.as_tensor(gw).cuda())
    torch.cuda.synchronize()
    ogp, ogV = oracle.grad3d_vos(m.V, m.F, P, gw=gw.astype(np.float64))
    _assert_rows(gp.cpu().numpy(), ogp, ATOL, "dw/dp")
    _check_vertex_grad(gV.cpu().numpy(), ogV, vid, "dw/dV")
    # Richardson-extrapolated central differences of the oracle's w, on the
    # queries at least 0.1 from the surface (truncation ~ (h / 0.1)^4 ~ 2e-6)
    far = np.nonzero(oracle.dist3d(m.V, m.F, m.points) > 0.1)[0][:16]
    assert len(far) >= 8
    P0, fd = _richardson_grad(m.V, m.F, m.points[far])
    g1, _ = mesh.backward(torch.as_tensor(P0).cuda(), torch.ones(len(P0), device="cuda"), want_V=False)
    torch.cuda.synchronize()
    _assert_rows(g1.cpu().numpy(), fd, ATOL, "dw/dp vs finite differences")


def test_gradients_near_edges(gwn, ctx):
    """Queries inside the sphere on a boundary edge as diameter (a.b < 0, the
    endpoint weights through |a x E|^2 / (|a||b| - a.b)), queries on the
    extension of an edge (a, b nearly parallel) and random queries, in one
    call: the warps then mix lanes of both branches.  320 boundary edges, so
    one full block of edges and one partial block.  Per query and per vertex
    against the FP64 oracle gradient."""
    import torch
    m = gen.slit_torus(n_u=48, n_v=160, n_queries=512, seed=5)
    mesh = gwn.Mesh(ctx, m.V, m.F)
    off, vid = mesh.boundary()
    assert len(vid) == 320
    rng = np.random.default_rng(11)
    V = m.V.astype(np.float64)
    pts = []
    for lp in range(len(off) - 1):
        loop = vid[off[lp]:off[lp + 1]]
        for i in rng.choice(len(loop), 12, replace=False):
            A, B = V[loop[i]], V[loop[(i + 1) % len(loop)]]
            E = B - A
            L = np.linalg.norm(E)
            n = np.cross(E, rng.standard_normal(3))
            n /= np.linalg.norm(n)
            for t, dd in ((0.5, 0.02), (0.3, 0.1), (0.7, 0.3), (0.5, 0.45)):
                pts.append(A + t * E + dd * L * n)          # a.b < 0
            pts.append(B + 0.3 * E + 0.05 * L * n)          # beyond B, a.b > 0
    P = np.concatenate([np.asarray(pts, np.float32), m.points[:137]])     # 257 queries: a ragged group
    rng.shuffle(P)
    gw = rng.uniform(0.5, 1.5, len(P)).astype(np.float32)
    gp, gV = mesh.backward(torch.as_tensor(P).cuda(), torch.as_tensor(gw).cuda())
    torch.cuda.synchronize()
    ctx.check()
    ogp, ogV = oracle.grad3d_vos(m.V, m.F, P, gw=gw.astype(np.float64))
    _assert_rows(gp.cpu().numpy(), ogp, ATOL, "dw/dp near edges")
    _check_vertex_grad(gV.cpu().numpy(), ogV, vid, "dw/dV near edges")
    # each gradient alone takes its own kernels
    gp1, _ = mesh.backward(torch.as_tensor(P).cuda(), torch.as_tensor(gw).cuda(), want_V=False)
    _, gV1 = mesh.backward(torch.as_tensor(P).cuda(), torch.as_tensor(gw).cuda(), want_p=False)
    torch.cuda.synchronize()
    _assert_rows(gp1.cpu().numpy(), ogp, ATOL, "dw/dp alone near edges")
    _check_vertex_grad(gV1.cpu().numpy(), ogV, vid, "dw/dV alone near edges")


def test_backward_degenerate_inputs(gwn, ctx):
    """A closed surface has no boundary: both gradients are exactly zero (w is
    piecewise constant off the surface).  No queries: dw/dV is zero and
    nothing else is touched.  One query and one boundary loop of 3 edges
    (the single triangle): per query and per vertex against the oracle."""
    import torch
    Vs, Fs = gen.icosphere(2)
    mesh = gwn.Mesh(ctx, Vs.astype(np.float32), Fs.astype(np.int32))
    assert mesh.info()["n_boundary_edges"] == 0
    P = np.random.default_rng(3).uniform(-1.5, 1.5, (100, 3)).astype(np.float32)
    gp, gV = mesh.backward(torch.as_tensor(P).cuda(), torch.ones(len(P), device="cuda"))
    torch.cuda.synchronize()
    assert torch.count_nonzero(gp).item() == 0 and torch.count_nonzero(gV).item() == 0
    m = gen.slit_torus(n_u=16, n_v=12, n_queries=8, seed=1)
    mesh = gwn.Mesh(ctx, m.V, m.F)
    gp, gV = mesh.backward(torch.zeros((0, 3), device="cuda"), torch.zeros(0, device="cuda"))
    torch.cuda.synchronize()
    assert gp.shape == (0, 3) and torch.count_nonzero(gV).item() == 0
    V = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float32)
    F = np.array([[0, 1, 2]], np.int32)
    tri = gwn.Mesh(ctx, V, F)
    _, vid = tri.boundary()
    P = np.array([[0.2, 0.3, -0.4]], np.float32)
    gw = np.array([0.7], np.float32)
    gp, gV = tri.backward(torch.as_tensor(P).cuda(), torch.as_tensor(gw).cuda())
    torch.cuda.synchronize()
    ogp, ogV = oracle.grad3d_vos(V, F, P, gw=gw.astype(np.float64))
    _assert_rows(gp.cpu().numpy(), ogp, ATOL, "dw/dp single triangle")
    _check_vertex_grad(gV.cpu().numpy(), ogV, vid, "dw/dV single triangle")


def test_autograd_function(gwn, ctx):
    import torch
    m = gen.icosphere_cap(subdiv=2, seed=4)
    mesh = gwn.Mesh(ctx, m.V, m.F)
    _, vid = mesh.boundary()
    rng = np.random.default_rng(0)
    P = rng.uniform(-1.3, 1.3, (200, 3)).astype(np.float32)
    P = P[oracle.dist3d(m.V, m.F, P) > 0.05]
    Pt = torch.as_tensor(P).cuda().requires_grad_(True)
    Vt = torch.as_tensor(m.V).cuda().requires_grad_(True)
    w = gwn.gwn_apply(mesh, Pt, Vt, m.d)
    loss = (w * torch.arange(len(P), device="cuda", dtype=torch.float32)).sum()
    loss.backward()
    gw = np.arange(len(P), dtype=np.float64)
    ogp, ogV = oracle.grad3d_vos(m.V, m.F, P, gw=gw)
    _assert_rows(Pt.grad.cpu().numpy(), ogp, ATOL * max(1.0, gw.max()), "autograd dw/dp")
    _check_vertex_grad(Vt.grad.cpu().numpy(), ogV, vid, "autograd dw/dV")
    wo, _, _ = oracle.w3d_oneshot(m.V, m.F, P, m.d)
    assert np.abs(w.detach().cpu().numpy() - wo).max() < 1e-6


def test_torus_full_size_sampled(gwn, ctx):
    """The differentiation workload at full size: 2.1M-triangle slit torus, 1M
    queries, forward + backward in the bench's launch configuration.  1024
    sampled queries: crossing counts exact and |dw| <= 1e-6 against the
    oracle, dw/dp per query against the oracle gradient; dw/dV of all 2048
    boundary vertices per vertex against the oracle over a 192-query
    subsample (its own backward call); translation invariance over all 1M."""
    import torch
    m = gen.slit_torus()
    mesh = gwn.Mesh(ctx, m.V, m.F)
    info = mesh.info()
    assert info["n_loops"] == 2 and info["n_boundary_edges"] == 2048
    _, vid = mesh.boundary()
    Pt = torch.as_tensor(m.points).cuda()
    r = mesh.eval(gwn.Points(Pt), m.d, want_chi=True)
    gw = torch.ones(len(Pt), device="cuda")
    gp, gV = mesh.backward(Pt, gw)
    torch.cuda.synchronize()
    ctx.check()
    rng = np.random.default_rng(8)
    idx = np.sort(rng.choice(len(Pt), 1024, replace=False))
    P = m.points[idx]
    wo, chio, _ = oracle.w3d_oneshot(m.V, m.F, P, m.d)
    assert np.array_equal(r["chi"].cpu().numpy()[idx], chio)
    assert np.abs(r["w"].cpu().numpy()[idx] - wo).max() <= 1e-6
    sub = idx[:192]
    gws = rng.uniform(0.5, 1.5, len(sub)).astype(np.float32)
    ogp, ogV = oracle.grad3d_vos(m.V, m.F, m.points[sub], gw=gws.astype(np.float64))
    _assert_rows(gp.cpu().numpy()[sub] * gws[:, None], ogp, ATOL, "dw/dp (full size)")
    sp, sV = mesh.backward(torch.as_tensor(m.points[sub]).cuda(), torch.as_tensor(gws).cuda())
    torch.cuda.synchronize()
    _assert_rows(sp.cpu().numpy(), ogp, ATOL, "dw/dp (subsample call)")
    _check_vertex_grad(sV.cpu().numpy(), ogV, vid, "dw/dV (full size)")
    # translation invariance of the summed gradients over all 1M queries:
    # sum_q dw/dp = -sum_v dw/dV, component by component
    s_p = gp.double().sum(0).cpu().numpy()
    s_v = gV.double().sum(0).cpu().numpy()
    assert np.all(np.abs(s_p + s_v) <= 1e-3 * np.abs(s_p).max())
