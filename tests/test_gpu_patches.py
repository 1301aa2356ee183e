"""GPU parity of the parametric-surface path (bicubic Bezier patches) against
the FP64 oracle.  The oracle's definition is the adaptive quadrature of the
solid-angle element over the patches; its crossing count is round(w - B) with
B the FP64 boundary term on a fine sampling of the boundary curves (2048
segments per curve, error ~1e-8), so it shares no step with the library's
degree computation.  Bars: crossing counts equal on every query away from the
surface; w equal to chi + B(the library's own polyline) to 1e-6 (float32
boundary term) and to the definition within the boundary sampling error."""
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


def _away(P, band):
    """queries whose distance from the origin differs from 1 by more than
    `band` (the spheroids lie within 1 +- amp of the unit sphere, so band =
    amp + margin keeps the queries at least the margin from the surface)"""
    r = np.linalg.norm(P.astype(np.float64), axis=1)
    return np.abs(r - 1.0) > band


def _oracle_chi(ctrl, P, d):
    wd = oracle.w3d_patches_quad(ctrl, P)
    V, E = oracle.patch_boundary(ctrl, 2048)
    Bf = oracle.bterm3d(V, E, P, d) if len(E[0]) else np.zeros(len(P))
    chi = np.rint(wd - Bf)
    assert np.abs(wd - Bf - chi).max() < 1e-6          # the oracle's own consistency
    return wd, chi.astype(np.int64)


def test_closed_patch_surface_is_integer(gwn, ctx):
    pc = gen.patch_spheroid(n=2, amp=0.08, seed=1)
    ps = gwn.Patches(ctx, pc.ctrl, segments=16)
    assert ps.info()["n_boundary_edges"] == 0
    g = gen.Grid((-1.3,) * 3, (1.3,) * 3, (14, 14, 14))
    r = ps.eval(gwn.Grid(g.lo, g.hi, g.dims), pc.d, want_chi=True)
    w, chi = r["w"].cpu().numpy(), r["chi"].cpu().numpy()
    P = gen.grid_points(g)
    keep = _away(P, 0.08 + 0.03)
    wd, chio = _oracle_chi(pc.ctrl, P[keep], pc.d)
    assert np.array_equal(chi[keep], chio)
    assert np.array_equal(w[keep], chi[keep].astype(np.float32))      # no boundary: w = chi exactly
    assert set(np.unique(chio)) <= {0, 1}
    import torch
    wp = torch.empty(g.n).pin_memory()                                 # kernels write the pinned buffer
    ps.eval_host(gwn.Grid(g.lo, g.hi, g.dims), pc.d, out=wp)
    assert np.array_equal(wp.numpy(), w)


@pytest.mark.parametrize("seed, n, amp", [(2, 2, 0.08), (3, 3, 0.15)])
def test_open_patch_surface(gwn, ctx, seed, n, amp):
    pc = gen.patch_spheroid(n=n, amp=amp, open_faces=(4,), seed=seed)
    seg = 64
    ps = gwn.Patches(ctx, pc.ctrl, segments=seg)
    info = ps.info()
    assert info["n_loops"] == 1 and info["n_boundary_edges"] == 4 * n * seg
    g = gen.Grid((-1.3,) * 3, (1.3,) * 3, (13, 13, 13))
    P = gen.grid_points(g)
    keep = _away(P, amp + 0.03)
    Pk = P[keep]
    wd, chio = _oracle_chi(pc.ctrl, Pk, pc.d)
    V, E = oracle.patch_boundary(pc.ctrl, seg)
    B64 = oracle.bterm3d(V, E, Pk, pc.d)
    for q in (gwn.Grid(g.lo, g.hi, g.dims), gwn.Points(P)):
        r = ps.eval(q, pc.d, want_chi=True)
        w, chi = r["w"].cpu().numpy()[keep], r["chi"].cpu().numpy()[keep]
        assert np.array_equal(chi, chio)
        assert np.abs(w - (chio + B64)).max() <= 1e-6          # float32 boundary term on the same polyline
        assert np.abs(w - wd).max() <= 2e-5                     # boundary sampling (64 segments per curve)
    assert np.any(chio != 0)


def test_direction_independence_and_near_queries(gwn, ctx):
    """w does not depend on d while chi does; queries 0.02 from the shell make
    the patches straddle the plane through the query (subdivision)."""
    pc = gen.patch_spheroid(n=2, amp=0.05, open_faces=(1, 4), seed=5)
    ps = gwn.Patches(ctx, pc.ctrl, segments=128)
    rng = np.random.default_rng(9)
    v = rng.standard_normal((400, 3))
    P = (rng.uniform(0.5, 1.3, (400, 1)) * v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
    P = P[_away(P, 0.05 + 0.02)]
    wd, _ = _oracle_chi(pc.ctrl, P, pc.d)
    ws, chis = [], []
    for k in range(3):
        d = gen.random_direction(100 + k)
        r = ps.eval(gwn.Points(P), d, want_chi=True)
        ws.append(r["w"].cpu().numpy())
        chis.append(r["chi"].cpu().numpy())
        _, chio = _oracle_chi(pc.ctrl, P, d)
        assert np.array_equal(chis[-1], chio)
        assert np.abs(ws[-1] - wd).max() <= 1e-5
    assert np.abs(ws[0] - ws[1]).max() <= 2e-6 and np.abs(ws[0] - ws[2]).max() <= 2e-6
    assert np.any(chis[0] != chis[1]) or np.any(chis[0] != chis[2])


def test_patch_errors(gwn, ctx):
    import paper_2408_04466_gb300 as pkg
    bad = gen.patch_spheroid(n=1).ctrl.copy()
    bad[0, 1, 1, 0] = np.nan
    with pytest.raises(pkg.GwnError):
        gwn.Patches(ctx, bad)
    with pytest.raises(pkg.GwnError):
        gwn.Patches(ctx, gen.patch_spheroid(n=1).ctrl, segments=0)


def test_boundary_sampling_has_no_jumps(gwn, ctx):
    """The boundary term runs over the sampled boundary, so the crossing count
    must be that of the surface bounded by the samples: a ray through the thin
    region between a boundary curve and its chords must not see w jump by one.
    With 8 and 16 segments per curve the regions are wide (sagitta ~1e-3):
    across a 96^3 grid the two results may differ only by the sampling error,
    never by a jump, and both match the definition within that error."""
    pc = gen.patch_spheroid(n=2, amp=0.08, open_faces=(4,), seed=7)
    g = gen.Grid((-1.3,) * 3, (1.3,) * 3, (96, 96, 96))
    grid = gwn.Grid(g.lo, g.hi, g.dims)
    w8 = gwn.Patches(ctx, pc.ctrl, segments=8).eval(grid, pc.d).cpu().numpy()
    w16 = gwn.Patches(ctx, pc.ctrl, segments=16).eval(grid, pc.d).cpu().numpy()
    P = gen.grid_points(g)
    away = _away(P, 0.08 + 0.05)
    dw = np.abs(w8 - w16)[away]
    assert dw.max() < 0.05, dw.max()
    rng = np.random.default_rng(1)
    idx = np.nonzero(away)[0]
    idx = np.concatenate([idx[np.argsort(-np.abs(w8 - w16)[idx])[:40]], rng.choice(idx, 200, replace=False)])
    wd = oracle.w3d_patches_quad(pc.ctrl, P[idx])
    assert np.abs(w16[idx] - wd).max() < 0.02


def test_flipped_face_and_collapsed_edge(gwn, ctx):
    """Inconsistent orientation: one face's patches reversed (u and v swapped),
    so the curves it shares with its neighbours run the same way on both sides
    (net multiplicity 2, sampled twice) while its inner edges still cancel; and
    a single patch with one edge collapsed to a point (that curve bounds
    nothing).  Both against the oracle: exact chi, w within the sampling
    error of the definition."""
    pc = gen.patch_spheroid(n=2, amp=0.06, open_faces=(5,), seed=11)
    ctrl = pc.ctrl.copy()
    ctrl[:4] = np.swapaxes(ctrl[:4], 1, 2)                 # the first face, reversed
    seg = 128
    ps = gwn.Patches(ctx, ctrl, segments=seg)
    info = ps.info()
    # the open face's 8 curves once (2 of them on the flipped face), the 6 curves
    # the flipped face shares with its 3 closed neighbours twice
    assert info["n_boundary_edges"] == (8 + 2 * 6) * seg
    rng = np.random.default_rng(4)
    v = rng.standard_normal((600, 3))
    P = (rng.uniform(0.3, 1.35, (600, 1)) * v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
    P = P[_away(P, 0.06 + 0.04)]
    wd, chio = _oracle_chi(ctrl, P, pc.d)
    r = ps.eval(gwn.Points(P), pc.d, want_chi=True)
    assert np.array_equal(r["chi"].cpu().numpy(), chio)
    assert np.abs(r["w"].cpu().numpy() - wd).max() <= 1e-5
    assert np.abs(np.rint(wd) - wd).max() > 0.1            # genuinely open: w not integer

    # one patch, its u = 0 edge collapsed to the apex (a cone-like cap)
    cap = np.zeros((1, 4, 4, 3), np.float32)
    for i in range(4):
        for j in range(4):
            r_ = i / 3.0
            th = 0.5 * np.pi * j / 3.0
            cap[0, i, j] = (r_ * np.cos(th), r_ * np.sin(th), 0.4 * (1.0 - r_ * r_))
    ps1 = gwn.Patches(ctx, cap, segments=256)
    assert ps1.info()["n_boundary_edges"] == 3 * 256
    Q = (rng.uniform(-1.0, 1.0, (400, 3)) * np.array([1.2, 1.2, 1.0])).astype(np.float32)
    d1 = oracle.dist3d(*_cap_mesh(cap), Q)
    Q = Q[d1 > 0.05]
    wd1, chio1 = _oracle_chi(cap, Q, pc.d)
    r1 = ps1.eval(gwn.Points(Q), pc.d, want_chi=True)
    assert np.array_equal(r1["chi"].cpu().numpy(), chio1)
    assert np.abs(r1["w"].cpu().numpy() - wd1).max() <= 1e-5


def _cap_mesh(cap, k=64):
    """a fine triangle mesh of the patch (only to keep test queries off it)"""
    u = np.linspace(0, 1, k + 1)
    b = np.stack([(1 - u) ** 3, 3 * u * (1 - u) ** 2, 3 * u ** 2 * (1 - u), u ** 3], 1)
    X = np.einsum("ai,bj,ijc->abc", b, b, cap[0].astype(np.float64)).reshape(-1, 3).astype(np.float32)
    F = []
    for a in range(k):
        for c in range(k):
            i0 = a * (k + 1) + c
            F += [(i0, i0 + k + 1, i0 + 1), (i0 + 1, i0 + k + 1, i0 + k + 2)]
    return X, np.array(F, np.int32)


def test_patch_benchmark_workload_sampled(gwn, ctx):
    """The benchmark configuration itself (320 patches, one face open, 64
    segments per boundary curve, the full 256^3 grid in one call): exact chi
    and w against the oracle on a seeded sample of the queries away from the
    surface."""
    pc = gen.patch_spheroid(n=8, amp=0.08, open_faces=(4,), grid_n=256, seed=0)
    ps = gwn.Patches(ctx, pc.ctrl, segments=64)
    g = pc.grid
    r = ps.eval(gwn.Grid(g.lo, g.hi, g.dims), pc.d, want_chi=True)
    rng = np.random.default_rng(17)
    idx = rng.choice(g.n, 6000, replace=False)
    P = gen.grid_points(g, index=idx)
    keep = _away(P, 0.08 + 0.02)
    idx, P = idx[keep][:1500], P[keep][:1500]
    wd, chio = _oracle_chi(pc.ctrl, P, pc.d)
    V, E = oracle.patch_boundary(pc.ctrl, 64)
    B64 = oracle.bterm3d(V, E, P, pc.d)
    w = r["w"].cpu().numpy()[idx]
    assert np.array_equal(r["chi"].cpu().numpy()[idx], chio)
    assert np.abs(w - (chio + B64)).max() <= 1e-6
    assert np.abs(w - wd).max() <= 2e-5
