"""GPU backward (dw/dp, dw/dV) against the FP64 oracle gradient of the
per-triangle solid-angle sum and against central finite differences of the
oracle's w; relative tolerance 1e-4."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu
RTOL = 1e-4
# Where dw/dp nearly vanishes, the float32 sum over boundary edges cancels
# and relative error loses meaning; the per-query bar is
#   |g_gpu - g_oracle| <= RTOL * |g_oracle| + ATOL,
# with ATOL far below the gradient magnitudes of these workloads (1e-2 .. 1):
# a float32 sum of ~2000 edge terms of size ~1e-3 .. 1 cancels to ~1e-7.
ATOL = 1e-7


def _close(g, ref):
    return np.linalg.norm(g - ref) <= RTOL * np.linalg.norm(ref) + ATOL


@pytest.fixture(scope="module")
def gwn(cuda_available):
    import paper_2408_04466_gb300 as pkg
    from paper_2408_04466_gb300 import build
    build.build()
    return pkg


@pytest.fixture(scope="module")
def ctx(gwn):
    return gwn.Context(0)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_small_torus_gradients(gwn, ctx):
    import torch
    m = gen.slit_torus(n_u=48, n_v=32, n_queries=256, seed=2)
    mesh = gwn.Mesh(ctx, m.V, m.F)
    P = m.points[:64]
    gw = np.random.default_rng(1).standard_normal(len(P)).astype(np.float32)
    gp, gV = mesh.backward(torch.as_tensor(P).cuda(), torch.as_tensor(gw).cuda())
    torch.cuda.synchronize()
    gp = gp.cpu().numpy().astype(np.float64)
    gV = gV.cpu().numpy().astype(np.float64)
    ogp, ogV = oracle.grad3d_vos(m.V, m.F, P, gw=gw.astype(np.float64))
    for q in range(len(P)):
        assert _close(gp[q], ogp[q]), (q, gp[q], ogp[q])
    assert _rel(gV, ogV) < RTOL
    # finite differences of the oracle's w on a few queries
    for q in range(4):
        fd = np.zeros(3)
        for k in range(3):
            hi, lo = P[q].copy(), P[q].copy()
            hi[k] = np.float32(hi[k] + 1e-3)
            lo[k] = np.float32(lo[k] - 1e-3)
            w2 = oracle.w3d_vos(m.V, m.F, np.stack([hi, lo]))
            fd[k] = (w2[0] - w2[1]) / (float(hi[k]) - float(lo[k]))
        assert _rel(gp[q] / gw[q], fd) < 5 * RTOL
    # only boundary vertices carry gradient
    off, vid = mesh.boundary()
    interior = np.setdiff1d(np.arange(len(m.V)), vid)
    assert np.all(gV[interior] == 0)


def test_autograd_function(gwn, ctx):
    import torch
    m = gen.icosphere_cap(subdiv=2, seed=4)
    mesh = gwn.Mesh(ctx, m.V, m.F)
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
    assert _rel(Pt.grad.cpu().numpy(), ogp) < RTOL
    assert _rel(Vt.grad.cpu().numpy(), ogV) < RTOL
    wo, _, _ = oracle.w3d_oneshot(m.V, m.F, P, m.d)
    assert np.abs(w.detach().cpu().numpy() - wo).max() < 1e-6


def test_torus_full_size_sampled(gwn, ctx):
    """The differentiation workload at full size: 2.1M-triangle slit torus, 1M
    queries, forward + backward; sampled queries checked against the oracle."""
    import torch
    m = gen.slit_torus()
    mesh = gwn.Mesh(ctx, m.V, m.F)
    info = mesh.info()
    assert info["n_loops"] == 2 and info["n_boundary_edges"] == 2048
    Pt = torch.as_tensor(m.points).cuda()
    r = mesh.eval(gwn.Points(Pt), m.d, want_chi=True)
    gw = torch.ones(len(Pt), device="cuda")
    gp, gV = mesh.backward(Pt, gw)
    torch.cuda.synchronize()
    ctx.check()
    rng = np.random.default_rng(8)
    idx = np.sort(rng.choice(len(Pt), 24, replace=False))
    P = m.points[idx]
    wo, chio, _ = oracle.w3d_oneshot(m.V, m.F, P, m.d)
    assert np.array_equal(r["chi"].cpu().numpy()[idx], chio)
    assert np.abs(r["w"].cpu().numpy()[idx] - wo).max() <= 1e-6
    ogp, _ = oracle.grad3d_vos(m.V, m.F, P, want_V=False)
    g = gp.cpu().numpy()[idx].astype(np.float64)
    for q in range(len(idx)):
        assert _close(g[q], ogp[q]), (q, g[q], ogp[q])
    # translation invariance of the summed gradients: sum_q dw/dp = -sum_v dw/dV
    s_p = gp.double().sum(0).cpu().numpy()
    s_v = gV.double().sum(0).cpu().numpy()
    assert _rel(s_p, -s_v) < 1e-3
