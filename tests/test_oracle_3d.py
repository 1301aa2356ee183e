"""Pins for the 3D oracle: closed forms, invariants and brute force.

Nothing here compares the oracle with itself: every expected value is a
closed form (tests/golden/closed_forms.json), a mathematical invariant, or a
second, independent method (the per-triangle solid-angle sum versus the
one-shot crossing count + boundary term).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import gen
import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))
DIRS = [gen.random_direction(s) for s in (11, 12, 13)]


def _cube():
    V = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], np.float32)
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    F = []
    for a, b, c, d in quads:
        F += [(a, b, c), (a, c, d)]
    F = np.array(F, np.int32)
    # orient outward
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    flip = np.einsum("ij,ij->i", n, V[F].mean(1)) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


def test_octant_triangle_is_one_eighth():
    g = GOLD["octant_triangle"]
    V = np.array(g["vertices"], np.float32)
    F = np.array(g["faces"], np.int32)
    P = np.array([g["query"]], np.float32)
    assert abs(oracle.w3d_vos(V, F, P)[0] - g["w"]) < 1e-15
    for d in DIRS:
        w, chi, B = oracle.w3d_oneshot(V, F, P, d)
        assert abs(w[0] - g["w"]) < 1e-14


def test_cube_faces_and_closed_cube():
    V, F = _cube()
    centre = np.zeros((1, 3), np.float32)
    for f in range(6):
        w = oracle.w3d_vos(V, F[2 * f:2 * f + 2], centre)[0]
        assert abs(w - GOLD["cube_face_from_centre"]["w_per_face"]) < 1e-14
    rng = np.random.default_rng(0)
    inside = rng.uniform(-0.9, 0.9, (200, 3)).astype(np.float32)
    outside = rng.uniform(-3, 3, (2000, 3)).astype(np.float32)
    outside = outside[np.abs(outside).max(1) > 1.1][:200]
    for d in DIRS:
        w, chi, B = oracle.w3d_oneshot(V, F, inside, d)
        assert np.all(chi == 1) and np.abs(B).max() < 1e-15 and np.abs(w - 1).max() < 1e-15
        w, chi, B = oracle.w3d_oneshot(V, F, outside, d)
        assert np.all(chi == 0) and np.abs(w).max() < 1e-15
    assert np.abs(oracle.w3d_vos(V, F, inside) - 1).max() < 1e-13
    assert np.abs(oracle.w3d_vos(V, F, outside)).max() < 1e-13


def test_closed_icosphere_integer_and_no_boundary():
    V, F = gen.icosphere(3)
    V = V.astype(np.float32)
    F = F.astype(np.int32)
    src, dst, m = oracle.boundary_edges(F)
    assert len(src) == 0
    rng = np.random.default_rng(1)
    P = rng.uniform(-1.5, 1.5, (400, 3)).astype(np.float32)
    r = np.linalg.norm(P, axis=1)
    P = P[(r < 0.9) | (r > 1.1)]
    r = np.linalg.norm(P, axis=1)
    for d in DIRS:
        w, chi, B = oracle.w3d_oneshot(V, F, P, d)
        assert np.all(B == 0)
        assert np.all(chi == (r < 1).astype(np.int32))
    wv = oracle.w3d_vos(V, F, P)
    assert np.abs(wv - (r < 1)).max() < 1e-12


def _hemisphere(n_ring=24, n_lat=8):
    """Triangulated upper hemisphere whose rim (equator) lies exactly in z = 0;
    normals point away from the centre."""
    V = [[0.0, 0.0, 1.0]]
    for k in range(1, n_lat + 1):
        th = 0.5 * math.pi * k / n_lat
        for j in range(n_ring):
            ph = 2 * math.pi * (j + 0.5 * (k % 2)) / n_ring
            z = 0.0 if k == n_lat else math.cos(th)
            V.append([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), z])
    V = np.array(V, np.float32)
    F = []
    for j in range(n_ring):
        F.append((0, 1 + j, 1 + (j + 1) % n_ring))
    for k in range(1, n_lat):
        a0 = 1 + (k - 1) * n_ring
        b0 = 1 + k * n_ring
        for j in range(n_ring):
            j1 = (j + 1) % n_ring
            F.append((a0 + j, b0 + j, b0 + j1))
            F.append((a0 + j, b0 + j1, a0 + j1))
    F = np.array(F, np.int32)
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    flip = np.einsum("ij,ij->i", n, V[F].mean(1)) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


def test_hemisphere_from_centre_is_half():
    V, F = _hemisphere()
    P = np.zeros((1, 3), np.float32)
    # normals point away from the centre: the centre is behind -> +1/2
    assert abs(oracle.w3d_vos(V, F, P)[0] - 0.5) < 1e-14
    for d in DIRS:
        w, chi, B = oracle.w3d_oneshot(V, F, P, d)
        assert abs(w[0] - 0.5) < 1e-14
    # reversed orientation -> -1/2
    assert abs(oracle.w3d_vos(V, F[:, [0, 2, 1]], P)[0] + 0.5) < 1e-14


@pytest.mark.parametrize("n", [3, 5, 17])
def test_regular_ngon_on_axis(n):
    R = 1.0
    ang = 2 * np.pi * np.arange(n) / n
    V = np.concatenate([[[0, 0, 0]], np.stack([R * np.cos(ang), R * np.sin(ang), 0 * ang], 1)]).astype(np.float32)
    F = np.array([(0, 1 + j, 1 + (j + 1) % n) for j in range(n)], np.int32)  # normal +z
    Vd = V.astype(np.float64)
    for h in (2.0, 0.5, 0.05, 1e-3):
        P = np.array([[0, 0, -h]], np.float32)
        hh = -float(P[0, 2])
        # actual float32 vertex radius of the polygon
        Rv = float(np.hypot(Vd[1, 0], Vd[1, 1]))
        alpha = math.atan2(Rv, hh)
        area = 2 * math.pi - 2 * n * math.atan(math.tan(math.pi / n) * math.cos(alpha))
        expect = area / (4 * math.pi)      # below the polygon = behind its +z normal
        got = oracle.w3d_vos(V, F, P)[0]
        # the float32 ring vertices are not exactly co-circular: allow 1e-7
        assert abs(got - expect) < 1e-7, (n, h, got, expect)
        for d in DIRS:
            w, chi, B = oracle.w3d_oneshot(V, F, P, d)
            assert abs(w[0] - got) < 1e-13


def test_jump_of_one_across_the_surface():
    m = gen.icosphere_cap(subdiv=3)
    V = m.V.astype(np.float64)
    rng = np.random.default_rng(3)
    for t in rng.choice(len(m.F), 20, replace=False):
        a, b, c = V[m.F[t]]
        n = np.cross(b - a, c - a)
        n /= np.linalg.norm(n)
        cen = (a + b + c) / 3
        eps = 1e-4
        P = np.array([cen - eps * n, cen + eps * n], np.float32)
        wv = oracle.w3d_vos(m.V, m.F, P)
        assert abs((wv[0] - wv[1]) - GOLD["jump_across_surface"]["w_behind_minus_w_front"]) < 1e-3
        w, chi, B = oracle.w3d_oneshot(m.V, m.F, P, m.d)
        assert abs((w[0] - w[1]) - 1.0) < 1e-3
        assert np.abs(w - wv).max() < 1e-11


def test_oneshot_matches_definition_on_soups():
    """Per-triangle identity: the solid-angle sum equals crossings + boundary
    term for arbitrary soups (non-manifold, inconsistently oriented)."""
    rng = np.random.default_rng(5)
    for trial in range(4):
        nv = 40
        V = rng.standard_normal((nv, 3)).astype(np.float32)
        F = rng.integers(0, nv, (60, 3)).astype(np.int32)
        F = F[(F[:, 0] != F[:, 1]) & (F[:, 1] != F[:, 2]) & (F[:, 0] != F[:, 2])]
        F = np.concatenate([F, F[:5]])       # duplicated faces -> multiplicity 2 edges
        P = (2.5 * rng.standard_normal((1500, 3))).astype(np.float32)
        dist = oracle.dist3d(V, F, P)
        P = P[dist > 1e-3]
        wv = oracle.w3d_vos(V, F, P)
        for d in DIRS[:2]:
            w, chi, B = oracle.w3d_oneshot(V, F, P, d)
            assert np.abs(w - wv).max() < 1e-11


def test_d_independence():
    m = gen.icosphere_cap(subdiv=3)
    P = gen.grid_points(gen.Grid((-1.2,) * 3, (1.2,) * 3, (11, 11, 11)))
    dist = oracle.dist3d(m.V, m.F, P)
    P = P[dist > 1e-3]
    ws, chis = [], []
    for d in DIRS:
        w, chi, B = oracle.w3d_oneshot(m.V, m.F, P, d)
        ws.append(w)
        chis.append(chi)
    assert np.abs(ws[0] - ws[1]).max() < 1e-12 and np.abs(ws[0] - ws[2]).max() < 1e-12
    assert np.any(chis[0] != chis[1]) or np.any(chis[0] != chis[2])


def test_continuity_across_the_ray_shadow_of_a_boundary_edge():
    """Where the ray p + t d crosses a boundary edge, chi and B jump by one in
    opposite directions; w stays continuous."""
    m = gen.icosphere_cap(subdiv=3)
    src, dst, mult = oracle.boundary_edges(m.F)
    d = m.d.astype(np.float64)
    V = m.V.astype(np.float64)
    jumps = 0
    for e in range(0, len(src), 3):
        A, Bv = V[src[e]], V[dst[e]]
        mid = 0.5 * (A + Bv)
        side = np.cross(Bv - A, d)
        side /= np.linalg.norm(side)
        base = mid - 0.7 * d
        P = np.array([base - 1e-5 * side, base + 1e-5 * side], np.float32)
        w, chi, B = oracle.w3d_oneshot(m.V, m.F, P, m.d)
        wv = oracle.w3d_vos(m.V, m.F, P)
        jumps += int(chi[0] != chi[1])
        assert abs(w[0] - w[1]) < 1e-4
        assert np.abs(w - wv).max() < 1e-11
    assert jumps > 0


def test_cap_boundary_is_one_loop_of_unit_edges():
    m = gen.icosphere_cap(subdiv=6)
    src, dst, mult = oracle.boundary_edges(m.F)
    assert np.all(mult == 1)
    # every boundary vertex has in-degree == out-degree == 1 -> disjoint cycles
    assert sorted(src.tolist()) == sorted(dst.tolist())
    assert len(set(src.tolist())) == len(src)
    nxt = dict(zip(src.tolist(), dst.tolist()))
    v0 = int(src[0])
    v, n = v0, 0
    while True:
        v = nxt[v]
        n += 1
        if v == v0:
            break
    assert n == len(src)        # one loop
    assert len(src) == 252


# ---------------------------------------------------------------------------
# predicates against Python rational arithmetic
# ---------------------------------------------------------------------------
def _fr(x):
    return Fraction(float(np.float32(x)))


def _det3_exact(r0, r1, r2):
    return (r0[0] * (r1[1] * r2[2] - r1[2] * r2[1]) - r0[1] * (r1[0] * r2[2] - r1[2] * r2[0])
            + r0[2] * (r1[0] * r2[1] - r1[1] * r2[0]))


def _sgn(x):
    return (x > 0) - (x < 0)


def test_predicates_match_rational_arithmetic():
    rng = np.random.default_rng(7)
    n_zero = 0
    for trial in range(400):
        kind = trial % 4
        A = rng.standard_normal(3).astype(np.float32)
        B = rng.standard_normal(3).astype(np.float32)
        D = rng.standard_normal(3).astype(np.float32)
        if kind == 0:
            P = rng.standard_normal(3).astype(np.float32)
        elif kind == 1:      # P nearly on the plane through A, B spanned with D
            t = rng.uniform(-2, 2)
            P = (A + t * (B - A) + rng.uniform(-1, 1) * D.astype(np.float64)).astype(np.float32)
        elif kind == 2:      # small integers: exact zeros are common
            A = rng.integers(-3, 4, 3).astype(np.float32)
            B = rng.integers(-3, 4, 3).astype(np.float32)
            D = rng.integers(-3, 4, 3).astype(np.float32)
            P = rng.integers(-3, 4, 3).astype(np.float32)
        else:                # wide exponent range
            s = np.float32(2.0) ** rng.integers(-40, 40, 3).astype(np.float32)
            P = (rng.standard_normal(3) * s).astype(np.float32)
        a = [_fr(A[i]) - _fr(P[i]) for i in range(3)]
        b = [_fr(B[i]) - _fr(P[i]) for i in range(3)]
        dd = [_fr(D[i]) for i in range(3)]
        exact = _sgn(_det3_exact(a, b, dd))
        n_zero += exact == 0
        assert oracle.exact_det_abd(A, B, P, D) == exact
        cross = [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]
        sos = exact
        for k in range(3):
            if sos == 0:
                sos = _sgn(cross[k])
        assert oracle.sign_edge(A, B, P, D) == sos
        C = rng.standard_normal(3).astype(np.float32) if kind != 2 else rng.integers(-3, 4, 3).astype(np.float32)
        c = [_fr(C[i]) - _fr(P[i]) for i in range(3)]
        o = _sgn(_det3_exact(a, b, c))
        assert oracle.exact_orient(A, B, C, P) == o
        assert oracle.sign_orient(A, B, C, P) == o
    assert n_zero > 5


def test_triangle_crossing_brute_force_by_sampling():
    """Eq. chi on one triangle: the exact crossing decision agrees with a
    direct float64 ray/plane intersection on well-separated cases."""
    rng = np.random.default_rng(9)
    agree = 0
    for _ in range(3000):
        v = rng.standard_normal((3, 3)).astype(np.float32)
        p = rng.standard_normal(3).astype(np.float32)
        d = rng.standard_normal(3).astype(np.float32)
        v64, p64, d64 = v.astype(np.float64), p.astype(np.float64), d.astype(np.float64)
        n = np.cross(v64[1] - v64[0], v64[2] - v64[0])
        nd = n @ d64
        if abs(nd) < 1e-3:
            continue
        t = n @ (v64[0] - p64) / nd
        x = p64 + t * d64
        # barycentric
        def area(a, b, c):
            return np.cross(b - a, c - a) @ n
        l0, l1, l2 = area(x, v64[1], v64[2]), area(v64[0], x, v64[2]), area(v64[0], v64[1], x)
        tot = l0 + l1 + l2
        l0, l1, l2 = l0 / tot, l1 / tot, l2 / tot
        if min(abs(l0), abs(l1), abs(l2)) < 1e-6 or abs(t) < 1e-6:
            continue
        inside = l0 > 0 and l1 > 0 and l2 > 0 and t > 0
        expect = int(np.sign(nd)) if inside else 0
        assert oracle.tri_crossing(v[0], v[1], v[2], p, d) == expect
        agree += 1
    assert agree > 2000


# ---------------------------------------------------------------------------
# gradient
# ---------------------------------------------------------------------------
def _biot_savart(Vd, edges, p):
    """Gradient of w at p from the boundary alone (line integral of the
    Biot-Savart kernel over each straight edge)."""
    src, dst, m = edges
    g = np.zeros(3)
    for s, t, k in zip(src, dst, m):
        a = Vd[s] - p
        b = Vd[t] - p
        E = b - a
        axb = np.cross(a, b)
        g += k * axb / (axb @ axb) * (E @ b / np.linalg.norm(b) - E @ a / np.linalg.norm(a))
    return g / (4 * np.pi)


def test_gradient_against_fd_biot_savart_and_invariants():
    m = gen.icosphere_cap(subdiv=2)
    rng = np.random.default_rng(4)
    P = rng.uniform(-1.3, 1.3, (40, 3)).astype(np.float32)
    P = P[oracle.dist3d(m.V, m.F, P) > 0.05][:12]
    gp, gV = oracle.grad3d_vos(m.V, m.F, P)
    edges = oracle.boundary_edges(m.F)
    Vd = m.V.astype(np.float64)
    for q in range(len(P)):
        p = P[q].astype(np.float64)
        # central differences on float32 inputs: use the actually representable step
        fd = np.zeros(3)
        for k in range(3):
            hi = P[q].copy()
            lo = P[q].copy()
            hi[k] = np.float32(hi[k] + 1e-3)
            lo[k] = np.float32(lo[k] - 1e-3)
            w2 = oracle.w3d_vos(m.V, m.F, np.stack([hi, lo]))
            fd[k] = (w2[0] - w2[1]) / (float(hi[k]) - float(lo[k]))
        assert np.allclose(gp[q], fd, rtol=2e-4, atol=2e-5), (gp[q], fd)
        bs = _biot_savart(Vd, edges, p)
        assert np.allclose(gp[q], bs, rtol=1e-9, atol=1e-11), (gp[q], bs)
    # translation invariance: dw/dp = - sum over vertices of dw/dv
    gp1, gV1 = oracle.grad3d_vos(m.V, m.F, P[:1])
    assert np.allclose(gp1[0], -gV1.sum(0), atol=1e-12)
    # interior vertices do not influence w
    bverts = np.unique(np.concatenate([edges[0], edges[1]]))
    interior = np.setdiff1d(np.unique(m.F), bverts)
    assert np.abs(gV1[interior]).max() < 1e-10
    assert np.abs(gV1[bverts]).max() > 1e-4


def _grid_plate():
    V = np.array([[x, y, 0.0] for x in range(4) for y in range(4)], np.float32)
    F = []
    for i in range(3):
        for j in range(3):
            a, b, c, dd = 4 * i + j, 4 * (i + 1) + j, 4 * (i + 1) + j + 1, 4 * i + j + 1
            F += [(a, b, c), (a, c, dd)]
    return V, np.array(F, np.int32)


def test_rays_exactly_through_boundary_vertices():
    """Axis-aligned directions on grid-aligned data: rays pass exactly through
    boundary vertices and along edge lines.  The one-shot value (crossing count
    under the perturbed direction + boundary term as the limit under the same
    perturbation) must equal the per-triangle definition."""
    V, F = _grid_plate()
    g = np.arange(-1, 5, 0.5, dtype=np.float32)
    P = np.array([[x, y, z] for x in g for y in g for z in (-1.0, -0.5, 0.5, 1.0)], np.float32)
    wv = oracle.w3d_vos(V, F, P)
    for d in ([0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1, 1], [1, 1, 0], [0, 0, 3]):
        w, chi, B = oracle.w3d_oneshot(V, F, P, np.array(d, np.float32))
        assert np.abs(w - wv).max() < 1e-12, d


# ---- Algorithm 1 in 3D by a spherical arrangement (third evaluation) --------

def test_alg1_closed_forms():
    """Algorithm 1 (arrangement, one ray, propagation across the arcs,
    area-weighted sum) reproduces the closed forms: the octant triangle seen
    from the origin (1/8; its image splits the sphere into two regions), the
    hemisphere seen from just off its centre (equal to the definition, both
    orientations) and a closed mesh (integer, one region)."""
    V = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float32)
    F = np.array([[0, 1, 2]], np.int32)
    w, info = oracle.w3d_alg1(V, F, np.zeros((1, 3), np.float32))
    assert abs(w[0] - 0.125) < 1e-14 and info[0, 0] == 2
    assert abs(info[0, 1] - 3.5 * math.pi) < 1e-12          # largest region: 4 pi - pi / 2
    Vh, Fh = _hemisphere(n_ring=24, n_lat=6)
    P0 = np.zeros((1, 3), np.float32)
    # from the centre itself the rim's arcs would share one great circle (a
    # degenerate arrangement); just above it they lie on a small circle
    w, info = oracle.w3d_alg1(Vh, Fh, P0 + np.float32([0, 0, 1e-3]))
    assert abs(w[0] - oracle.w3d_vos(Vh, Fh, P0 + np.float32([0, 0, 1e-3]))[0]) < 1e-12
    w, _ = oracle.w3d_alg1(Vh, Fh[:, [0, 2, 1]], P0 + np.float32([0, 0, -1e-3]))
    assert abs(w[0] - oracle.w3d_vos(Vh, Fh[:, [0, 2, 1]], P0 + np.float32([0, 0, -1e-3]))[0]) < 1e-12
    Vs, Fs = gen.icosphere(2)
    w, info = oracle.w3d_alg1(Vs, Fs, np.array([[0.1, -0.2, 0.05], [1.7, 0.3, 0.2]], np.float32))
    assert np.array_equal(w, [1.0, 0.0]) and np.all(info[:, 0] == 1)


def test_alg1_matches_definition_on_soups_and_meshes():
    """On random soups (several loops joined by zero-weight bridges,
    self-crossing projections, multiplicity-2 edges, non-manifold edges) and on
    the capped icosphere (one loop of 252 arcs), the arrangement evaluation
    equals the per-triangle solid-angle sum and the closed form chi + B."""
    rng = np.random.default_rng(11)
    for trial in range(3):
        nv = 14
        V = rng.standard_normal((nv, 3)).astype(np.float32)
        F = rng.integers(0, nv, (10, 3)).astype(np.int32)
        F = F[(F[:, 0] != F[:, 1]) & (F[:, 1] != F[:, 2]) & (F[:, 0] != F[:, 2])]
        F = np.concatenate([F, F[:2]])
        P = (1.5 * rng.standard_normal((40, 3))).astype(np.float32)
        P = P[oracle.dist3d(V, F, P) > 1e-3][:12]
        wa, info = oracle.w3d_alg1(V, F, P)
        wv = oracle.w3d_vos(V, F, P)
        wo, _, _ = oracle.w3d_oneshot(V, F, P, DIRS[0])
        assert np.abs(wa - wv).max() < 1e-11, trial
        assert np.abs(wa - wo).max() < 1e-11, trial
        assert info[:, 0].max() > 4                # a real arrangement, not one split
    m = gen.icosphere_cap(subdiv=2)
    P = np.array([[0.0, 0.0, 0.2], [0.3, -0.2, 1.3], [0.9, 0.9, 0.1], [0.05, 0.02, -1.6]], np.float32)
    wa, info = oracle.w3d_alg1(m.V, m.F, P)
    wv = oracle.w3d_vos(m.V, m.F, P)
    assert np.abs(wa - wv).max() < 1e-11


# ---- parametric surfaces: bicubic Bezier patches ----------------------------

def test_patch_quadrature_closed_forms():
    """The patch definition (adaptive quadrature of (f - p).(f_u x f_v) /
    |f - p|^3) against closed forms: a flat square patch (control points on a
    uniform grid, so f is the square itself, normal +z) seen from its axis,
    Omega = 4 atan(a^2 / (h sqrt(2 a^2 + h^2))) (below the square: behind its
    normal, +); a closed surface of patches gives 0 or 1."""
    a = 0.7
    s = np.linspace(-a, a, 4)
    ctrl = np.zeros((1, 4, 4, 3), np.float32)
    for i in range(4):
        for j in range(4):
            ctrl[0, i, j] = (s[i], s[j], 0.0)
    for h in (2.0, 0.4, 0.05):
        P = np.array([[0.0, 0.0, -h]], np.float32)
        hh = -float(P[0, 2])
        aa = float(np.float32(a))
        expect = 4 * math.atan(aa * aa / (hh * math.sqrt(2 * aa * aa + hh * hh))) / (4 * math.pi)
        assert abs(oracle.w3d_patches_quad(ctrl, P)[0] - expect) < 1e-12
        assert abs(oracle.w3d_patches_quad(ctrl, -P)[0] + expect) < 1e-12
    pc = gen.patch_spheroid(n=2, amp=0.1, seed=3)
    P = np.array([[0, 0, 0], [0.2, -0.3, 0.1], [1.5, 0.2, 0.0], [0.0, -1.4, 0.3]], np.float32)
    w = oracle.w3d_patches_quad(pc.ctrl, P)
    assert np.abs(w - np.array([1, 1, 0, 0])).max() < 1e-12
    V, E = oracle.patch_boundary(pc.ctrl, 8)
    assert len(E[0]) == 0


def test_patch_boundary_sampling_converges():
    """With one cube face left out, the definition minus the FP64 boundary term
    on the sampled boundary curves tends to an integer (the crossing count) at
    the rate of the polyline's sagitta, O(K^-2)."""
    po = gen.patch_spheroid(n=2, amp=0.08, open_faces=(4,), seed=0)
    P = np.array([[0.3, -0.2, 0.1], [1.5, 0, 0], [0.2, 0.1, 1.25], [-0.9, 0.9, 0.9], [0.1, 0.2, -0.3]], np.float32)
    w = oracle.w3d_patches_quad(po.ctrl, P)
    errs = []
    for K in (32, 128, 512):
        V, E = oracle.patch_boundary(po.ctrl, K)
        assert len(E[0]) == 4 * 2 * K                 # one loop of the 8 edge curves around the hole
        r = w - oracle.bterm3d(V, E, P, po.d)
        errs.append(np.abs(r - np.rint(r)).max())
    assert errs[2] < 1e-6 and errs[0] / errs[1] > 10 and errs[1] / errs[2] > 10
