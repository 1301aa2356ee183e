"""Pins for the oracle's distance functions, which decide the queries every
parity test excludes (w is undefined on the geometry, Background; the bar
applies beyond 1e-4 x bbox diagonal).

3D (``oracle.dist3d``, closest point by the Voronoi regions of a triangle):
hand-computed distances for a point in every region of one triangle (three
vertices, three edges, the face from both sides), each case repeated under all
six vertex orders so that every branch of the region test is taken; a needle
triangle; random triangles against an independent decomposition (distance to
the plane when the projection falls inside, else the nearest of the three
edge segments).

2D (``oracle.dist2d``, dense sampling plus golden-section refinement): a
straight cubic against the point-segment distance; a 16-segment cubic circle
against | |p| - 1 | within the curve's measured radial deviation; random
chains bracketed by a brute-force sampling of the curve."""
import itertools
import math

import numpy as np

import oracle

PERMS = list(itertools.permutations(range(3)))


def _tri_dist(T, p):
    return float(oracle.dist3d(np.asarray(T, np.float32), np.array([[0, 1, 2]], np.int32),
                               np.asarray([p], np.float32))[0])


def _f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def test_triangle_voronoi_regions():
    T = np.array([[0, 0, 0], [2, 0, 0], [0, 1, 0]], np.float32)
    s5 = math.sqrt(5.0)
    cases = [
        # (point, closest point on the triangle) -- region named in the comment
        ((-1.0, -1.0, 0.5), (0, 0, 0)),                     # vertex (0,0,0)
        ((3.0, -1.0, 0.0), (2, 0, 0)),                      # vertex (2,0,0)
        ((-0.5, 2.0, 0.0), (0, 1, 0)),                      # vertex (0,1,0)
        ((1.0, -1.0, 0.5), (1, 0, 0)),                      # edge (0,0,0)-(2,0,0)
        ((-1.0, 0.5, -0.25), (0, 0.5, 0)),                  # edge (0,0,0)-(0,1,0)
        ((1 + 0.75 / s5, 0.5 + 1.5 / s5, 0.25), (1, 0.5, 0)),   # edge (2,0,0)-(0,1,0), outward in-plane normal
        ((0.5, 0.25, 0.75), (0.5, 0.25, 0)),                # face, above
        ((0.5, 0.25, -0.375), (0.5, 0.25, 0)),              # face, below
    ]
    for p, q in cases:
        want = float(np.linalg.norm(_f32(p) - np.asarray(q, np.float64)))
        for perm in PERMS:
            got = _tri_dist(T[list(perm)], p)
            assert abs(got - want) <= 1e-7 * max(1.0, want), (p, perm, got, want)


def test_needle_triangle():
    T = np.array([[0, 0, 0], [1, 0, 0], [0.5, 1e-7, 0]], np.float32)
    Td = T.astype(np.float64)
    cases = [
        ((0.5, 0.5, 0.0), Td[2]),                           # apex of the needle
        ((2.0, 0.0, 0.125), Td[1]),                         # beyond the tip
        ((0.25, -0.5, 0.0), (0.25, 0.0, 0.0)),              # the long edge, from below
    ]
    for p, q in cases:
        want = float(np.linalg.norm(_f32(p) - np.asarray(q, np.float64)))
        for perm in PERMS:
            assert abs(_tri_dist(T[list(perm)], p) - want) <= 1e-12 + 1e-9 * want


def _seg_dist(a, b, p):
    e = b - a
    t = np.clip(np.dot(p - a, e) / max(np.dot(e, e), 1e-300), 0.0, 1.0)
    return np.linalg.norm(a + t * e - p)


def _tri_dist_by_decomposition(a, b, c, p):
    n = np.cross(b - a, c - a)
    n2 = np.dot(n, n)
    best = min(_seg_dist(a, b, p), _seg_dist(b, c, p), _seg_dist(c, a, p))
    if n2 > 0:
        h = np.dot(p - a, n) / n2
        x = p - h * n                                   # projection on the plane
        # barycentric coordinates of x by signed areas
        l0 = np.dot(np.cross(b - x, c - x), n) / n2
        l1 = np.dot(np.cross(c - x, a - x), n) / n2
        l2 = 1.0 - l0 - l1
        if min(l0, l1, l2) >= 0:
            best = min(best, abs(h) * math.sqrt(n2))
    return best


def test_random_triangles_against_decomposition():
    rng = np.random.default_rng(5)
    for _ in range(300):
        T = rng.standard_normal((3, 3)).astype(np.float32)
        if rng.random() < 0.2:                              # thin ones too
            T[2] = (T[0] + (T[1] - T[0]) * rng.random() + 1e-3 * rng.standard_normal(3)).astype(np.float32)
        P = (1.5 * rng.standard_normal((8, 3))).astype(np.float32)
        got = oracle.dist3d(T, np.array([[0, 1, 2]], np.int32), P)
        Td = T.astype(np.float64)
        for p, g in zip(P.astype(np.float64), got):
            want = _tri_dist_by_decomposition(Td[0], Td[1], Td[2], p)
            assert abs(g - want) <= 1e-10 * max(1.0, want), (T.tolist(), p.tolist(), g, want)
    # a mesh: the minimum over its triangles
    V = rng.standard_normal((30, 3)).astype(np.float32)
    F = rng.integers(0, 30, (40, 3)).astype(np.int32)
    P = rng.standard_normal((20, 3)).astype(np.float32)
    got = oracle.dist3d(V, F, P)
    Vd = V.astype(np.float64)
    for p, g in zip(P.astype(np.float64), got):
        want = min(_tri_dist_by_decomposition(Vd[f[0]], Vd[f[1]], Vd[f[2]], p) for f in F)
        assert abs(g - want) <= 1e-10


def _bezier(ctrl4, u):
    u = np.asarray(u, np.float64)[:, None]
    B = np.concatenate([(1 - u) ** 3, 3 * u * (1 - u) ** 2, 3 * u ** 2 * (1 - u), u ** 3], 1)
    return B @ ctrl4


def test_straight_cubic_is_a_segment():
    rng = np.random.default_rng(2)
    for _ in range(40):
        s, e = rng.standard_normal((2, 2))
        ctrl = np.stack([s, s + (e - s) / 3, s + 2 * (e - s) / 3, e])
        P = 1.5 * rng.standard_normal((10, 2))
        got = oracle.dist2d(ctrl, P)
        for p, g in zip(P, got):
            assert abs(g - _seg_dist(s, e, p)) <= 1e-12


def test_cubic_circle():
    n = 16
    th = 2 * np.pi / n
    k = 4.0 / 3.0 * math.tan(th / 4)
    pts = [np.array([1.0, 0.0])]
    for i in range(n):
        a0, a1 = i * th, (i + 1) * th
        p0 = np.array([math.cos(a0), math.sin(a0)])
        p3 = np.array([math.cos(a1), math.sin(a1)])
        p1 = p0 + k * np.array([-math.sin(a0), math.cos(a0)])
        p2 = p3 - k * np.array([-math.sin(a1), math.cos(a1)])
        pts += [p1, p2, p3]
    ctrl = np.array(pts)
    # radial deviation of the cubic circle from the unit circle
    u = np.linspace(0, 1, 20001)
    dev = max(np.abs(np.linalg.norm(_bezier(ctrl[3 * i:3 * i + 4], u), axis=1) - 1).max() for i in range(n))
    assert dev < 1e-4
    rng = np.random.default_rng(3)
    r = np.concatenate([rng.uniform(0.0, 0.95, 100), rng.uniform(1.05, 3.0, 100), 1 + rng.uniform(-1e-3, 1e-3, 50)])
    a = rng.uniform(0, 2 * np.pi, len(r))
    P = np.stack([r * np.cos(a), r * np.sin(a)], 1)
    got = oracle.dist2d(ctrl, P)
    assert np.all(np.abs(got - np.abs(r - 1)) <= dev + 1e-12)


def test_random_chains_bracketed_by_sampling():
    rng = np.random.default_rng(4)
    for _ in range(10):
        nseg = int(rng.integers(1, 6))
        ctrl = rng.standard_normal((3 * nseg + 1, 2))
        P = 1.5 * rng.standard_normal((30, 2))
        got = oracle.dist2d(ctrl, P)
        u = np.linspace(0, 1, 40001)
        X = np.concatenate([_bezier(ctrl[3 * i:3 * i + 4], u) for i in range(nseg)])
        gap = max(np.linalg.norm(np.diff(_bezier(ctrl[3 * i:3 * i + 4], u), axis=0), axis=1).max()
                  for i in range(nseg))
        for p, g in zip(P, got):
            ds = np.linalg.norm(X - p, axis=1).min()
            assert ds - gap / 2 - 1e-12 <= g <= ds + 1e-12, (g, ds, gap)
