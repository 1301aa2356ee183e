"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds geometry and query generators only: it contains none of the
winding-number arithmetic (no boundary extraction, no solid angles, no ray
tests), so that both sides can consume the same bits without sharing method
code.  Every generator is deterministic in its ``seed``.

Workloads (the paper's experiments, Sec. "Validation and Results", are the
model for shapes and sizes; its datasets are not available, so these stand in):

* ``bezier_circle_chain``  one open C0 chain of cubic Beziers whose control
  points lie on a noisy unit circle (2D grid experiment, Sec. 2D Parametric
  Geometry).
* ``icosphere_cap``        icosphere with a removed polar cap: a mesh with few
  boundary edges and many faces (mesh timing table).
* ``star_chains``          many open chains of uneven length sampled from noisy
  star-shaped curves, each with its own regular grid (N=1000 random curves).
* ``slit_torus``           torus cut along one meridian: a two-loop boundary.
* ``holey_heightfield``    large heightfield disk with circular holes.
* ``patch_spheroid``       closed (or opened) surface of bicubic Bezier patches
  over the six faces of a cube, pushed onto a wavy sphere (parametric
  surfaces, Sec. "Parametric Surfaces").

Grid coordinates follow one rule everywhere: coordinate ``i`` of an axis with
``n`` samples on ``[lo, hi]`` is ``lo + i * ((hi - lo) / (n - 1))`` evaluated
in float64, then rounded to the working precision.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "grid_axis", "grid_points", "random_direction", "icosphere",
    "icosphere_cap", "slit_torus", "holey_heightfield", "bezier_circle_chain",
    "star_chains", "patch_spheroid", "Mesh", "Grid", "Chains", "Patches", "config",
]


# ----------------------------------------------------------------------------
# containers
# ----------------------------------------------------------------------------
@dataclass
class Grid:
    """Regular query grid: ``dims[k]`` samples on ``[lo[k], hi[k]]``.

    Flattened order: x fastest, then y, then z.
    """
    lo: tuple
    hi: tuple
    dims: tuple

    @property
    def n(self) -> int:
        return int(np.prod(self.dims))


@dataclass
class Mesh:
    V: np.ndarray            # float32 [nv, 3]
    F: np.ndarray            # int32 [nf, 3], counter-clockwise = +normal
    d: np.ndarray            # float32 [3] ray direction (unit up to rounding)
    grid: Grid | None = None
    points: np.ndarray | None = None   # float32 [nq, 3] when not a grid
    meta: dict = field(default_factory=dict)


@dataclass
class Chains:
    """Open C0 cubic Bezier chains: chain c owns ctrl[off[c]:off[c+1]]
    (3k+1 control points for k segments)."""
    ctrl: np.ndarray         # float32 or float64 [n_ctrl, 2]
    offsets: np.ndarray      # int64 [n_chains + 1]
    grids: list              # one Grid per chain
    meta: dict = field(default_factory=dict)


@dataclass
class Patches:
    """Bicubic Bezier patches: ctrl[t, i, j] is control point P_ij of patch t
    (i along u, j along v); the normal is f_u x f_v."""
    ctrl: np.ndarray         # float32 [n_patches, 4, 4, 3]
    d: np.ndarray            # float32 [3] ray direction
    grid: Grid | None = None
    meta: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------
# grids and directions
# ----------------------------------------------------------------------------
def grid_axis(lo: float, hi: float, n: int, dtype=np.float32) -> np.ndarray:
    """Inclusive linspace by the module's fixed rule, rounded to ``dtype``."""
    lo = float(lo)
    hi = float(hi)
    if n == 1:
        return np.array([lo], dtype=np.float64).astype(dtype)
    i = np.arange(n, dtype=np.float64)
    step = (hi - lo) / float(n - 1)
    return (lo + i * step).astype(dtype)


def grid_points(g: Grid, dtype=np.float32, index: np.ndarray | None = None) -> np.ndarray:
    """Explicit coordinates of grid points (all, or the flat ``index`` subset)."""
    axes = [grid_axis(g.lo[k], g.hi[k], g.dims[k], dtype) for k in range(len(g.dims))]
    if index is None:
        index = np.arange(g.n, dtype=np.int64)
    index = np.asarray(index, dtype=np.int64)
    out = np.empty((index.size, len(g.dims)), dtype=dtype)
    rem = index.copy()
    for k in range(len(g.dims)):
        out[:, k] = axes[k][rem % g.dims[k]]
        rem //= g.dims[k]
    return out


def random_direction(seed: int) -> np.ndarray:
    """Unit direction from N(0, I3), normalised in float64, rounded to float32."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(3)
    v /= np.linalg.norm(v)
    return v.astype(np.float32)


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------
def _orient_outward(V: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Flip faces of a star-shaped closed surface so normals point away from 0."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", n, a + b + c) < 0
    F = F.copy()
    F[flip] = F[flip][:, [0, 2, 1]]
    return F


def icosphere(subdiv: int):
    """Unit icosphere (float64 vertices, outward counter-clockwise faces)."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    V = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    F = _orient_outward(V, F)
    for _ in range(subdiv):
        e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
        e.sort(axis=1)
        key = e[:, 0] * (len(V) + 1) + e[:, 1]
        uniq, inv = np.unique(key, return_inverse=True)
        ua = uniq // (len(V) + 1)
        ub = uniq % (len(V) + 1)
        mid = V[ua] + V[ub]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        base = len(V)
        V = np.concatenate([V, mid])
        nf = len(F)
        m01 = base + inv[:nf]
        m12 = base + inv[nf:2 * nf]
        m20 = base + inv[2 * nf:]
        a, b, c = F[:, 0], F[:, 1], F[:, 2]
        F = np.concatenate([
            np.stack([a, m01, m20], 1), np.stack([b, m12, m01], 1),
            np.stack([c, m20, m12], 1), np.stack([m01, m12, m20], 1)])
    return V, F


def _compact(V: np.ndarray, F: np.ndarray):
    used = np.unique(F)
    remap = -np.ones(len(V), dtype=np.int64)
    remap[used] = np.arange(len(used))
    return V[used], remap[F]


def icosphere_cap(subdiv: int = 6, cap_z: float = 0.8, sigma: float = 1e-3,
                  grid_n: int = 256, extent: float = 1.2, seed: int = 0) -> Mesh:
    """Icosphere with the triangles whose (noise-free) centroid has z > cap_z
    removed, then Gaussian vertex noise of std ``sigma``; 256^3 grid on
    [-1.2, 1.2]^3 and a random unit direction."""
    V, F = icosphere(subdiv)
    cz = V[F].mean(axis=1)[:, 2]
    F = F[cz <= cap_z]
    V, F = _compact(V, F)
    rng = np.random.default_rng(seed)
    V = V + sigma * rng.standard_normal(V.shape)
    g = Grid((-extent,) * 3, (extent,) * 3, (grid_n,) * 3)
    return Mesh(V.astype(np.float32), F.astype(np.int32), random_direction(seed + 1), grid=g,
                meta=dict(name="icosphere_cap", subdiv=subdiv, cap_z=cap_z, sigma=sigma, seed=seed))


def slit_torus(n_u: int = 1024, n_v: int = 1024, R: float = 1.0, r: float = 0.35,
               sigma: float = 1e-3, n_queries: int = 1 << 20, min_dist: float = 1e-3,
               seed: int = 0) -> Mesh:
    """Torus on an n_u x n_v vertex grid with the quad column between major
    index n_u-1 and 0 removed, so the boundary is two distinct meridian loops.
    Queries: uniform in the padded bbox, rejected when closer than
    ``min_dist`` + the largest noise displacement to the ideal torus."""
    rng = np.random.default_rng(seed)
    u = 2 * np.pi * np.arange(n_u) / n_u
    v = 2 * np.pi * np.arange(n_v) / n_v
    U, Vv = np.meshgrid(u, v, indexing="ij")
    X = np.stack([(R + r * np.cos(Vv)) * np.cos(U), (R + r * np.cos(Vv)) * np.sin(U),
                  r * np.sin(Vv)], -1).reshape(-1, 3)
    noise = sigma * rng.standard_normal(X.shape)
    X = X + noise
    idx = np.arange(n_u * n_v).reshape(n_u, n_v)
    i = np.arange(n_u - 1)[:, None]
    j = np.arange(n_v)[None, :]
    a = idx[i, j]
    b = idx[i + 1, j]
    c = idx[i + 1, (j + 1) % n_v]
    dd = idx[i, (j + 1) % n_v]
    F = np.concatenate([np.stack([a, b, c], -1).reshape(-1, 3),
                        np.stack([a, c, dd], -1).reshape(-1, 3)])
    # outward orientation check on the noise-free torus
    P = X - noise
    n = np.cross(P[F[:, 1]] - P[F[:, 0]], P[F[:, 2]] - P[F[:, 0]])
    cen = P[F].mean(1)
    rho = np.hypot(cen[:, 0], cen[:, 1])
    ring = np.stack([R * cen[:, 0] / rho, R * cen[:, 1] / rho, np.zeros_like(rho)], -1)
    if np.einsum("ij,ij->i", n, cen - ring).mean() < 0:
        F = F[:, [0, 2, 1]]
    margin = min_dist + float(np.abs(noise).max()) * math.sqrt(3.0)
    lo = np.array([-(R + r), -(R + r), -r]) - 0.05
    hi = -lo
    pts = []
    have = 0
    while have < n_queries:
        cand = lo + (hi - lo) * rng.random((n_queries, 3))
        rr = np.hypot(np.hypot(cand[:, 0], cand[:, 1]) - R, cand[:, 2])
        keep = cand[np.abs(rr - r) > margin]
        pts.append(keep)
        have += len(keep)
    Q = np.concatenate(pts)[:n_queries].astype(np.float32)
    return Mesh(X.astype(np.float32), F.astype(np.int32), random_direction(seed + 1), points=Q,
                meta=dict(name="slit_torus", n_u=n_u, n_v=n_v, R=R, r=r, sigma=sigma, seed=seed,
                          min_dist=min_dist))


def holey_heightfield(n: int = 2048, n_holes: int = 32, amp: float = 0.05, n_waves: int = 16,
                      grid_n: int = 512, extent: float = 1.1, seed: int = 0) -> Mesh:
    """(n+1)^2 vertex grid on [-1,1]^2 mapped to the unit disk by the
    concentric square-to-disk map, height = sum of ``n_waves`` sinusoids of
    amplitude ``amp``; triangles whose xy-centroid falls inside one of
    ``n_holes`` disjoint circles (centres in r <= 0.85, radius U(0.01, 0.05))
    are removed."""
    rng = np.random.default_rng(seed)
    s = np.linspace(-1.0, 1.0, n + 1)
    A, B = np.meshgrid(s, s, indexing="xy")
    a = A.ravel()
    b = B.ravel()
    # concentric (Shirley-Chiu) map
    r = np.where(np.abs(a) > np.abs(b), a, b)
    with np.errstate(divide="ignore", invalid="ignore"):
        phi = np.where(np.abs(a) > np.abs(b), (np.pi / 4) * (b / a),
                       np.pi / 2 - (np.pi / 4) * (a / b))
    phi = np.where((a == 0) & (b == 0), 0.0, phi)
    x = r * np.cos(phi)
    y = r * np.sin(phi)
    k = rng.uniform(2 * np.pi, 8 * np.pi, n_waves)
    th = rng.uniform(0, 2 * np.pi, n_waves)
    ph = rng.uniform(0, 2 * np.pi, n_waves)
    z = np.zeros_like(x)
    for w in range(n_waves):
        z += amp * np.sin(k[w] * (np.cos(th[w]) * x + np.sin(th[w]) * y) + ph[w])
    X = np.stack([x, y, z], -1)
    idx = np.arange((n + 1) * (n + 1)).reshape(n + 1, n + 1)
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    v00, v01 = idx[i, j], idx[i, j + 1]
    v10, v11 = idx[i + 1, j], idx[i + 1, j + 1]
    F = np.concatenate([np.stack([v00, v01, v11], -1).reshape(-1, 3),
                        np.stack([v00, v11, v10], -1).reshape(-1, 3)])
    nrm = np.cross(X[F[:, 1]] - X[F[:, 0]], X[F[:, 2]] - X[F[:, 0]])
    F = np.where((nrm[:, 2] < 0)[:, None], F[:, [0, 2, 1]], F)
    centres, radii = [], []
    while len(centres) < n_holes:
        rc = 0.85 * math.sqrt(rng.random())
        tc = 2 * math.pi * rng.random()
        c = np.array([rc * math.cos(tc), rc * math.sin(tc)])
        rad = rng.uniform(0.01, 0.05)
        if all(np.linalg.norm(c - c2) > rad + r2 + 0.02 for c2, r2 in zip(centres, radii)):
            centres.append(c)
            radii.append(rad)
    cen = X[F].mean(1)[:, :2]
    keep = np.ones(len(F), dtype=bool)
    for c, rad in zip(centres, radii):
        keep &= np.hypot(cen[:, 0] - c[0], cen[:, 1] - c[1]) > rad
    F = F[keep]
    Vc, Fc = _compact(X, F)
    g = Grid((-extent,) * 3, (extent,) * 3, (grid_n,) * 3)
    return Mesh(Vc.astype(np.float32), Fc.astype(np.int32), random_direction(seed + 1), grid=g,
                meta=dict(name="holey_heightfield", n=n, n_holes=n_holes, amp=amp, seed=seed,
                          hole_centres=np.array(centres), hole_radii=np.array(radii)))


# ----------------------------------------------------------------------------
# 2D Bezier chains
# ----------------------------------------------------------------------------
def bezier_circle_chain(n_seg: int = 32, noise: float = 0.3, grid_n: int = 128,
                        extent: float = 1.5, seed: int = 0, dtype=np.float64) -> Chains:
    """One open chain of ``n_seg`` cubic segments: 3*n_seg+1 control points at
    angles 2*pi*k/(3*n_seg+1) on a circle of radius 1 + U(-noise, noise)."""
    rng = np.random.default_rng(seed)
    m = 3 * n_seg + 1
    th = 2 * np.pi * np.arange(m) / m
    rad = 1.0 + rng.uniform(-noise, noise, m)
    ctrl = np.stack([rad * np.cos(th), rad * np.sin(th)], -1).astype(dtype)
    g = Grid((-extent, -extent), (extent, extent), (grid_n, grid_n))
    return Chains(ctrl, np.array([0, m], dtype=np.int64), [g],
                  meta=dict(name="bezier_circle_chain", n_seg=n_seg, seed=seed))


def star_chains(n_chains: int = 1024, seg_lo: int = 8, seg_hi: int = 2048, amp: float = 0.3,
                noise: float = 0.2, grid_n: int = 256, pad: float = 0.05, seed: int = 0,
                dtype=np.float32) -> Chains:
    """``n_chains`` open chains; chain c has n = round(exp(U(ln lo, ln hi)))
    segments, control points on r(t) = 1 + amp*cos(L t + phi) + U(-noise, noise)
    with L in {5..12}; each chain has its own grid_n^2 grid on its control
    point bbox padded by ``pad`` of the extent on every side."""
    rng = np.random.default_rng(seed)
    ctrls, offs, grids = [], [0], []
    for _ in range(n_chains):
        n = int(round(math.exp(rng.uniform(math.log(seg_lo), math.log(seg_hi)))))
        n = max(seg_lo, min(seg_hi, n))
        L = int(rng.integers(5, 13))
        phi = rng.uniform(0, 2 * np.pi)
        m = 3 * n + 1
        th = 2 * np.pi * np.arange(m) / m
        rad = 1.0 + amp * np.cos(L * th + phi) + rng.uniform(-noise, noise, m)
        c = np.stack([rad * np.cos(th), rad * np.sin(th)], -1).astype(dtype)
        ctrls.append(c)
        offs.append(offs[-1] + m)
        lo = c.astype(np.float64).min(0)
        hi = c.astype(np.float64).max(0)
        ext = hi - lo
        grids.append(Grid(tuple(lo - pad * ext), tuple(hi + pad * ext), (grid_n, grid_n)))
    return Chains(np.concatenate(ctrls), np.array(offs, dtype=np.int64), grids,
                  meta=dict(name="star_chains", n_chains=n_chains, seed=seed))


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------
def patch_spheroid(n: int = 2, amp: float = 0.08, open_faces: tuple = (), grid_n: int = 32,
                   extent: float = 1.3, seed: int = 0) -> Patches:
    """Six cube faces, each an n x n array of bicubic patches whose control
    points are the points of a (3n+1)^2 grid on the face, pushed radially onto
    r(x) = 1 + amp sin(3x + a) sin(2y + b) cos(z + c) (a, b, c from the seed).
    Neighbouring patches (also across cube edges) share their edge control
    points bit for bit, so the closed surface has no boundary; the faces
    listed in ``open_faces`` (0..5: +x, -x, +y, -y, +z, -z) are left out.
    Normals point outwards."""
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0.0, 2.0 * math.pi, 3)
    m = 3 * n
    s = np.array([-1.0 + 2.0 * k / m for k in range(m + 1)])
    S, T = np.meshgrid(s, s, indexing="ij")
    one = np.ones_like(S)
    faces = [np.stack([one, S, T], -1), np.stack([-one, T, S], -1), np.stack([T, one, S], -1),
             np.stack([S, -one, T], -1), np.stack([S, T, one], -1), np.stack([T, S, -one], -1)]
    ctrl = []
    for f, G in enumerate(faces):
        if f in open_faces:
            continue
        X = G / np.linalg.norm(G, axis=-1, keepdims=True)
        r = 1.0 + amp * np.sin(3 * X[..., 0] + ph[0]) * np.sin(2 * X[..., 1] + ph[1]) * np.cos(X[..., 2] + ph[2])
        X = (X * r[..., None]).astype(np.float32)
        for a in range(n):
            for b in range(n):
                ctrl.append(X[3 * a:3 * a + 4, 3 * b:3 * b + 4])
    ctrl = np.ascontiguousarray(np.array(ctrl, np.float32))
    return Patches(ctrl=ctrl, d=random_direction(seed), grid=Grid((-extent,) * 3, (extent,) * 3, (grid_n,) * 3),
                   meta={"n": n, "amp": amp, "open_faces": tuple(open_faces), "n_patches": len(ctrl)})


def config(name: str, seed: int = 0, small: bool = False):
    """The five workloads by name; ``small=True`` gives a reduced variant of
    the same construction for fast tests."""
    if name == "circle_chain_fp64":
        return bezier_circle_chain(seed=seed)
    if name == "icosphere_cap":
        return icosphere_cap(subdiv=4 if small else 6, grid_n=32 if small else 256, seed=seed)
    if name == "star_chains":
        return star_chains(n_chains=16 if small else 1024, seg_hi=256 if small else 2048,
                           grid_n=64 if small else 256, seed=seed)
    if name == "slit_torus":
        return slit_torus(n_u=64 if small else 1024, n_v=64 if small else 1024,
                          n_queries=4096 if small else (1 << 20), seed=seed)
    if name == "holey_heightfield":
        return holey_heightfield(n=128 if small else 2048, n_holes=4 if small else 32,
                                 grid_n=32 if small else 512, seed=seed)
    raise KeyError(name)
