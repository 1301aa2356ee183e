"""FP64 CPU oracle for generalized winding numbers -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library (``paper_2408_04466_gb300``) and never imports it.

The heavy loops live in ``gwn_oracle.c`` (plain C, float64, exact predicates
by big-integer arithmetic on float32 inputs); this module compiles it with gcc
on first use and wraps it with ctypes.  Functions and the passages they follow:

* ``w3d_vos``        3D definition, sum of per-triangle solid angles
                     (Background: w_M(p) = (1/4pi) int_M dOmega).
* ``chi3d``          signed crossing count of the ray p + t d (Eq. chi),
                     brute force over all triangles, exact predicates.
* ``boundary_edges`` boundary edges with net multiplicity.
* ``bterm3d``        boundary term relative to d (Lemma 1, Lemma 2, and the
                     closure argument of the proof in Appendix A).
* ``w3d_oneshot``    chi3d + bterm3d.
* ``w3d_patches_quad`` 3D definition for bicubic Bezier patches (adaptive
                     tensor Gauss-Legendre of the solid-angle element).
* ``patch_boundary``  boundary curves of a patch set (net multiplicity of
                     the patch edge curves) sampled as a polyline.
* ``w3d_alg1``       Algorithm 1 in 3D, literally: arrangement of the
                     projected boundary on the unit sphere, region areas,
                     one ray in the largest region, counts propagated across
                     the arcs (Lemma 2), area-weighted sum (tiny inputs).
* ``grad3d_vos``     gradient of the 3D definition (chain rule on the
                     per-triangle solid angle).
* ``w2d_quad``       2D definition, adaptive Gauss-Kronrod per segment
                     (Background: w_C(p) = (1/2pi) int_C dtheta).
* ``w2d_alg1``       Algorithm 1 in 2D (regions on the circle, one ray in the
                     largest region, pairwise difference, area-weighted sum).
* ``w2d_closed_x``   the +x-ray closed form (count + chord closure).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gwn_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-ffp-contract=off", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB_PATH)
            P = C.c_void_p
            I64 = C.c_int64
            I = C.c_int
            sigs = {
                "oracle_w3d_vos": (None, [P, P, I64, P, I64, P, I]),
                "oracle_chi3d": (None, [P, P, I64, P, I64, P, P, I]),
                "oracle_boundary_edges": (I64, [P, I64, P, P, P]),
                "oracle_bterm3d": (None, [P, P, P, P, I64, P, I64, P, P, I]),
                "oracle_grad3d_vos": (I, [P, I64, P, I64, P, I64, P, P, P, I]),
                "oracle_w2d_quad": (None, [P, I64, P, I64, P, C.c_double, I]),
                "oracle_w2d_alg1": (None, [P, I64, P, I64, P, I]),
                "oracle_w2d_closed_x": (None, [P, I64, P, I64, P, P, P, I]),
                "oracle_sign_edge": (I, [P, P, P, P]),
                "oracle_exact_det_abd": (I, [P, P, P, P]),
                "oracle_sign_orient": (I, [P, P, P, P]),
                "oracle_exact_orient": (I, [P, P, P, P]),
                "oracle_tri_crossing": (I, [P, P, P, P, P]),
                "oracle_solid_angle": (C.c_double, [P, P, P]),
                "oracle_chain_ray_crossings": (I, [P, I64, P, P]),
                "oracle_dist3d": (None, [P, P, I64, P, I64, P, I]),
                "oracle_dist2d": (None, [P, I64, P, I64, P, I]),
                "oracle_w3d_alg1": (I, [P, I64, P, I64, P, P, P]),
                "oracle_w3d_patches_quad": (None, [P, I64, P, I64, P, C.c_double, I]),
            }
            for name, (res, args) in sigs.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _f32(a, shape_last=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape_last is not None:
        assert a.shape[-1] == shape_last
    return a


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


# ----------------------------------------------------------------------------
# 3D
# ----------------------------------------------------------------------------
def w3d_vos(V, F, P, threads: int | None = None) -> np.ndarray:
    """w(p) = (1/4pi) * sum over triangles of the Van Oosterom-Strackee solid angle."""
    V, F, P = _f32(V, 3), _i32(F), _f32(P, 3)
    w = np.empty(len(P), dtype=np.float64)
    _load().oracle_w3d_vos(_ptr(V), _ptr(F), len(F), _ptr(P), len(P), _ptr(w),
                           threads or default_threads())
    return w


def chi3d(V, F, P, d, threads: int | None = None) -> np.ndarray:
    """Signed crossings of p + t d (t > 0) with all triangles (Eq. chi), exact."""
    V, F, P, d = _f32(V, 3), _i32(F), _f32(P, 3), _f32(d, 3)
    chi = np.empty(len(P), dtype=np.int32)
    _load().oracle_chi3d(_ptr(V), _ptr(F), len(F), _ptr(P), len(P), _ptr(d), _ptr(chi),
                         threads or default_threads())
    return chi


def boundary_edges(F):
    """Directed boundary edges (src, dst, multiplicity > 0), sorted by the
    undirected pair."""
    F = _i32(F)
    cap = max(1, 3 * len(F))
    src = np.empty(cap, np.int32)
    dst = np.empty(cap, np.int32)
    m = np.empty(cap, np.int32)
    n = _load().oracle_boundary_edges(_ptr(F), len(F), _ptr(src), _ptr(dst), _ptr(m))
    if n < 0:
        raise MemoryError("oracle_boundary_edges")
    return src[:n].copy(), dst[:n].copy(), m[:n].copy()


def bterm3d(V, edges, P, d, threads: int | None = None) -> np.ndarray:
    """B_d(p) = (1/4pi) sum_e m_e Omega(A_e - p, B_e - p, -d)."""
    V, P, d = _f32(V, 3), _f32(P, 3), _f32(d, 3)
    src, dst, m = (_i32(x) for x in edges)
    B = np.empty(len(P), dtype=np.float64)
    _load().oracle_bterm3d(_ptr(V), _ptr(src), _ptr(dst), _ptr(m), len(src), _ptr(P), len(P),
                           _ptr(d), _ptr(B), threads or default_threads())
    return B


def w3d_oneshot(V, F, P, d, threads: int | None = None, edges=None):
    """One-shot w = chi_d + B_d; returns (w, chi, B)."""
    if edges is None:
        edges = boundary_edges(F)
    chi = chi3d(V, F, P, d, threads)
    B = bterm3d(V, edges, P, d, threads)
    return chi + B, chi, B


def w3d_alg1(V, F, P):
    """Algorithm 1 in 3D by a spherical arrangement, one query at a time
    (tiny, generic inputs).  Returns (w, info) with info[q] = (regions, area
    of the largest region, its crossing count); raises on degenerate input."""
    V = _f32(V, 3)
    F = _i32(F).reshape(-1, 3)
    P = _f32(P, 3).reshape(-1, 3)
    w = np.empty(len(P), np.float64)
    info = np.zeros((len(P), 3), np.float64)
    lib = _load()
    for q in range(len(P)):
        out = C.c_double(0.0)
        rc = lib.oracle_w3d_alg1(_ptr(V), len(V), _ptr(F), len(F), _ptr(P[q]), C.byref(out),
                                 _ptr(info[q]))
        if rc != 0:
            raise ValueError(f"w3d_alg1: query {q}: status {rc}")
        w[q] = out.value
    return w, info


def w3d_patches_quad(ctrl, P, tol: float = 1e-13, threads: int | None = None) -> np.ndarray:
    """Definition for bicubic patches ctrl [n, 4, 4, 3] (float32)."""
    ctrl = _f32(ctrl).reshape(-1, 48)
    P = _f32(P, 3).reshape(-1, 3)
    w = np.empty(len(P), np.float64)
    _load().oracle_w3d_patches_quad(_ptr(ctrl), len(ctrl), _ptr(P), len(P), _ptr(w), tol,
                                    threads or default_threads())
    return w


def patch_boundary(ctrl, k: int):
    """Boundary of a set of bicubic patches as a polyline (V float32, edges
    (src, dst, mult) int32 arrays) for the FP64 boundary term.  Each patch
    contributes its four edge curves in the direction of the counter-clockwise
    boundary of the (u, v) square (the orientation of f_u x f_v); a curve and
    its reverse cancel; a curve with net multiplicity m != 0 is sampled at k
    segments (float64 Bernstein evaluation rounded to float32, so its ends are
    its end control points exactly)."""
    ctrl = np.asarray(ctrl, np.float32).reshape(-1, 4, 4, 3)
    net = {}
    for t in range(len(ctrl)):
        P = ctrl[t]
        for cur in (P[:, 0], P[3, :], P[::-1, 3], P[0, ::-1]):
            fwd = tuple(cur.reshape(-1).view(np.uint32).tolist())
            rev = tuple(cur[::-1].reshape(-1).view(np.uint32).tolist())
            key, sgn = (fwd, 1) if fwd <= rev else (rev, -1)
            net[key] = net.get(key, 0) + sgn
    pts, index = [], {}

    def vid(x):
        key = tuple(np.asarray(x, np.float32).view(np.uint32).tolist())
        if key not in index:
            index[key] = len(pts)
            pts.append(np.asarray(x, np.float32))
        return index[key]

    src, dst, mul = [], [], []
    s = np.arange(k + 1) / k
    B = np.stack([(1 - s) ** 3, 3 * s * (1 - s) ** 2, 3 * s ** 2 * (1 - s), s ** 3], 1)
    for key, m in sorted(net.items()):
        if m == 0:
            continue
        c = np.array(key, np.uint32).view(np.float32).reshape(4, 3).astype(np.float64)
        if np.all(c == c[0]):
            continue                                  # a collapsed edge bounds nothing
        X = (B @ c).astype(np.float32)
        X[0], X[-1] = c[0].astype(np.float32), c[3].astype(np.float32)
        ids = [vid(x) for x in X]
        for a, b in zip(ids[:-1], ids[1:]):
            if m > 0:
                src.append(a); dst.append(b); mul.append(m)
            else:
                src.append(b); dst.append(a); mul.append(-m)
    V = np.array(pts, np.float32).reshape(-1, 3)
    return V, (np.array(src, np.int32), np.array(dst, np.int32), np.array(mul, np.int32))


def grad3d_vos(V, F, P, gw=None, want_p=True, want_V=True, threads: int | None = None):
    """Analytic FP64 gradient of the solid-angle sum: (gw * dw/dp per query,
    sum_q gw_q * dw_q/dV)."""
    V, F, P = _f32(V, 3), _i32(F), _f32(P, 3)
    g = None if gw is None else _f64(gw)
    gp = np.empty((len(P), 3), np.float64) if want_p else None
    gV = np.zeros((len(V), 3), np.float64) if want_V else None
    rc = _load().oracle_grad3d_vos(_ptr(V), len(V), _ptr(F), len(F), _ptr(P), len(P), _ptr(g),
                                   _ptr(gp), _ptr(gV), threads or default_threads())
    if rc != 0:
        raise MemoryError("oracle_grad3d_vos")
    return gp, gV


def solid_angle(a, b, c) -> float:
    a, b, c = _f64(a), _f64(b), _f64(c)
    return _load().oracle_solid_angle(_ptr(a), _ptr(b), _ptr(c))


def sign_edge(A, B, P, D) -> int:
    """Sign of det[A-P, B-P, D_eps] with the symbolic perturbation of D."""
    A, B, P, D = (_f32(x, 3) for x in (A, B, P, D))
    return _load().oracle_sign_edge(_ptr(A), _ptr(B), _ptr(P), _ptr(D))


def exact_det_abd(A, B, P, D) -> int:
    A, B, P, D = (_f32(x, 3) for x in (A, B, P, D))
    return _load().oracle_exact_det_abd(_ptr(A), _ptr(B), _ptr(P), _ptr(D))


def sign_orient(V0, V1, V2, P) -> int:
    V0, V1, V2, P = (_f32(x, 3) for x in (V0, V1, V2, P))
    return _load().oracle_sign_orient(_ptr(V0), _ptr(V1), _ptr(V2), _ptr(P))


def exact_orient(V0, V1, V2, P) -> int:
    V0, V1, V2, P = (_f32(x, 3) for x in (V0, V1, V2, P))
    return _load().oracle_exact_orient(_ptr(V0), _ptr(V1), _ptr(V2), _ptr(P))


def tri_crossing(v0, v1, v2, p, d) -> int:
    v0, v1, v2, p, d = (_f32(x, 3) for x in (v0, v1, v2, p, d))
    return _load().oracle_tri_crossing(_ptr(v0), _ptr(v1), _ptr(v2), _ptr(p), _ptr(d))


# ----------------------------------------------------------------------------
# 2D
# ----------------------------------------------------------------------------
def _chain(ctrl):
    ctrl = _f64(ctrl)
    assert ctrl.ndim == 2 and ctrl.shape[1] == 2 and (len(ctrl) - 1) % 3 == 0
    return ctrl, (len(ctrl) - 1) // 3


def w2d_quad(ctrl, P, tol: float = 1e-14, threads: int | None = None) -> np.ndarray:
    ctrl, nseg = _chain(ctrl)
    P = _f64(P)
    w = np.empty(len(P), np.float64)
    _load().oracle_w2d_quad(_ptr(ctrl), nseg, _ptr(P), len(P), _ptr(w), tol,
                            threads or default_threads())
    return w


def w2d_alg1(ctrl, P, threads: int | None = None) -> np.ndarray:
    ctrl, nseg = _chain(ctrl)
    P = _f64(P)
    w = np.empty(len(P), np.float64)
    _load().oracle_w2d_alg1(_ptr(ctrl), nseg, _ptr(P), len(P), _ptr(w), threads or default_threads())
    return w


def w2d_closed_x(ctrl, P, threads: int | None = None, want_unc: bool = False):
    """Returns (w, chi) with chi = crossings of the +x ray with chain + chord
    (and, with want_unc, a bool array marking the queries whose count is not
    certified: a crossing, or the chord, within its float64 error bound of
    the query -- the query lies on the geometry at float64 resolution)."""
    ctrl, nseg = _chain(ctrl)
    P = _f64(P)
    w = np.empty(len(P), np.float64)
    chi = np.empty(len(P), np.int32)
    unc = np.zeros(len(P), np.int8)
    _load().oracle_w2d_closed_x(_ptr(ctrl), nseg, _ptr(P), len(P), _ptr(w), _ptr(chi), _ptr(unc),
                                threads or default_threads())
    if want_unc:
        return w, chi, unc.astype(bool)
    return w, chi


def chain_ray_crossings(ctrl, p, q) -> int:
    ctrl, nseg = _chain(ctrl)
    p, q = _f64(p), _f64(q)
    return _load().oracle_chain_ray_crossings(_ptr(ctrl), nseg, _ptr(p), _ptr(q))


# ----------------------------------------------------------------------------
# distances (used by the tests to exclude queries near the surface, where w
# is undefined)
# ----------------------------------------------------------------------------
def dist3d(V, F, P, threads: int | None = None) -> np.ndarray:
    """Euclidean distance from each query to the closest triangle (float64)."""
    V, F, P = _f32(V, 3), _i32(F), _f32(P, 3)
    out = np.empty(len(P), np.float64)
    _load().oracle_dist3d(_ptr(V), _ptr(F), len(F), _ptr(P), len(P), _ptr(out),
                          threads or default_threads())
    return out


def dist2d(ctrl, P, threads: int | None = None) -> np.ndarray:
    """Distance from each query to a cubic chain (dense sampling + refinement)."""
    ctrl, nseg = _chain(ctrl)
    P = _f64(P)
    out = np.empty(len(P), np.float64)
    _load().oracle_dist2d(_ptr(ctrl), nseg, _ptr(P), len(P), _ptr(out), threads or default_threads())
    return out
