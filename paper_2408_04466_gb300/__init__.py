"""GB300-native one-shot generalized winding numbers.

Thin Python binding over ``libgwn.so`` (C ABI declared in include/gwn.h).
PyTorch provides device memory and streams; every step of the evaluation
runs in the library's CUDA kernels.  There is no CPU fallback: if the
library is missing, construction raises.

    ctx  = Context()                       # current device, current stream
    mesh = Mesh(ctx, V, F)                 # float32 [nv,3], int32 [nf,3]
    w    = mesh.eval(Grid(lo, hi, dims), d)  # float32 tensor on the GPU
    ch   = Bezier2D(ctx, ctrl, offsets)    # cubic chains, float32/float64
    w2   = ch.eval(Grid(lo, hi, (nx, ny)))
"""
from __future__ import annotations

import atexit
import ctypes as C
import weakref
from dataclasses import dataclass

import numpy as np

from . import _capi
from ._capi import (F32, F64, MEM_DEVICE, MEM_HOST, QUERY_GRID, QUERY_POINTS, GwnError, check, gwn_geom_info,
                    gwn_plan, gwn_queries, gwn_stats, load)

__all__ = ["Context", "Mesh", "Bezier2D", "Patches", "Grid", "Points", "GwnFunction", "gwn_apply", "GwnError", "load",
           "boundary_extract_host", "monotone_split_host"]


def _torch():
    import torch
    return torch


@dataclass
class Grid:
    """Regular grid: dims[k] samples on [lo[k], hi[k]] (x fastest)."""
    lo: tuple
    hi: tuple
    dims: tuple

    @property
    def n(self) -> int:
        return int(np.prod(self.dims))

    def to_c(self, dtype: int = F32) -> gwn_queries:
        q = gwn_queries()
        q.kind = QUERY_GRID
        q.dtype = dtype
        q.mem_kind = MEM_DEVICE
        q.dim = len(self.dims)
        for k in range(len(self.dims)):
            q.lo[k] = float(self.lo[k])
            q.hi[k] = float(self.hi[k])
            q.dims[k] = int(self.dims[k])
        return q


class Points:
    """Explicit query points: a CUDA tensor [n, dim] (kept alive by this object)."""

    def __init__(self, pts, dtype=None):
        torch = _torch()
        if not isinstance(pts, torch.Tensor):
            pts = torch.as_tensor(np.asarray(pts))
        self.t = pts.contiguous()
        self.n = int(self.t.shape[0])

    def to_c(self, dtype: int = F32) -> gwn_queries:
        torch = _torch()
        q = gwn_queries()
        q.kind = QUERY_POINTS
        q.dtype = F64 if self.t.dtype == torch.float64 else F32
        q.mem_kind = MEM_DEVICE if self.t.is_cuda else MEM_HOST
        q.dim = int(self.t.shape[1])
        q.pts = self.t.data_ptr() if self.n else None
        q.n = self.n
        return q



class BatchQueries:
    """One grid per chain, marshalled once into the C array that
    gwn_eval_batch takes, with each chain's offset in the flat output."""

    def __init__(self, grids, dtype: int = F32):
        self.n_chains = len(grids)
        self.arr = (gwn_queries * self.n_chains)()
        self.offs = np.zeros(self.n_chains, np.int64)
        tot = 0
        for c, g in enumerate(grids):
            self.arr[c] = g.to_c(dtype)
            self.offs[c] = tot
            tot += g.n
        self.total = tot

# Live handles, closed geometries-first at interpreter exit (while CUDA and
# the streams they use are still alive); the library itself keeps a context
# alive until its last geometry is destroyed.
_live_geoms = weakref.WeakSet()
_live_ctxs = weakref.WeakSet()


@atexit.register
def _close_all():
    for g in list(_live_geoms):
        g.close()
    for c in list(_live_ctxs):
        c.close()


class Context:
    """A library context on one CUDA device, bound to a CUDA stream (default:
    torch's current stream at construction)."""

    def __init__(self, device: int | None = None, stream=None):
        torch = _torch()
        self.lib = load()
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = C.c_void_p()
        check(self.lib.gwn_ctx_create(C.byref(h), device, C.c_void_p(stream.cuda_stream)), "gwn_ctx_create")
        self.h = h
        _live_ctxs.add(self)

    def set_stream(self, stream):
        self.stream = stream
        check(self.lib.gwn_ctx_set_stream(self.h, C.c_void_p(stream.cuda_stream)), "gwn_ctx_set_stream")

    def check(self):
        check(self.lib.gwn_ctx_check(self.h), "gwn_ctx_check")

    def close(self):
        if getattr(self, "h", None):
            self.lib.gwn_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Geom:
    def info(self) -> dict:
        i = gwn_geom_info()
        check(self.lib.gwn_geom_info_get(self.h, C.byref(i)), "gwn_geom_info_get")
        return {k: getattr(i, k) for k, _ in i._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.gwn_geom_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _as_tensor(x, dtype):
    torch = _torch()
    if isinstance(x, torch.Tensor):
        return x.to(dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x)).to(dtype).contiguous()


def _dir(d):
    d = np.ascontiguousarray(np.asarray(d, dtype=np.float32).reshape(3))
    return d, d.ctypes.data_as(C.c_void_p)


class Mesh(_Geom):
    """Triangle mesh (float32 vertices, int32 faces, counter-clockwise = +normal)."""

    def __init__(self, ctx: Context, V, F):
        torch = _torch()
        self.ctx = ctx
        self.lib = ctx.lib
        Vt = _as_tensor(V, torch.float32)
        Ft = _as_tensor(F, torch.int32)
        mem = MEM_DEVICE if Vt.is_cuda else MEM_HOST
        if Ft.is_cuda != Vt.is_cuda:
            Ft = Ft.to(Vt.device)
        self.nv, self.nf = int(Vt.shape[0]), int(Ft.shape[0])
        h = C.c_void_p()
        check(self.lib.gwn_mesh_create(ctx.h, Vt.data_ptr() if self.nv else None, self.nv,
                                       Ft.data_ptr() if self.nf else None, self.nf, mem, C.byref(h)),
              "gwn_mesh_create")
        self.h = h
        _live_geoms.add(self)

    def set_index(self, index: str):
        """Crossing index: "auto" (2D bins when compact, else the LBVH) or
        "tree" (always the LBVH); the crossing counts are the same."""
        check(self.lib.gwn_mesh_set_index(self.h, {"auto": 0, "tree": 1}[index]), "gwn_mesh_set_index")

    def prepare(self, d):
        dd, dp = _dir(d)
        check(self.lib.gwn_mesh_prepare(self.h, dp), "gwn_mesh_prepare")

    def boundary(self):
        info = self.info()
        off = np.zeros(info["n_loops"] + 1, np.int64)
        vid = np.zeros(max(1, info["n_boundary_edges"]), np.int32)
        check(self.lib.gwn_mesh_boundary(self.h, off.ctypes.data_as(C.c_void_p), vid.ctypes.data_as(C.c_void_p)),
              "gwn_mesh_boundary")
        return off, vid[:info["n_boundary_edges"]]

    def eval(self, queries, d, want_chi=False, want_b=False, stats=False, out=None):
        torch = _torch()
        if not isinstance(queries, (Grid, Points)):
            queries = Points(queries)
        qc = queries.to_c(F32)
        n = queries.n
        dev = torch.device("cuda", self.ctx.device)
        w = out if out is not None else torch.empty(n, dtype=torch.float32, device=dev)
        chi = torch.empty(n, dtype=torch.int32, device=dev) if want_chi else None
        b = torch.empty(n, dtype=torch.float32, device=dev) if want_b else None
        st = gwn_stats() if stats else None
        dd, dp = _dir(d)
        check(self.lib.gwn_eval(self.h, C.byref(qc), dp, w.data_ptr() if n else None,
                                chi.data_ptr() if chi is not None and n else None,
                                b.data_ptr() if b is not None and n else None,
                                C.byref(st) if st is not None else None), "gwn_eval")
        res = {"w": w}
        if want_chi:
            res["chi"] = chi
        if want_b:
            res["b"] = b
        if stats:
            res["stats"] = st.as_dict()
        return res if (want_chi or want_b or stats) else w

    def inside(self, queries, d, out=None):
        """Inside test (voxelization): uint8 tensor, 1 where w >= 0.5."""
        torch = _torch()
        if not isinstance(queries, (Grid, Points)):
            queries = Points(queries)
        qc = queries.to_c(F32)
        n = queries.n
        r = out if out is not None else torch.empty(n, dtype=torch.uint8, device=torch.device("cuda", self.ctx.device))
        dd, dp = _dir(d)
        check(self.lib.gwn_eval_inside(self.h, C.byref(qc), dp, r.data_ptr() if n else None), "gwn_eval_inside")
        return r

    def eval_host(self, queries, d, out=None):
        """End-to-end entry point: host queries in, host w out.  out: an
        optional host float32 buffer of n entries (numpy array or CPU tensor;
        a page-locked one is written by the kernels directly)."""
        if isinstance(queries, Grid):
            qc = queries.to_c(F32)
            n = queries.n
            keep = None
        else:
            keep = np.ascontiguousarray(np.asarray(queries, dtype=np.float32))
            qc = gwn_queries()
            qc.kind = QUERY_POINTS
            qc.dtype = F32
            qc.mem_kind = MEM_HOST
            qc.dim = 3
            qc.pts = keep.ctypes.data_as(C.c_void_p)
            qc.n = len(keep)
            n = len(keep)
        if out is None:
            out = np.empty(n, np.float32)
        if isinstance(out, np.ndarray):
            assert out.dtype == np.float32 and out.size == n and out.flags["C_CONTIGUOUS"]
            ptr = out.ctypes.data
        else:
            assert (not out.is_cuda and out.dtype == _torch().float32 and out.numel() == n
                    and out.is_contiguous())
            ptr = out.data_ptr()
        dd, dp = _dir(d)
        check(self.lib.gwn_eval_host(self.h, C.byref(qc), dp, C.c_void_p(ptr)), "gwn_eval_host")
        return out

    def backward(self, P, grad_w, want_p=True, want_V=True):
        torch = _torch()
        pts = Points(P)
        qc = pts.to_c(F32)
        gw = _as_tensor(grad_w, torch.float32).to(pts.t.device)
        gp = torch.empty((pts.n, 3), dtype=torch.float32, device=pts.t.device) if want_p else None
        gV = torch.empty((self.nv, 3), dtype=torch.float32, device=pts.t.device) if want_V else None
        check(self.lib.gwn_backward(self.h, C.byref(qc), None, gw.data_ptr() if pts.n else None,
                                    gp.data_ptr() if gp is not None and pts.n else None,
                                    gV.data_ptr() if gV is not None else None), "gwn_backward")
        return gp, gV

    def bruteforce(self, queries):
        torch = _torch()
        if not isinstance(queries, (Grid, Points)):
            queries = Points(queries)
        qc = queries.to_c(F32)
        w = torch.empty(queries.n, dtype=torch.float32, device=torch.device("cuda", self.ctx.device))
        check(self.lib.gwn_eval_bruteforce(self.h, C.byref(qc), w.data_ptr()), "gwn_eval_bruteforce")
        return w


class Patches(_Geom):
    """Surface of bicubic Bezier patches: ctrl [n, 4, 4, 3] float32 (P_ij at
    [t, i, j], i along u, j along v; normal f_u x f_v); boundary curves sampled
    at `segments` intervals for the boundary term."""

    def __init__(self, ctx: Context, ctrl, segments: int = 64):
        torch = _torch()
        self.ctx = ctx
        self.lib = ctx.lib
        ct = _as_tensor(np.asarray(ctrl, np.float32).reshape(-1, 48) if not hasattr(ctrl, "is_cuda") else ctrl,
                        torch.float32).reshape(-1, 48).contiguous()
        mem = MEM_DEVICE if ct.is_cuda else MEM_HOST
        self.n = int(ct.shape[0])
        h = C.c_void_p()
        check(self.lib.gwn_patches_create(ctx.h, ct.data_ptr() if self.n else None, self.n, int(segments), mem,
                                          C.byref(h)), "gwn_patches_create")
        self.h = h
        _live_geoms.add(self)

    def eval(self, queries, d, want_chi=False, want_b=False, stats=False, out=None):
        return Mesh.eval(self, queries, d, want_chi=want_chi, want_b=want_b, stats=stats, out=out)

    def eval_host(self, queries, d, out=None):
        return Mesh.eval_host(self, queries, d, out=out)

    def inside(self, queries, d, out=None):
        return Mesh.inside(self, queries, d, out=out)


class Bezier2D(_Geom):
    """Open C0 cubic Bezier chains: ctrl [n_ctrl, 2] (float32 or float64),
    chain c = ctrl[offsets[c]:offsets[c+1]] (3k+1 points)."""

    def __init__(self, ctx: Context, ctrl, offsets):
        torch = _torch()
        self.ctx = ctx
        self.lib = ctx.lib
        if isinstance(ctrl, torch.Tensor):
            ct = ctrl.contiguous()
        else:
            arr = np.ascontiguousarray(ctrl)
            ct = torch.as_tensor(arr)
        self.dtype = F64 if ct.dtype == torch.float64 else F32
        if ct.dtype not in (torch.float32, torch.float64):
            ct = ct.float()
        self.tdtype = ct.dtype
        self.offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        mem = MEM_DEVICE if ct.is_cuda else MEM_HOST
        h = C.c_void_p()
        check(self.lib.gwn_bezier2d_create(ctx.h, ct.data_ptr(), self.dtype,
                                           self.offsets.ctypes.data_as(C.c_void_p), len(self.offsets) - 1, mem,
                                           C.byref(h)), "gwn_bezier2d_create")
        self.h = h
        _live_geoms.add(self)
        self.n_chains = len(self.offsets) - 1

    def eval(self, queries, want_chi=False, want_b=False, stats=False):
        """w at a Grid (one +x ray per grid row) or at Points [n, 2] in the
        chain dtype (one +x ray per point)."""
        torch = _torch()
        qc = queries.to_c(self.dtype)
        n = queries.n
        dev = torch.device("cuda", self.ctx.device)
        w = torch.empty(n, dtype=self.tdtype, device=dev)
        chi = torch.empty(n, dtype=torch.int32, device=dev) if want_chi else None
        b = torch.empty(n, dtype=self.tdtype, device=dev) if want_b else None
        st = gwn_stats() if stats else None
        check(self.lib.gwn_eval(self.h, C.byref(qc), None, w.data_ptr(), chi.data_ptr() if chi is not None else None,
                                b.data_ptr() if b is not None else None, C.byref(st) if st is not None else None),
              "gwn_eval")
        res = {"w": w}
        if want_chi:
            res["chi"] = chi
        if want_b:
            res["b"] = b
        if stats:
            res["stats"] = st.as_dict()
        return res if (want_chi or want_b or stats) else w

    def eval_host(self, grid: Grid) -> np.ndarray:
        qc = grid.to_c(self.dtype)
        out = np.empty(grid.n, np.float64 if self.dtype == F64 else np.float32)
        check(self.lib.gwn_eval_host(self.h, C.byref(qc), None, out.ctypes.data_as(C.c_void_p)), "gwn_eval_host")
        return out

    def batch_queries(self, grids):
        """Marshal one grid per chain once (a BatchQueries), for repeated
        eval_batch calls on the same grids."""
        return BatchQueries(grids, self.dtype)

    def eval_batch(self, grids, out=None, threads=0, rows=0, use_graph=True, stats=False):
        """Each chain c on its own grid grids[c] (a list of Grid or a
        BatchQueries); returns one flat tensor with chain c's grid at
        offsets[c] (and the offsets)."""
        torch = _torch()
        bq = grids if isinstance(grids, BatchQueries) else BatchQueries(grids, self.dtype)
        assert bq.n_chains == self.n_chains
        w = out if out is not None else torch.empty(bq.total, dtype=self.tdtype,
                                                    device=torch.device("cuda", self.ctx.device))
        plan = gwn_plan(threads, rows, 0, 1 if use_graph else 0)
        st = gwn_stats() if stats else None
        check(self.lib.gwn_eval_batch(self.h, bq.arr, bq.n_chains, bq.offs.ctypes.data_as(C.c_void_p), w.data_ptr(),
                                      C.byref(plan), C.byref(st) if st is not None else None), "gwn_eval_batch")
        if stats:
            return w, bq.offs, st.as_dict()
        return w, bq.offs

    def batch_plan(self):
        t, r = C.c_int32(), C.c_int32()
        check(self.lib.gwn_batch_plan_get(self.h, C.byref(t), C.byref(r)), "gwn_batch_plan_get")
        return t.value, r.value

    def bruteforce(self, grid: Grid):
        torch = _torch()
        qc = grid.to_c(self.dtype)
        w = torch.empty(grid.n, dtype=self.tdtype, device=torch.device("cuda", self.ctx.device))
        check(self.lib.gwn_eval_bruteforce(self.h, C.byref(qc), w.data_ptr()), "gwn_eval_bruteforce")
        return w


# ----------------------------------------------------------------------------
# autograd
# ----------------------------------------------------------------------------
def _make_function():
    torch = _torch()

    class GwnFunction(torch.autograd.Function):
        """w = GWN(P; V) for a fixed mesh topology; backward gives dw/dP and
        dw/dV from the boundary term (the crossing count is piecewise constant)."""

        @staticmethod
        def forward(ctx, P, V, mesh, d):
            ctx.mesh = mesh
            ctx.save_for_backward(P)
            return mesh.eval(Points(P.detach()), d)

        @staticmethod
        def backward(ctx, grad_w):
            (P,) = ctx.saved_tensors
            gp, gV = ctx.mesh.backward(P.detach(), grad_w.contiguous(), want_p=ctx.needs_input_grad[0],
                                       want_V=ctx.needs_input_grad[1])
            return gp, gV, None, None

    return GwnFunction


class _Lazy:
    _fn = None

    def __getattr__(self, item):
        if _Lazy._fn is None:
            _Lazy._fn = _make_function()
        return getattr(_Lazy._fn, item)


GwnFunction = _Lazy()


def eval_meshes(ctx: Context, meshes, queries, d, outs=None, tiles_per_item=0, blocks_per_sm=0, use_graph=True,
                stats=False):
    """w of every mesh at its own queries (Grid or device Points) in one
    persistent launch (gwn_eval_meshes).  The meshes must be prepared for d.
    Returns the list of float32 outputs (and the stats when asked)."""
    torch = _torch()
    n = len(meshes)
    assert n == len(queries) and n >= 1
    arr = (gwn_queries * n)()
    keep = []
    for i, q in enumerate(queries):
        if not isinstance(q, (Grid, Points)):
            raise TypeError("queries must be Grid or Points")
        arr[i] = q.to_c(F32)
        keep.append(q)
    dev = torch.device("cuda", ctx.device)
    if outs is None:
        outs = [torch.empty(q.n, dtype=torch.float32, device=dev) for q in queries]
    hs = (C.c_void_p * n)(*[m.h for m in meshes])
    ws = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    dd, dptr = _dir(d)
    plan = gwn_plan(blocks_per_sm, tiles_per_item, 0, 1 if use_graph else 0)
    st = gwn_stats() if stats else None
    check(ctx.lib.gwn_eval_meshes(ctx.h, hs, arr, n, dptr, ws,
                                  C.byref(plan) if (tiles_per_item or blocks_per_sm or not use_graph) else None,
                                  C.byref(st) if st is not None else None), "gwn_eval_meshes")
    if stats:
        return outs, st.as_dict()
    return outs


def meshes_plan(ctx: Context):
    """(tiles per work item, blocks per SM) of the most recent batched mesh plan."""
    t, b = C.c_int32(), C.c_int32()
    check(ctx.lib.gwn_meshes_plan_get(ctx.h, C.byref(t), C.byref(b)), "gwn_meshes_plan_get")
    return t.value, b.value


def gwn_apply(mesh: Mesh, P, V, d):
    """Differentiable w at query points P (CUDA float32 [n,3]); V must be the
    vertex tensor the mesh was built from (its gradient is dw/dV)."""
    return GwnFunction.apply(P, V, mesh, d)


# ----------------------------------------------------------------------------
# host-only helpers (no device needed)
# ----------------------------------------------------------------------------
def boundary_extract_host(F, nv: int):
    """Boundary loops of a triangle list by the library's host extraction:
    returns (loop_offsets int64[n_loops+1], vertex ids int32[n_edges])."""
    lib = load()
    F = np.ascontiguousarray(np.asarray(F, dtype=np.int32))
    cap = 3 * len(F) + 1
    off = np.zeros(cap, np.int64)
    vid = np.zeros(max(1, 3 * len(F)), np.int32)
    nl, ne = C.c_int64(), C.c_int64()
    check(lib.gwn_boundary_extract_host(F.ctypes.data_as(C.c_void_p), len(F), int(nv),
                                        off.ctypes.data_as(C.c_void_p), vid.ctypes.data_as(C.c_void_p),
                                        C.byref(nl), C.byref(ne)), "gwn_boundary_extract_host")
    return off[:nl.value + 1].copy(), vid[:ne.value].copy()


def monotone_split_host(ctrl8):
    """Parameter intervals of the y-monotone pieces of one cubic segment."""
    lib = load()
    c = np.ascontiguousarray(np.asarray(ctrl8, dtype=np.float64).reshape(8))
    u = np.zeros(6, np.float64)
    n = C.c_int32()
    check(lib.gwn_bezier_monotone_split_host(c.ctypes.data_as(C.c_void_p), u.ctypes.data_as(C.c_void_p),
                                             C.byref(n)), "gwn_bezier_monotone_split_host")
    return u[:2 * n.value].reshape(-1, 2)
