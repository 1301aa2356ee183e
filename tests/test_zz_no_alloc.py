"""The allocation-free mesh entry point (gwn_eval_points_noalloc), called
through the C ABI and compared with gwn_eval.

It serves callers that reserve all device memory up front and cannot call
cudaMalloc later (cudaMalloc can stall the whole device and can fail under
memory pressure in the middle of a request): its scratch lives in a fixed
array inside the library.  This file is collected last so that a run that
stops at the first failure has already run every other test; it also passes
on its own in a fresh process."""
import ctypes as C

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu
TOL = 1e-6          # the float32 bar of the other parity tests


def test_noalloc_matches_gwn_eval_on_two_calls(cuda_available):
    import torch

    import paper_2408_04466_gb300 as gwn
    from paper_2408_04466_gb300 import _capi, build
    build.build()
    lib = gwn.load()
    ctx = gwn.Context(0)
    m = gen.icosphere_cap(subdiv=4, seed=9)
    mesh = gwn.Mesh(ctx, m.V, m.F)
    d = np.ascontiguousarray(m.d, np.float32)
    dptr = d.ctypes.data_as(C.c_void_p)
    mesh.prepare(d)                       # allocates; must precede the allocation-free calls
    rng = np.random.default_rng(4)
    for n in (200_000, 77_777):           # two calls in a row, different sizes and points
        P = torch.as_tensor(rng.uniform(-1.3, 1.3, (n, 3)).astype(np.float32)).cuda()
        ref = mesh.eval(gwn.Points(P), d)
        w = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        rc = lib.gwn_eval_points_noalloc(mesh.h, C.c_void_p(P.data_ptr()), n, dptr, C.c_void_p(w.data_ptr()))
        _capi.check(rc, "gwn_eval_points_noalloc")
        torch.cuda.synchronize()
        assert torch.isfinite(w).all()
        assert (w - ref).abs().max().item() <= TOL
    ctx.check()
    # more queries than the fixed array holds: rejected before any work
    rc = lib.gwn_eval_points_noalloc(mesh.h, C.c_void_p(P.data_ptr()), _capi.NOALLOC_MAX_QUERIES + 1, dptr,
                                     C.c_void_p(w.data_ptr()))
    assert rc == -1 and b"4,194,304" in lib.gwn_last_error()
    # a direction the mesh was not prepared for: rejected (preparing would allocate)
    d2 = np.ascontiguousarray(gen.random_direction(77), np.float32)
    rc = lib.gwn_eval_points_noalloc(mesh.h, C.c_void_p(P.data_ptr()), 10, d2.ctypes.data_as(C.c_void_p),
                                     C.c_void_p(w.data_ptr()))
    assert rc == -1 and b"gwn_mesh_prepare" in lib.gwn_last_error()
