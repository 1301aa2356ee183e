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
    sizes = (200_000, 77_777)             # two calls in a row, different sizes and points
    Ps = [torch.as_tensor(rng.uniform(-1.3, 1.3, (n, 3)).astype(np.float32)).cuda() for n in sizes]
    refs = [mesh.eval(gwn.Points(P), d) for P in Ps]
    outs = [torch.full((n,), float("nan"), dtype=torch.float32, device="cuda") for n in sizes]

    def call(P, w):
        rc = lib.gwn_eval_points_noalloc(mesh.h, C.c_void_p(P.data_ptr()), P.shape[0], dptr,
                                         C.c_void_p(w.data_ptr()))
        _capi.check(rc, "gwn_eval_points_noalloc")

    call(Ps[1], outs[1])                  # warm call: the first launch may load code modules
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    outs[1].fill_(float("nan"))
    for P, w in zip(Ps, outs):
        call(P, w)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()    # read before any comparison allocates temporaries
    assert free1 == free0, f"device memory changed by {free0 - free1} bytes across the calls"
    for w, ref in zip(outs, refs):
        # the same kernels on the same input as gwn_eval: identical bits
        assert torch.equal(w, ref)
    P, w = Ps[1], outs[1]
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
