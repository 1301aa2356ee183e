"""ctypes declarations mirroring include/gwn.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgwn.so")

GWN_OK = 0
NOALLOC_MAX_QUERIES = 4194304
STATUS = {0: "GWN_OK", -1: "GWN_E_INVALID", -2: "GWN_E_OOM", -3: "GWN_E_CUDA", -4: "GWN_E_STACK_OVERFLOW",
          -5: "GWN_E_TIMEOUT", -6: "GWN_E_UNSUPPORTED", -7: "GWN_E_INTERNAL"}
MEM_HOST, MEM_DEVICE = 0, 1
F32, F64 = 0, 1
QUERY_POINTS, QUERY_GRID = 0, 1
GEOM_MESH, GEOM_BEZIER2D = 1, 2


class gwn_queries(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dtype", C.c_int32), ("mem_kind", C.c_int32), ("dim", C.c_int32),
                ("pts", C.c_void_p), ("n", C.c_int64), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("dims", C.c_int64 * 3)]


class gwn_stats(C.Structure):
    _fields_ = [("n_queries", C.c_int64), ("n_pairs", C.c_int64), ("n_cut_sign", C.c_int64),
                ("n_fp64_filter", C.c_int64), ("n_exact", C.c_int64), ("n_stack_overflow", C.c_int64),
                ("n_tri_tests", C.c_int64), ("ms_prepare", C.c_float), ("ms_traverse", C.c_float),
                ("ms_boundary", C.c_float), ("ms_total", C.c_float), ("n_deferred_traverse", C.c_int64),
                ("n_deferred_boundary", C.c_int64), ("n_root_iters", C.c_int64), ("n_cert", C.c_int64),
                ("n_cert_fixed", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gwn_geom_info(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dtype", C.c_int32), ("n_vertices", C.c_int64), ("n_primitives", C.c_int64),
                ("n_boundary_edges", C.c_int64), ("n_loops", C.c_int64), ("n_pieces", C.c_int64),
                ("n_chains", C.c_int64), ("n_bins", C.c_int64), ("n_bin_entries", C.c_int64),
                ("bin_maxlen", C.c_int64)]


class gwn_plan(C.Structure):
    _fields_ = [("threads_per_block", C.c_int32), ("rows_per_item", C.c_int32), ("pieces_per_item", C.c_int32),
                ("use_graph", C.c_int32)]


P = C.c_void_p
I64 = C.c_int64
I32 = C.c_int32
ST = C.c_int
_SIGS = {
    "gwn_version": (C.c_char_p, []),
    "gwn_last_error": (C.c_char_p, []),
    "gwn_ctx_create": (ST, [C.POINTER(P), C.c_int, P]),
    "gwn_ctx_set_stream": (ST, [P, P]),
    "gwn_ctx_check": (ST, [P]),
    "gwn_ctx_destroy": (None, [P]),
    "gwn_mesh_create": (ST, [P, P, I64, P, I64, C.c_int, C.POINTER(P)]),
    "gwn_mesh_prepare": (ST, [P, P]),
    "gwn_bezier2d_create": (ST, [P, P, C.c_int, P, I64, C.c_int, C.POINTER(P)]),
    "gwn_patches_create": (ST, [P, P, I64, C.c_int, C.c_int, C.POINTER(P)]),
    "gwn_geom_info_get": (ST, [P, C.POINTER(gwn_geom_info)]),
    "gwn_geom_destroy": (None, [P]),
    "gwn_mesh_set_index": (ST, [P, I32]),
    "gwn_mesh_boundary": (ST, [P, P, P]),
    "gwn_boundary_extract_host": (ST, [P, I64, I64, P, P, C.POINTER(I64), C.POINTER(I64)]),
    "gwn_bezier_monotone_split_host": (ST, [P, P, C.POINTER(I32)]),
    "gwn_eval": (ST, [P, C.POINTER(gwn_queries), P, P, P, P, C.POINTER(gwn_stats)]),
    "gwn_eval_host": (ST, [P, C.POINTER(gwn_queries), P, P]),
    "gwn_eval_inside": (ST, [P, C.POINTER(gwn_queries), P, P]),
    "gwn_eval_batch": (ST, [P, C.POINTER(gwn_queries), I64, P, P, C.POINTER(gwn_plan), C.POINTER(gwn_stats)]),
    "gwn_batch_plan_get": (ST, [P, C.POINTER(I32), C.POINTER(I32)]),
    "gwn_backward": (ST, [P, C.POINTER(gwn_queries), P, P, P, P]),
    "gwn_eval_bruteforce": (ST, [P, C.POINTER(gwn_queries), P]),
    "gwn_eval_points_noalloc": (ST, [P, P, I64, P, P]),
    "gwn_eval_meshes": (ST, [P, P, C.POINTER(gwn_queries), I64, P, P, C.POINTER(gwn_plan), C.POINTER(gwn_stats)]),
    "gwn_meshes_plan_get": (ST, [P, C.POINTER(I32), C.POINTER(I32)]),
}

_lib = None


def load(path: str | None = None):
    """Load libgwn.so from the package's build folder.  Raises if it is
    missing: there is no fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libgwn.so not built ({path}); run paper_2408_04466_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class GwnError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}: {msg}")
        self.code = code


def check(code: int, where: str):
    if code != GWN_OK:
        raise GwnError(code, where, load().gwn_last_error().decode(errors="replace"))


def exported_symbols():
    return list(_SIGS)
