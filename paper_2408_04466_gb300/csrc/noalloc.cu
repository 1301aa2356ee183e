// noalloc.cu -- mesh evaluation that allocates no device memory.
//
// gwn_eval keeps the crossing counts of a call in a grow-only scratch buffer
// that it allocates on demand.  Some callers cannot allow that: services and
// plug-ins that reserve all device memory up front and must not call
// cudaMalloc afterwards (it can block on the whole device and can fail under
// memory pressure in the middle of a request).  This variant takes its
// scratch -- the per-query crossing counts between the traversal and the
// boundary-term kernel -- from a fixed array in the library's own device
// data, so a call allocates nothing.  The same array holds the boundary
// term's deferred-query list (indices of the queries its careful pass
// recomputes); the list's length lives in the context's preallocated counter.
//
// Limits and rules (also stated in include/gwn.h):
//   * at most GWN_NOALLOC_MAX_QUERIES (4,194,304) queries per call; the array
//     (two int32 entries per query) occupies 32 MiB on every GPU that loads
//     the library, until the process exits;
//   * query points must already be in device memory, and the mesh's
//     hierarchy must already be built for d (gwn_mesh_prepare);
//   * a call not under stream capture looks up the array's device address
//     (and on the first call loads its code module); the first call on a
//     device must come before any stream capture;
//   * every call shares the one array, whose contents persist between calls:
//     calls whose work overlaps on the GPU (different streams, or contexts on
//     the same device) race on it.  Serialise them.
#include <mutex>

#include <string.h>

#include "gwn_internal.h"

namespace gwn {

// [0, MAX): crossing counts of the current call; [MAX, 2 MAX): its deferred-
// query list.  Every entry read is written first in the same call, so no
// clearing is needed.
static __device__ __align__(256) int32_t g_noalloc_chi[2 * GWN_NOALLOC_MAX_QUERIES];

static std::mutex g_noalloc_mu;
static int32_t *g_noalloc_ptr[256];

// Device address of the array on `device` (current).  It is looked up again
// on every call that is not being captured into a CUDA graph, so a device
// reset or a new primary context between calls is picked up (the lookup
// allocates nothing).  A call under stream capture uses the address cached by
// the last uncaptured call on that device, and fails if there was none.
static gwn_status noalloc_scratch(int device, cudaStream_t stream, int32_t **out) {
    if (device < 0 || device >= 256) {
        set_error("gwn_eval_points_noalloc: device ordinal out of range");
        return GWN_E_INVALID;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &cs);
    if (e != cudaSuccess) return cuda_fail(e, "gwn_eval_points_noalloc: cudaStreamIsCapturing");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        int32_t *ptr = nullptr;
        e = cudaGetSymbolAddress((void **)&ptr, g_noalloc_chi);
        if (e != cudaSuccess) return cuda_fail(e, "gwn_eval_points_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[device] = ptr;
    } else if (!g_noalloc_ptr[device]) {
        set_error("gwn_eval_points_noalloc: the first call on a device must not be under stream capture");
        return GWN_E_INVALID;
    }
    *out = g_noalloc_ptr[device];
    return GWN_OK;
}

}  // namespace gwn

using namespace gwn;

extern "C" GWN_API gwn_status gwn_eval_points_noalloc(gwn_geom *g, const float *pts, int64_t n, const float d[3],
                                                      float *w_out) {
    if (!g || g->kind != GWN_GEOM_MESH || !d || n < 0 || (n > 0 && (!pts || !w_out))) {
        set_error("gwn_eval_points_noalloc: bad arguments");
        return GWN_E_INVALID;
    }
    if (n > GWN_NOALLOC_MAX_QUERIES) {
        set_error("gwn_eval_points_noalloc: more than 4,194,304 queries in one call; split the batch "
                  "(or use gwn_eval)");
        return GWN_E_INVALID;
    }
    if (!g->bvh.valid || memcmp(g->bvh.dkey, d, sizeof(float) * 3) != 0) {
        set_error("gwn_eval_points_noalloc: the mesh is not prepared for this direction; call "
                  "gwn_mesh_prepare(g, d) first (preparation allocates)");
        return GWN_E_INVALID;
    }
    gwn_ctx *ctx = g->ctx;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    int32_t *chi = nullptr;
    gwn_status s = noalloc_scratch(ctx->device, ctx->stream, &chi);
    if (s != GWN_OK) return s;
    if (n == 0) return GWN_OK;
    QuerySrc src;
    memset(&src, 0, sizeof(src));
    src.kind = GWN_QUERY_POINTS;
    src.dim = 3;
    src.pts = pts;
    src.n = n;
    e = launch_traverse(g->bvh, src, chi, chi + GWN_NOALLOC_MAX_QUERIES, ctx->d_defer_count, ctx->d_tpairs,
                        ctx->d_tpair_count, nullptr, nullptr, ctx->d_status, ctx->sm_count, ctx->stream,
                        g->crossing_index != GWN_INDEX_TREE);
    if (e != cudaSuccess) return cuda_fail(e, "gwn_eval_points_noalloc: traversal");
    e = launch_bterm3d(g->bseq, g->bvh.bframe, g->n_bseq, g->bvh.frame, make_frame64(d), src, chi, w_out, nullptr,
                       chi + GWN_NOALLOC_MAX_QUERIES, ctx->d_defer_count, nullptr, ctx->d_status, ctx->sm_count,
                       ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "gwn_eval_points_noalloc: boundary term");
    return GWN_OK;
}
