// api.cpp -- C ABI of the gwn library: contexts, geometry handles, host-side
// boundary extraction and monotone splitting, evaluation dispatch.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <cstdio>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "gwn_internal.h"

namespace gwn {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

gwn_status cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return e == cudaErrorMemoryAllocation ? GWN_E_OOM : GWN_E_CUDA;
}

void *arena_get(gwn_ctx *ctx, int slot, size_t bytes, cudaError_t *err) {
    Arena &a = ctx->scratch[slot];
    *err = cudaSuccess;
    if (bytes == 0) bytes = 16;
    if (a.bytes >= bytes) return a.ptr;
    if (a.ptr) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) { *err = e; return nullptr; }
        cudaFree(a.ptr);
        a.ptr = nullptr;
        a.bytes = 0;
    }
    size_t want = bytes + bytes / 4;
    cudaError_t e = cudaMalloc(&a.ptr, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        a.ptr = nullptr;
        *err = e;
        return nullptr;
    }
    a.bytes = want;
    return a.ptr;
}

// Frame of direction d: n = -d/|d|, e1 = normalize(h x n) for the coordinate
// axis h least aligned with n, e2 = n x e1 (so e1 x e2 = n), dh = d/|d|.
Frame make_frame(const float d[3]) {
    Frame f;
    double dd[3] = {d[0], d[1], d[2]};
    double len = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
    double dh[3] = {dd[0] / len, dd[1] / len, dd[2] / len};
    double n[3] = {-dh[0], -dh[1], -dh[2]};
    int k = 0;
    for (int i = 1; i < 3; i++)
        if (fabs(n[i]) < fabs(n[k])) k = i;
    double h[3] = {0, 0, 0};
    h[k] = 1.0;
    double e1[3] = {h[1] * n[2] - h[2] * n[1], h[2] * n[0] - h[0] * n[2], h[0] * n[1] - h[1] * n[0]};
    double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int i = 0; i < 3; i++) e1[i] /= l1;
    double e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0]};
    for (int i = 0; i < 3; i++) {
        f.e1[i] = (float)e1[i];
        f.e2[i] = (float)e2[i];
        f.n[i] = (float)n[i];
        f.dh[i] = (float)dh[i];
        f.d[i] = d[i];
    }
    return f;
}

Frame64 make_frame64(const float d[3]) {
    Frame64 f;
    double dd[3] = {d[0], d[1], d[2]};
    double len = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
    double dh[3] = {dd[0] / len, dd[1] / len, dd[2] / len};
    double n[3] = {-dh[0], -dh[1], -dh[2]};
    int k = 0;
    for (int i = 1; i < 3; i++)
        if (fabs(n[i]) < fabs(n[k])) k = i;
    double h[3] = {0, 0, 0};
    h[k] = 1.0;
    double e1[3] = {h[1] * n[2] - h[2] * n[1], h[2] * n[0] - h[0] * n[2], h[0] * n[1] - h[1] * n[0]};
    double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int i = 0; i < 3; i++) e1[i] /= l1;
    double e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0]};
    for (int i = 0; i < 3; i++) {
        f.e1[i] = e1[i];
        f.e2[i] = e2[i];
        f.n[i] = n[i];
        f.dh[i] = dh[i];
        f.dp[i] = 0.0;
    }
    for (int c = 0; c < 3; c++) {
        double e[3] = {0, 0, 0};
        e[c] = 1.0;
        double t = e[0] * dh[0] + e[1] * dh[1] + e[2] * dh[2];
        double q[3] = {e[0] - t * dh[0], e[1] - t * dh[1], e[2] - t * dh[2]};
        if (fabs(q[0]) + fabs(q[1]) + fabs(q[2]) > 1e-12) {
            for (int i = 0; i < 3; i++) f.dp[i] = q[i];
            break;
        }
    }
    return f;
}

// ---------------------------------------------------------------------------
// boundary extraction (host)
// ---------------------------------------------------------------------------
// Net multiplicity of every undirected edge {u < v}: (#u->v) - (#v->u) over
// the directed triangle edges i->j, j->k, k->i.  Nonzero pairs are boundary
// edges; one of multiplicity m is split into |m| unit edges in the direction
// of its sign.  Unit edges are chained into closed loops by walking unused
// out-edges from the smallest vertex that still has one; since every vertex
// has equal in- and out-degree, a walk can only stop at its start.

static gwn_status extract_boundary(const int32_t *F, int64_t nf, int64_t nv, BoundaryLoops &out) {
    out.off.assign(1, 0);
    out.vid.clear();
    if (nf == 0) return GWN_OK;
    // bucket directed edges by their smaller vertex (CSR)
    std::vector<int64_t> cnt(nv + 1, 0);
    for (int64_t t = 0; t < nf; t++)
        for (int k = 0; k < 3; k++) {
            int32_t a = F[3 * t + k], b = F[3 * t + (k + 1) % 3];
            if (a == b) continue;
            cnt[std::min(a, b) + 1]++;
        }
    for (int64_t v = 0; v < nv; v++) cnt[v + 1] += cnt[v];
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    std::vector<int32_t> other(cnt[nv]);
    std::vector<int8_t> sgn(cnt[nv]);
    for (int64_t t = 0; t < nf; t++)
        for (int k = 0; k < 3; k++) {
            int32_t a = F[3 * t + k], b = F[3 * t + (k + 1) % 3];
            if (a == b) continue;
            int32_t u = std::min(a, b), w = std::max(a, b);
            int64_t pos = fill[u]++;
            other[pos] = w;
            sgn[pos] = a < b ? 1 : -1;
        }
    // net multiplicities -> unit boundary edges (out-adjacency as CSR)
    std::vector<std::pair<int32_t, int32_t>> bedges;
    std::vector<std::pair<int32_t, int8_t>> tmp;
    for (int64_t u = 0; u < nv; u++) {
        int64_t lo = cnt[u], hi = cnt[u + 1];
        if (lo == hi) continue;
        tmp.clear();
        for (int64_t i = lo; i < hi; i++) tmp.emplace_back(other[i], sgn[i]);
        std::sort(tmp.begin(), tmp.end(),
                  [](const std::pair<int32_t, int8_t> &x, const std::pair<int32_t, int8_t> &y) {
                      return x.first < y.first;
                  });
        for (size_t i = 0; i < tmp.size();) {
            size_t j = i;
            int m = 0;
            while (j < tmp.size() && tmp[j].first == tmp[i].first) m += tmp[j++].second;
            for (int r = 0; r < m; r++) bedges.emplace_back((int32_t)u, tmp[i].first);
            for (int r = 0; r < -m; r++) bedges.emplace_back(tmp[i].first, (int32_t)u);
            i = j;
        }
    }
    return chain_unit_edges(bedges, nv, out);
}

// Unit edges are chained into closed loops by walking unused out-edges from
// the smallest vertex that still has one; since every vertex has equal in- and
// out-degree, a walk can only stop at its start.
gwn_status chain_unit_edges(std::vector<std::pair<int32_t, int32_t>> &bedges, int64_t nv, BoundaryLoops &out) {
    out.off.assign(1, 0);
    out.vid.clear();
    if (bedges.empty()) return GWN_OK;
    // the walk runs over the boundary's own vertices, renumbered in increasing
    // order (a monotone map, so "smallest vertex first" is unchanged)
    std::vector<int32_t> ids;
    ids.reserve(2 * bedges.size());
    for (auto &e : bedges) { ids.push_back(e.first); ids.push_back(e.second); }
    std::sort(ids.begin(), ids.end());
    ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
    for (auto &e : bedges) {
        e.first = (int32_t)(std::lower_bound(ids.begin(), ids.end(), e.first) - ids.begin());
        e.second = (int32_t)(std::lower_bound(ids.begin(), ids.end(), e.second) - ids.begin());
    }
    nv = (int64_t)ids.size();
    std::vector<int64_t> ooff(nv + 1, 0);
    for (auto &e : bedges) ooff[e.first + 1]++;
    for (int64_t v = 0; v < nv; v++) ooff[v + 1] += ooff[v];
    std::vector<int32_t> odst(bedges.size());
    {
        std::vector<int64_t> f2(ooff.begin(), ooff.end() - 1);
        std::sort(bedges.begin(), bedges.end());
        for (auto &e : bedges) odst[f2[e.first]++] = e.second;
    }
    std::vector<int64_t> next(ooff.begin(), ooff.end() - 1);   // next unused out-edge
    int64_t used = 0, total = (int64_t)bedges.size();
    for (int64_t s = 0; s < nv && used < total; s++) {
        while (next[s] < ooff[s + 1]) {
            int32_t cur = (int32_t)s;
            int64_t guard = 0;
            do {
                if (next[cur] >= ooff[cur + 1] || guard++ > total) {
                    set_error("boundary extraction: unbalanced boundary (internal error)");
                    return GWN_E_INTERNAL;
                }
                out.vid.push_back(cur);
                int32_t nx = odst[next[cur]++];
                used++;
                cur = nx;
            } while (cur != (int32_t)s);
            out.off.push_back((int64_t)out.vid.size());
        }
    }
    for (auto &v : out.vid) v = ids[v];
    return GWN_OK;
}

// ---------------------------------------------------------------------------
// 2D: y-monotone split of a cubic (host)
// ---------------------------------------------------------------------------
// dy/du of B(u) = sum P_k b_k(u) is 3 [d0 (1-u)^2 + 2 d1 u (1-u) + d2 u^2] with
// d_k = y_{k+1} - y_k; its roots in (0, 1) split [0, 1] into monotone pieces.
static int monotone_split(const double c[8], double u[6]) {
    double d0 = c[3] - c[1], d1 = c[5] - c[3], d2 = c[7] - c[5];
    double A = d0 - 2 * d1 + d2, B = 2 * (d1 - d0), C = d0;
    double r[2];
    int nr = 0;
    double scale = fabs(A) + fabs(B) + fabs(C);
    if (scale == 0.0) {
        u[0] = 0.0; u[1] = 1.0;
        return 1;
    }
    if (fabs(A) <= 1e-14 * scale) {
        if (B != 0.0) r[nr++] = -C / B;
    } else {
        double disc = B * B - 4 * A * C;
        if (disc > 0) {
            double sq = sqrt(disc);
            double q = -0.5 * (B + (B >= 0 ? sq : -sq));
            r[nr++] = q / A;
            if (q != 0.0) r[nr++] = C / q;
        }
    }
    if (nr == 2 && r[0] > r[1]) std::swap(r[0], r[1]);
    double cuts[4];
    int nc = 0;
    cuts[nc++] = 0.0;
    for (int i = 0; i < nr; i++)
        if (r[i] > 0.0 && r[i] < 1.0 && r[i] > cuts[nc - 1]) cuts[nc++] = r[i];
    cuts[nc++] = 1.0;
    int n = 0;
    for (int i = 0; i + 1 < nc; i++) {
        u[2 * n] = cuts[i];
        u[2 * n + 1] = cuts[i + 1];
        n++;
    }
    return n;
}

static double bez_y(const double c[8], double u) {
    if (u == 0.0) return c[1];
    if (u == 1.0) return c[7];
    double v = 1.0 - u;
    return v * v * v * c[1] + 3 * u * v * v * c[3] + 3 * u * u * v * c[5] + u * u * u * c[7];
}

}  // namespace gwn

using namespace gwn;

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

extern "C" {

GWN_API const char *gwn_version(void) { return "gwn-oneshot 1.0 (sm_103a)"; }

GWN_API const char *gwn_last_error(void) { return g_last_error.c_str(); }

GWN_API gwn_status gwn_ctx_create(gwn_ctx **out, int device, void *cuda_stream) {
    if (!out) { set_error("gwn_ctx_create: out is NULL"); return GWN_E_INVALID; }
    *out = nullptr;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) { set_error("gwn_ctx_create: no such device"); return GWN_E_INVALID; }
    CK(cudaSetDevice(device), "cudaSetDevice");
    gwn_ctx *c = new (std::nothrow) gwn_ctx();
    if (!c) { set_error("gwn_ctx_create: out of host memory"); return GWN_E_OOM; }
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_cnt, sizeof(unsigned long long) * CNT_NUM);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_defer_count, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tpairs, sizeof(int2) * GWN_TPAIR_CAP);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tpair_count, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_work_counter, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_cert, sizeof(int4) * 2 * GWN_CERT_CAP);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_cert_count, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_cnt, 0, sizeof(unsigned long long) * CNT_NUM);
    for (int i = 0; i < 8 && e == cudaSuccess; i++) e = cudaEventCreate(&c->ev[i]);
    if (e != cudaSuccess) {
        gwn_status s = cuda_fail(e, "gwn_ctx_create");
        gwn_ctx_destroy(c);
        return s;
    }
    c->events = true;
    *out = c;
    return GWN_OK;
}

GWN_API gwn_status gwn_ctx_set_stream(gwn_ctx *ctx, void *cuda_stream) {
    if (!ctx) { set_error("gwn_ctx_set_stream: NULL ctx"); return GWN_E_INVALID; }
    ctx->stream = (cudaStream_t)cuda_stream;
    return GWN_OK;
}

GWN_API gwn_status gwn_ctx_check(gwn_ctx *ctx) {
    if (!ctx) { set_error("gwn_ctx_check: NULL ctx"); return GWN_E_INVALID; }
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    int st = 0;
    CK(cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost), "read status");
    CK(cudaMemset(ctx->d_status, 0, sizeof(int)), "clear status");
    if (st & ST_STACK_OVERFLOW) { set_error("traversal stack overflow"); return GWN_E_STACK_OVERFLOW; }
    if (st & ST_TIMEOUT) { set_error("device iteration limit reached"); return GWN_E_TIMEOUT; }
    if (st & ST_EXPANSION_OVERFLOW) { set_error("exact predicate expansion overflow"); return GWN_E_INTERNAL; }
    if (st & ST_BAD_INPUT) { set_error("invalid input detected on device"); return GWN_E_INVALID; }
    if (st & ST_CERT_OVERFLOW) {
        set_error("2D certification list overflow: crossing counts of queries within float rounding of a curve "
                  "may be off");
        return GWN_E_INTERNAL;
    }
    return GWN_OK;
}

static std::mutex g_ctx_life_mu;

// release the context's resources (no geometry refers to it any more)
static void ctx_release(gwn_ctx *ctx) {
    if (cudaSetDevice(ctx->device) == cudaErrorCudartUnloading) {   // process exit: the driver reclaims memory
        delete ctx;
        return;
    }
    cudaStreamSynchronize(ctx->stream);
    for (auto &a : ctx->scratch)
        if (a.ptr) cudaFree(a.ptr);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->d_cnt) cudaFree(ctx->d_cnt);
    if (ctx->d_defer_count) cudaFree(ctx->d_defer_count);
    if (ctx->d_tpairs) cudaFree(ctx->d_tpairs);
    if (ctx->d_tpair_count) cudaFree(ctx->d_tpair_count);
    if (ctx->d_work_counter) cudaFree(ctx->d_work_counter);
    if (ctx->mesh_batch_cache) mesh_batch_cache_free(ctx->mesh_batch_cache);
    if (ctx->d_cert) cudaFree(ctx->d_cert);
    if (ctx->d_cert_count) cudaFree(ctx->d_cert_count);
    for (auto &c : ctx->axis_cache)
        if (c.dev) cudaFree(c.dev);
    if (ctx->events)
        for (int i = 0; i < 8; i++) cudaEventDestroy(ctx->ev[i]);
    delete ctx;
}

GWN_API void gwn_ctx_destroy(gwn_ctx *ctx) {
    if (!ctx) return;
    bool now;
    {
        std::lock_guard<std::mutex> lk(g_ctx_life_mu);
        ctx->destroy_requested = true;
        now = ctx->geom_refs == 0;
    }
    if (now) ctx_release(ctx);
}

// a new geometry on ctx / a geometry of ctx destroyed
static void ctx_ref(gwn_ctx *ctx) {
    std::lock_guard<std::mutex> lk(g_ctx_life_mu);
    ctx->geom_refs++;
}

}  // extern "C"

// for geometry constructors in other translation units
void gwn::ctx_add_geometry(gwn_ctx *ctx) { ctx_ref(ctx); }

extern "C" {

static void ctx_unref(gwn_ctx *ctx) {
    bool now;
    {
        std::lock_guard<std::mutex> lk(g_ctx_life_mu);
        now = --ctx->geom_refs == 0 && ctx->destroy_requested;
    }
    if (now) ctx_release(ctx);
}

GWN_API gwn_status gwn_boundary_extract_host(const int32_t *F, int64_t nf, int64_t nv, int64_t *loop_offsets,
                                             int32_t *vert_ids, int64_t *n_loops, int64_t *n_edges) {
    if ((nf > 0 && !F) || nf < 0 || nv < 0) { set_error("gwn_boundary_extract_host: bad arguments"); return GWN_E_INVALID; }
    for (int64_t i = 0; i < 3 * nf; i++)
        if (F[i] < 0 || F[i] >= nv) { set_error("gwn_boundary_extract_host: face index out of range"); return GWN_E_INVALID; }
    BoundaryLoops bl;
    gwn_status s;
    try {
        s = extract_boundary(F, nf, nv, bl);
    } catch (const std::bad_alloc &) {
        set_error("gwn_boundary_extract_host: out of host memory");
        return GWN_E_OOM;
    }
    if (s != GWN_OK) return s;
    if (n_loops) *n_loops = (int64_t)bl.off.size() - 1;
    if (n_edges) *n_edges = (int64_t)bl.vid.size();
    if (loop_offsets) memcpy(loop_offsets, bl.off.data(), sizeof(int64_t) * bl.off.size());
    if (vert_ids && !bl.vid.empty()) memcpy(vert_ids, bl.vid.data(), sizeof(int32_t) * bl.vid.size());
    return GWN_OK;
}

GWN_API gwn_status gwn_bezier_monotone_split_host(const double ctrl[8], double u_out[6], int32_t *n_out) {
    if (!ctrl || !u_out || !n_out) { set_error("gwn_bezier_monotone_split_host: NULL argument"); return GWN_E_INVALID; }
    *n_out = monotone_split(ctrl, u_out);
    return GWN_OK;
}

static void free_geom_device(gwn_geom *g) {
    if (g->dV) cudaFree(g->dV);
    if (g->dF) cudaFree(g->dF);
    if (g->bseq) cudaFree(g->bseq);
    if (g->bseq_vid) cudaFree(g->bseq_vid);
    if (g->d_edge_rec) cudaFree(g->d_edge_rec);
    if (g->d_bvert) cudaFree(g->d_bvert);
    if (g->d_brec_off) cudaFree(g->d_brec_off);
    if (g->d_brecs) cudaFree(g->d_brecs);
    bvh_free(g->bvh);
    ChainSet &cs = g->cs;
    if (cs.ctrl) cudaFree(cs.ctrl);
    if (cs.chain_off) cudaFree(cs.chain_off);
    if (cs.piece_y) cudaFree(cs.piece_y);
    if (cs.piece_yT && cs.piece_yT != (void *)cs.piece_y) cudaFree(cs.piece_yT);
    if (cs.piece_xT) cudaFree(cs.piece_xT);
    if (cs.piece_rec) cudaFree(cs.piece_rec);
    if (cs.piece_seg) cudaFree(cs.piece_seg);
    if (cs.piece_u) cudaFree(cs.piece_u);
    if (cs.piece_part) cudaFree(cs.piece_part);
    if (cs.piece_eps) cudaFree(cs.piece_eps);
    if (cs.bucket_off) cudaFree(cs.bucket_off);
    if (cs.bucket_idx) cudaFree(cs.bucket_idx);
    patches_free(g->ps);
}

GWN_API void gwn_geom_destroy(gwn_geom *g) {
    if (!g) return;
    bool unloading = false;
    if (g->ctx) {
        unloading = cudaSetDevice(g->ctx->device) == cudaErrorCudartUnloading;
        if (!unloading) cudaStreamSynchronize(g->ctx->stream);
    }
    if (!unloading) {                      // at process exit the driver reclaims device memory
        if (g->batch_cache) batch_cache_free(g->batch_cache);
        free_geom_device(g);
    }
    gwn_ctx *ctx = g->ctx;
    delete g;
    if (ctx) ctx_unref(ctx);
}

GWN_API gwn_status gwn_mesh_create(gwn_ctx *ctx, const float *V, int64_t nv, const int32_t *F, int64_t nf,
                                   int mem_kind, gwn_geom **out) {
    if (!out) { set_error("gwn_mesh_create: out is NULL"); return GWN_E_INVALID; }
    *out = nullptr;
    if (!ctx || nv < 0 || nf < 0 || (nv > 0 && !V) || (nf > 0 && !F) ||
        (mem_kind != GWN_MEM_HOST && mem_kind != GWN_MEM_DEVICE)) {
        set_error("gwn_mesh_create: bad arguments");
        return GWN_E_INVALID;
    }
    if (nv > 0x7fffffff || nf > 0x7fffffff / 3) { set_error("gwn_mesh_create: mesh too large"); return GWN_E_INVALID; }
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    std::unique_ptr<gwn_geom> g(new (std::nothrow) gwn_geom());
    if (!g) { set_error("gwn_mesh_create: out of host memory"); return GWN_E_OOM; }
    g->ctx = ctx;
    g->kind = GWN_GEOM_MESH;
    g->dtype = GWN_F32;
    g->nv = nv;
    g->nf = nf;
    cudaStream_t st = ctx->stream;
    // upload, then checks and boundary edges on the device (the intake
    // synchronises, so the caller's buffers are free again on return)
    const cudaMemcpyKind kind = mem_kind == GWN_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaError_t e = cudaSuccess;
    if (nv) e = cudaMalloc(&g->dV, sizeof(float) * 3 * nv);
    if (e == cudaSuccess && nf) e = cudaMalloc(&g->dF, sizeof(int32_t) * 3 * nf);
    if (e == cudaSuccess && nv) e = cudaMemcpyAsync(g->dV, V, sizeof(float) * 3 * nv, kind, st);
    if (e == cudaSuccess && nf) e = cudaMemcpyAsync(g->dF, F, sizeof(int32_t) * 3 * nf, kind, st);
    if (e != cudaSuccess) {
        free_geom_device(g.get());
        return cuda_fail(e, "gwn_mesh_create");
    }
    BoundaryLoops bl;
    std::vector<int32_t> code;
    gwn_status s;
    try {
        std::vector<std::pair<int32_t, int32_t>> bedges;
        s = mesh_intake_device(ctx, g->dV, nv, g->dF, nf, bedges);
        if (s == GWN_OK) s = chain_unit_edges(bedges, nv, bl);
        if (s == GWN_OK) {
            // loop sequence records: each loop's vertices, then its first again
            int64_t L = (int64_t)bl.off.size() - 1;
            code.reserve(bl.vid.size() + L);
            for (int64_t j = 0; j < L; j++)
                for (int64_t i = bl.off[j]; i <= bl.off[j + 1]; i++) {
                    int32_t v = bl.vid[i < bl.off[j + 1] ? i : bl.off[j]];
                    code.push_back(i == bl.off[j] ? ~v : v);
                }
        }
    } catch (const std::bad_alloc &) {
        set_error("gwn_mesh_create: out of host memory");
        s = GWN_E_OOM;
    }
    if (s != GWN_OK) {
        free_geom_device(g.get());
        return s;
    }
    g->loop_off = bl.off;
    g->loop_vid = bl.vid;
    g->n_bseq = (int64_t)code.size();
    if (g->n_bseq) {
        int32_t *dcode = (int32_t *)arena_get(ctx, 6, sizeof(int32_t) * g->n_bseq, &e);
        if (!dcode) {
            free_geom_device(g.get());
            return cuda_fail(e, "gwn_mesh_create");
        }
        e = cudaMalloc(&g->bseq, sizeof(float4) * g->n_bseq);
        if (e == cudaSuccess) e = cudaMalloc(&g->bseq_vid, sizeof(int32_t) * g->n_bseq);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dcode, code.data(), sizeof(int32_t) * g->n_bseq, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = launch_bseq(g->dV, dcode, g->n_bseq, g->bseq, g->bseq_vid, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the host copy of code goes out of scope
        if (e != cudaSuccess) {
            free_geom_device(g.get());
            return cuda_fail(e, "gwn_mesh_create");
        }
    }
    ctx_ref(ctx);
    *out = g.release();
    return GWN_OK;
}

GWN_API gwn_status gwn_mesh_set_index(gwn_geom *g, int index) {
    if (!g || g->kind != GWN_GEOM_MESH || (index != GWN_INDEX_AUTO && index != GWN_INDEX_TREE)) {
        set_error("gwn_mesh_set_index: bad arguments");
        return GWN_E_INVALID;
    }
    g->crossing_index = index;
    return GWN_OK;
}

GWN_API gwn_status gwn_mesh_prepare(gwn_geom *g, const float d[3]) {
    if (!g || g->kind != GWN_GEOM_MESH || !d) { set_error("gwn_mesh_prepare: bad arguments"); return GWN_E_INVALID; }
    if (!isfinite(d[0]) || !isfinite(d[1]) || !isfinite(d[2]) || (d[0] == 0.f && d[1] == 0.f && d[2] == 0.f)) {
        set_error("gwn_mesh_prepare: direction must be finite and nonzero");
        return GWN_E_INVALID;
    }
    if (g->bvh.valid && memcmp(g->bvh.dkey, d, sizeof(float) * 3) == 0) return GWN_OK;
    CK(cudaSetDevice(g->ctx->device), "cudaSetDevice");
    Frame fr = make_frame(d);
    cudaError_t e = bvh_build(g, fr, g->ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "LBVH build");
    return GWN_OK;
}

}  // extern "C"

namespace {

// Index for 2D point queries (one +x ray per query, no ray reuse): the
// y-range [ymin, ymax] of all pieces is cut into buckets; a piece is listed in
// every bucket its y-range touches, widened by one bucket on each side so that
// the rounding of the bucket map cannot drop it (the exact half-open y-test is
// made per piece on the device).  Each piece also gets a conservative x-range,
// the x-range of its segment's control points (convex hull property).
template <typename T>
static int bucket_of(T y, T y0, T inv_h, int nb) {
    T v = (y - y0) * inv_h;
    if (!(v >= T(0))) return 0;
    if (v >= T(nb)) return nb - 1;
    int b = (int)v;
    return b < nb ? b : nb - 1;
}

static cudaError_t build_point_index(ChainSet &cs, const std::vector<double> &P, const std::vector<int64_t> &pseg,
                                     const std::vector<double> &py, int dtype) {
    const int64_t np = cs.n_pieces;
    const size_t npa = (size_t)std::max<int64_t>(np, 1);
    std::vector<double> xr(2 * npa, 0.0);
    double ylo = 0.0, yhi = 0.0;
    for (int64_t p = 0; p < np; p++) {
        const double *c = &P[2 * pseg[p]];
        double x0 = c[0], x1 = c[0];
        for (int k = 1; k < 4; k++) {
            x0 = std::min(x0, c[2 * k]);
            x1 = std::max(x1, c[2 * k]);
        }
        xr[2 * p] = x0;
        xr[2 * p + 1] = x1;
        double a = std::min(py[2 * p], py[2 * p + 1]), b = std::max(py[2 * p], py[2 * p + 1]);
        if (p == 0 || a < ylo) ylo = a;
        if (p == 0 || b > yhi) yhi = b;
    }
    // about two pieces per bucket, fewer buckets while tall pieces would make
    // the index exceed 2^26 entries
    int nb = (int)std::min<int64_t>(std::max<int64_t>(np / 2, 1), 1 << 22);
    double span = yhi - ylo;
    double inv_h = 0.0;
    std::vector<int32_t> b0(npa), b1(npa);
    for (;;) {
        inv_h = span > 0.0 ? (double)nb / span : 0.0;
        int64_t total = 0;
        for (int64_t p = 0; p < np; p++) {
            // bucket range of every piece, in the chain precision (the device map)
            double a = std::min(py[2 * p], py[2 * p + 1]), b = std::max(py[2 * p], py[2 * p + 1]);
            int lo, hi;
            if (dtype == GWN_F64) {
                lo = bucket_of<double>(a, ylo, inv_h, nb);
                hi = bucket_of<double>(b, ylo, inv_h, nb);
            } else {
                lo = bucket_of<float>((float)a, (float)ylo, (float)inv_h, nb);
                hi = bucket_of<float>((float)b, (float)ylo, (float)inv_h, nb);
            }
            b0[p] = std::max(lo - 1, 0);
            b1[p] = std::min(hi + 1, nb - 1);
            total += b1[p] - b0[p] + 1;
        }
        if (total <= (int64_t(1) << 26) || nb == 1) break;
        nb = std::max(nb / 4, 1);
    }
    cs.n_buckets = nb;
    cs.bucket_y0 = ylo;
    cs.bucket_inv_h = inv_h;
    std::vector<int32_t> cnt(nb + 1, 0);
    for (int64_t p = 0; p < np; p++)
        for (int k = b0[p]; k <= b1[p]; k++) cnt[k + 1]++;
    for (int k = 0; k < nb; k++) cnt[k + 1] += cnt[k];
    std::vector<int32_t> idx(std::max<int32_t>(cnt[nb], 1));
    std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t p = 0; p < np; p++)
        for (int k = b0[p]; k <= b1[p]; k++) idx[fill[k]++] = (int32_t)p;
    size_t esz = dtype == GWN_F64 ? 8 : 4;
    std::vector<char> xt(esz * 2 * npa);
    for (size_t i = 0; i < 2 * npa; i++) {
        if (dtype == GWN_F64) ((double *)xt.data())[i] = xr[i];
        else ((float *)xt.data())[i] = (float)xr[i];
    }
    // float32 chains: a conservative x-range after rounding (round outward)
    if (dtype == GWN_F32)
        for (size_t p = 0; p < npa; p++) {
            float *f = (float *)xt.data();
            f[2 * p] = nextafterf(f[2 * p], -INFINITY);
            f[2 * p + 1] = nextafterf(f[2 * p + 1], INFINITY);
        }
    cudaError_t e = cudaMalloc(&cs.piece_xT, xt.size());
    if (e == cudaSuccess) e = cudaMemcpy(cs.piece_xT, xt.data(), xt.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&cs.bucket_off, sizeof(int32_t) * (nb + 1));
    if (e == cudaSuccess) e = cudaMemcpy(cs.bucket_off, cnt.data(), sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&cs.bucket_idx, sizeof(int32_t) * idx.size());
    if (e == cudaSuccess) e = cudaMemcpy(cs.bucket_idx, idx.data(), sizeof(int32_t) * idx.size(), cudaMemcpyHostToDevice);
    return e;
}

}  // namespace

extern "C" {

GWN_API gwn_status gwn_bezier2d_create(gwn_ctx *ctx, const void *ctrl, int dtype, const int64_t *chain_offsets,
                                       int64_t n_chains, int mem_kind, gwn_geom **out) {
    if (!out) { set_error("gwn_bezier2d_create: out is NULL"); return GWN_E_INVALID; }
    *out = nullptr;
    if (!ctx || !ctrl || !chain_offsets || n_chains <= 0 || (dtype != GWN_F32 && dtype != GWN_F64) ||
        (mem_kind != GWN_MEM_HOST && mem_kind != GWN_MEM_DEVICE)) {
        set_error("gwn_bezier2d_create: bad arguments");
        return GWN_E_INVALID;
    }
    int64_t n_ctrl = chain_offsets[n_chains];
    if (chain_offsets[0] != 0 || n_ctrl <= 0 || n_ctrl > 0x7fffffff) {
        set_error("gwn_bezier2d_create: bad chain offsets");
        return GWN_E_INVALID;
    }
    for (int64_t c = 0; c < n_chains; c++) {
        int64_t m = chain_offsets[c + 1] - chain_offsets[c];
        if (m < 4 || (m - 1) % 3 != 0) {
            set_error("gwn_bezier2d_create: each chain needs 3k+1 control points, k >= 1");
            return GWN_E_INVALID;
        }
    }
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    size_t esz = dtype == GWN_F64 ? 8 : 4;
    std::vector<char> raw(esz * 2 * n_ctrl);
    if (mem_kind == GWN_MEM_HOST) memcpy(raw.data(), ctrl, raw.size());
    else CK(cudaMemcpy(raw.data(), ctrl, raw.size(), cudaMemcpyDeviceToHost), "copy ctrl");
    std::vector<double> P(2 * n_ctrl);
    for (int64_t i = 0; i < 2 * n_ctrl; i++)
        P[i] = dtype == GWN_F64 ? ((const double *)raw.data())[i] : (double)((const float *)raw.data())[i];
    for (double v : P)
        if (!isfinite(v)) { set_error("gwn_bezier2d_create: non-finite control point"); return GWN_E_INVALID; }
    std::unique_ptr<gwn_geom> g(new (std::nothrow) gwn_geom());
    if (!g) { set_error("gwn_bezier2d_create: out of host memory"); return GWN_E_OOM; }
    g->ctx = ctx;
    g->kind = GWN_GEOM_BEZIER2D;
    g->dtype = dtype;
    ChainSet &cs = g->cs;
    cs.dtype = dtype;
    cs.n_chains = n_chains;
    cs.n_ctrl = n_ctrl;
    cs.h_chain_off.assign(chain_offsets, chain_offsets + n_chains + 1);
    std::vector<int64_t> pseg;
    std::vector<double> pu, py;
    std::vector<int32_t> pch;
    cs.h_chain_piece_off.assign(1, 0);
    // a chain's pieces are kept in order of their lowest y (in the chain's
    // precision), with the running maximum of their highest y: the pieces
    // that can reach a band of rows are then one contiguous run
    // An end of a piece strictly inside (0, 1) is an extremum of y: its value
    // y(u) is rounded (to the chain's precision, after a float64 evaluation),
    // so the row test of the two pieces that share it is uncertain within
    // eps of it; eps bounds |stored value - curve value| there (the float64
    // evaluation error of B_y is below 4 ulps of sum |P_y|).  Ends at u = 0 or
    // 1 are control points, stored exactly.
    struct PieceH { int64_t seg; double u0, u1, y0, y1, lo_t, eps0, eps1; int64_t id, part0, part1; };
    auto to_t = [dtype](double v) { return dtype == GWN_F64 ? v : (double)(float)v; };
    std::vector<int2> ppart;
    std::vector<double> peps;
    int64_t next_id = 0;
    for (int64_t c = 0; c < n_chains; c++) {
        std::vector<PieceH> ch;
        for (int64_t i = chain_offsets[c]; i + 3 < chain_offsets[c + 1]; i += 3) {
            double cc[8];
            for (int k = 0; k < 8; k++) cc[k] = P[2 * i + k];
            double u[6];
            int np = monotone_split(cc, u);
            cs.n_seg++;
            const double sy = fabs(cc[1]) + fabs(cc[3]) + fabs(cc[5]) + fabs(cc[7]);
            auto end_eps = [&](double uu, double y) {
                if (uu <= 0.0 || uu >= 1.0) return 0.0;
                cs.eps_abs = std::max(cs.eps_abs, 8e-15 * sy);
                return fabs(to_t(y) - y) + 4e-15 * sy;
            };
            int64_t prev_id = -1;          // the last kept piece of this segment
            double prev_u1 = -1.0;
            for (int k = 0; k < np; k++) {
                double y0 = bez_y(cc, u[2 * k]), y1 = bez_y(cc, u[2 * k + 1]);
                if (y0 == y1) { prev_id = -1; continue; }   // flat piece: never crossed by the half-open rule
                PieceH h{i, u[2 * k], u[2 * k + 1], y0, y1, to_t(std::min(y0, y1)), end_eps(u[2 * k], y0),
                         end_eps(u[2 * k + 1], y1), next_id++, -1, -1};
                if (prev_id >= 0 && prev_u1 == h.u0 && h.eps0 > 0.0) {
                    h.part0 = prev_id;
                    ch.back().part1 = h.id;
                }
                ch.push_back(h);
                prev_id = h.id;
                prev_u1 = h.u1;
            }
        }
        std::stable_sort(ch.begin(), ch.end(), [](const PieceH &a, const PieceH &b) { return a.lo_t < b.lo_t; });
        // partner ids -> indices in the sorted order (partners share a segment,
        // hence a chain)
        std::map<int64_t, int64_t> where;
        for (size_t k = 0; k < ch.size(); k++) where[ch[k].id] = (int64_t)pch.size() + (int64_t)k;
        double hmax = -INFINITY;
        for (const PieceH &q : ch) {
            pseg.push_back(q.seg);
            pu.push_back(q.u0);
            pu.push_back(q.u1);
            py.push_back(q.y0);
            py.push_back(q.y1);
            pch.push_back((int32_t)c);
            ppart.push_back(make_int2(q.part0 >= 0 ? (int)where[q.part0] : -1, q.part1 >= 0 ? (int)where[q.part1] : -1));
            peps.push_back(q.eps0);
            peps.push_back(q.eps1);
            // the run of pieces a block of rows can reach is widened by eps, so
            // a row just past a rounded extremum still sees both its pieces
            hmax = std::max(hmax, to_t(std::max(q.y0, q.y1) + std::max(q.eps0, q.eps1)));
            cs.h_piece_lo.push_back(q.lo_t);
            cs.h_piece_hmax.push_back(hmax);
        }
        cs.h_chain_piece_off.push_back((int64_t)pch.size());
    }
    cs.n_pieces = (int64_t)pch.size();
    cudaError_t e = cudaMalloc(&cs.ctrl, raw.size());
    if (e == cudaSuccess) e = cudaMemcpy(cs.ctrl, raw.data(), raw.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&cs.chain_off, sizeof(int64_t) * (n_chains + 1));
    if (e == cudaSuccess)
        e = cudaMemcpy(cs.chain_off, chain_offsets, sizeof(int64_t) * (n_chains + 1), cudaMemcpyHostToDevice);
    size_t np = (size_t)std::max<int64_t>(cs.n_pieces, 1);
    if (e == cudaSuccess) e = cudaMalloc(&cs.piece_y, sizeof(double) * 2 * np);
    if (e == cudaSuccess && cs.n_pieces)
        e = cudaMemcpy(cs.piece_y, py.data(), sizeof(double) * 2 * cs.n_pieces, cudaMemcpyHostToDevice);
    // the kernels read the piece tables in the chain's precision
    if (e == cudaSuccess && dtype == GWN_F64) {
        cs.piece_yT = cs.piece_y;
    } else if (e == cudaSuccess) {
        std::vector<float> fy(py.begin(), py.end());
        fy.resize(2 * np);
        e = cudaMalloc(&cs.piece_yT, sizeof(float) * 2 * np);
        if (e == cudaSuccess) e = cudaMemcpy(cs.piece_yT, fy.data(), sizeof(float) * 2 * np, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {        // per-piece records for the row kernel
        // the piece [u0, u1] reparametrised to t in [0, 1], u = u0 + t h, in
        // power form: for B(u) = c3 u^3 + c2 u^2 + c1 u + c0 (c0 = P0,
        // c1 = 3 (P1 - P0), c2 = 3 (P2 - 2 P1 + P0), c3 = P3 - 3 P2 + 3 P1 - P0),
        // B(u0 + t h) = a3 t^3 + a2 t^2 + a1 t + a0 with a3 = c3 h^3,
        // a2 = (3 c3 u0 + c2) h^2, a1 = (3 c3 u0^2 + 2 c2 u0 + c1) h, a0 = B(u0).
        // Record: x3 x2 x1 x0, y3 y2 y1 y(u0), 3 y3, 2 y2, y(u1), 0.
        std::vector<double> rec(12 * np, 0.0);
        for (int64_t q = 0; q < cs.n_pieces; q++) {
            const double *cc = &P[2 * pseg[q]];
            const double u0 = pu[2 * q], h = pu[2 * q + 1] - pu[2 * q];
            double a[2][4];
            for (int d = 0; d < 2; d++) {
                const double p0 = cc[d], p1 = cc[2 + d], p2 = cc[4 + d], p3 = cc[6 + d];
                const double c1 = 3.0 * (p1 - p0), c2 = 3.0 * (p2 - 2.0 * p1 + p0), c3 = p3 - 3.0 * p2 + 3.0 * p1 - p0;
                a[d][0] = c3 * h * h * h;
                a[d][1] = (3.0 * c3 * u0 + c2) * h * h;
                a[d][2] = ((3.0 * c3 * u0 + 2.0 * c2) * u0 + c1) * h;
                a[d][3] = ((c3 * u0 + c2) * u0 + c1) * u0 + p0;
            }
            double *r = &rec[12 * q];
            for (int k = 0; k < 4; k++) r[k] = a[0][k];
            r[4] = a[1][0];
            r[5] = a[1][1];
            r[6] = a[1][2];
            r[7] = py[2 * q];            // y(u0), the value the half-open row test uses
            r[8] = 3.0 * a[1][0];
            r[9] = 2.0 * a[1][1];
            r[10] = py[2 * q + 1];       // y(u1)
        }
        size_t bytes = esz * rec.size();
        e = cudaMalloc(&cs.piece_rec, bytes);
        if (e == cudaSuccess && dtype == GWN_F64) e = cudaMemcpy(cs.piece_rec, rec.data(), bytes, cudaMemcpyHostToDevice);
        else if (e == cudaSuccess) {
            std::vector<float> fr(rec.begin(), rec.end());
            e = cudaMemcpy(cs.piece_rec, fr.data(), bytes, cudaMemcpyHostToDevice);
        }
    }
    if (e == cudaSuccess) {        // per-piece data of the float64 certification
        std::vector<double2> pu2(np);
        for (int64_t q = 0; q < cs.n_pieces; q++) pu2[q] = make_double2(pu[2 * q], pu[2 * q + 1]);
        std::vector<int64_t> ps(pseg.begin(), pseg.end());
        ps.resize(np, 0);
        ppart.resize(np, make_int2(-1, -1));
        e = cudaMalloc(&cs.piece_seg, sizeof(int64_t) * np);
        if (e == cudaSuccess) e = cudaMemcpy(cs.piece_seg, ps.data(), sizeof(int64_t) * np, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&cs.piece_u, sizeof(double2) * np);
        if (e == cudaSuccess) e = cudaMemcpy(cs.piece_u, pu2.data(), sizeof(double2) * np, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&cs.piece_part, sizeof(int2) * np);
        if (e == cudaSuccess) e = cudaMemcpy(cs.piece_part, ppart.data(), sizeof(int2) * np, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&cs.piece_eps, esz * 2 * np);
        if (e == cudaSuccess) {
            peps.resize(2 * np, 0.0);
            if (dtype == GWN_F64) {
                e = cudaMemcpy(cs.piece_eps, peps.data(), esz * 2 * np, cudaMemcpyHostToDevice);
            } else {        // rounded up, so the float bound still covers the double one
                std::vector<float> fe(2 * np);
                for (size_t k = 0; k < fe.size(); k++) {
                    float f = (float)peps[k];
                    fe[k] = (double)f < peps[k] ? nextafterf(f, INFINITY) : f;
                }
                e = cudaMemcpy(cs.piece_eps, fe.data(), esz * 2 * np, cudaMemcpyHostToDevice);
            }
        }
    }
    if (e == cudaSuccess) e = build_point_index(cs, P, pseg, py, dtype);
    if (e != cudaSuccess) {
        free_geom_device(g.get());
        return cuda_fail(e, "gwn_bezier2d_create");
    }
    ctx_ref(ctx);
    *out = g.release();
    return GWN_OK;
}

GWN_API gwn_status gwn_geom_info_get(const gwn_geom *g, gwn_geom_info *out) {
    if (!g || !out) { set_error("gwn_geom_info_get: NULL argument"); return GWN_E_INVALID; }
    memset(out, 0, sizeof(*out));
    out->kind = g->kind;
    out->dtype = g->dtype;
    if (g->kind == GWN_GEOM_MESH) {
        out->n_vertices = g->nv;
        out->n_primitives = g->nf;
        out->n_boundary_edges = (int64_t)g->loop_vid.size();
        out->n_loops = (int64_t)g->loop_off.size() - 1;
        if (g->bvh.valid && g->bvh.n_bin_entries > 0) {
            out->n_bins = (int64_t)g->bvh.bins.nbx * g->bvh.bins.nby;
            out->n_bin_entries = g->bvh.n_bin_entries;
            out->bin_maxlen = g->bvh.bin_maxlen;
        }
    } else if (g->kind == GWN_GEOM_PATCHES) {
        out->n_vertices = g->nv;                      // boundary polyline vertices
        out->n_primitives = g->ps.n;
        out->n_boundary_edges = (int64_t)g->loop_vid.size();
        out->n_loops = (int64_t)g->loop_off.size() - 1;
    } else {
        out->n_vertices = g->cs.n_ctrl;
        out->n_primitives = g->cs.n_seg;
        out->n_boundary_edges = g->cs.n_chains;
        out->n_loops = g->cs.n_chains;
        out->n_pieces = g->cs.n_pieces;
        out->n_chains = g->cs.n_chains;
    }
    return GWN_OK;
}

GWN_API gwn_status gwn_mesh_boundary(const gwn_geom *g, int64_t *loop_offsets, int32_t *vert_ids) {
    if (!g || g->kind != GWN_GEOM_MESH) { set_error("gwn_mesh_boundary: not a mesh"); return GWN_E_INVALID; }
    if (loop_offsets) memcpy(loop_offsets, g->loop_off.data(), sizeof(int64_t) * g->loop_off.size());
    if (vert_ids && !g->loop_vid.empty()) memcpy(vert_ids, g->loop_vid.data(), sizeof(int32_t) * g->loop_vid.size());
    return GWN_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// evaluation
// ---------------------------------------------------------------------------
namespace gwn {

// per-axis coordinate tables for a grid (float64 rule, rounded to dtype)
void axis_table(double lo, double hi, int64_t n, std::vector<double> &out) {
    out.resize(n);
    if (n == 1) { out[0] = lo; return; }
    double step = (hi - lo) / (double)(n - 1);
    for (int64_t i = 0; i < n; i++) out[i] = lo + (double)i * step;
}

// device axis tables for grid q (cached per context; uploaded once per grid)
static gwn_status grid_tables(gwn_ctx *ctx, const gwn_queries *q, int dtype, QuerySrc &src) {
    auto &vec = ctx->axis_cache;
    for (auto &c : vec) {
        if (c.dim == q->dim && c.dtype == dtype && memcmp(c.lo, q->lo, sizeof(c.lo)) == 0 &&
            memcmp(c.hi, q->hi, sizeof(c.hi)) == 0 && memcmp(c.dims, q->dims, sizeof(c.dims)) == 0) {
            size_t off = 0;
            size_t esz = dtype == GWN_F64 ? 8 : 4;
            for (int k = 0; k < q->dim; k++) {
                if (dtype == GWN_F64) src.ax64[k] = (const double *)((char *)c.dev + off);
                else src.ax[k] = (const float *)((char *)c.dev + off);
                off += esz * q->dims[k];
            }
            return GWN_OK;
        }
    }
    if (vec.size() >= 64) {          // drop the oldest grid (cudaFree waits for work that may use it)
        CK(cudaFree(vec.front().dev), "grid tables");
        vec.erase(vec.begin());
    }
    AxisCache c;
    memset(&c, 0, sizeof(c));
    memcpy(c.lo, q->lo, sizeof(c.lo));
    memcpy(c.hi, q->hi, sizeof(c.hi));
    memcpy(c.dims, q->dims, sizeof(c.dims));
    c.dim = q->dim;
    c.dtype = dtype;
    size_t esz = dtype == GWN_F64 ? 8 : 4;
    size_t tot = 0;
    for (int k = 0; k < q->dim; k++) tot += esz * q->dims[k];
    std::vector<char> host(tot);
    size_t off = 0;
    for (int k = 0; k < q->dim; k++) {
        std::vector<double> ax;
        axis_table(q->lo[k], q->hi[k], q->dims[k], ax);
        for (int64_t i = 0; i < q->dims[k]; i++) {
            if (dtype == GWN_F64) ((double *)(host.data() + off))[i] = ax[i];
            else ((float *)(host.data() + off))[i] = (float)ax[i];
        }
        off += esz * q->dims[k];
    }
    CK(cudaMalloc(&c.dev, tot), "grid tables");
    cudaError_t e = cudaMemcpy(c.dev, host.data(), tot, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(c.dev);
        return cuda_fail(e, "grid tables");
    }
    c.bytes = tot;
    vec.push_back(c);
    return grid_tables(ctx, q, dtype, src);
}

static gwn_status check_queries(const gwn_queries *q, int dim) {
    if (!q) { set_error("queries is NULL"); return GWN_E_INVALID; }
    if (q->dim != dim) { set_error("queries: wrong dimension for this geometry"); return GWN_E_INVALID; }
    if (q->kind == GWN_QUERY_GRID) {
        int64_t n = 1;
        for (int k = 0; k < dim; k++) {
            if (q->dims[k] < 1 || q->dims[k] > (1 << 24) || !isfinite(q->lo[k]) || !isfinite(q->hi[k])) {
                set_error("queries: bad grid");
                return GWN_E_INVALID;
            }
            n *= q->dims[k];
        }
        if (n > 0x7fffffffLL) { set_error("queries: more than 2^31-1 grid points"); return GWN_E_INVALID; }
        return GWN_OK;
    }
    if (q->kind != GWN_QUERY_POINTS) { set_error("queries: unknown kind"); return GWN_E_INVALID; }
    if (q->n < 0 || q->n > 0x7fffffffLL || (q->n > 0 && !q->pts)) { set_error("queries: bad point list"); return GWN_E_INVALID; }
    if (q->mem_kind != GWN_MEM_DEVICE && q->mem_kind != GWN_MEM_HOST) { set_error("queries: bad mem_kind"); return GWN_E_INVALID; }
    return GWN_OK;
}

int64_t query_count(const gwn_queries *q) {
    if (q->kind == GWN_QUERY_GRID) {
        int64_t n = 1;
        for (int k = 0; k < q->dim; k++) n *= q->dims[k];
        return n;
    }
    return q->n;
}

// Build the device query view; host point lists are staged in arena slot 1.
static gwn_status make_query_src(gwn_ctx *ctx, const gwn_queries *q, int dtype, QuerySrc &src) {
    memset(&src, 0, sizeof(src));
    src.kind = q->kind;
    src.dim = q->dim;
    src.n = query_count(q);
    for (int k = 0; k < 3; k++) src.dims[k] = q->kind == GWN_QUERY_GRID ? q->dims[k] : 0;
    if (q->kind == GWN_QUERY_GRID) return grid_tables(ctx, q, dtype, src);
    size_t esz = (q->dtype == GWN_F64) ? 8 : 4;
    if (q->dtype != dtype) { set_error("queries: dtype does not match the geometry"); return GWN_E_INVALID; }
    const void *p = q->pts;
    if (q->mem_kind == GWN_MEM_HOST && src.n > 0) {
        cudaError_t e;
        void *dst = arena_get(ctx, 1, esz * q->dim * src.n, &e);
        if (!dst) return cuda_fail(e, "stage queries");
        CK(cudaMemcpyAsync(dst, q->pts, esz * q->dim * src.n, cudaMemcpyHostToDevice, ctx->stream), "stage queries");
        p = dst;
    }
    if (dtype == GWN_F64) src.pts64 = (const double *)p;
    else src.pts = (const float *)p;
    return GWN_OK;
}

static gwn_status read_stats(gwn_ctx *ctx, gwn_stats *st, int64_t nq, int64_t pairs, bool prepared) {
    if (!st) return GWN_OK;
    CK(cudaStreamSynchronize(ctx->stream), "sync");
    unsigned long long c[CNT_NUM];
    CK(cudaMemcpy(c, ctx->d_cnt, sizeof(c), cudaMemcpyDeviceToHost), "read counters");
    memset(st, 0, sizeof(*st));
    st->n_queries = nq;
    st->n_pairs = pairs;
    st->n_cut_sign = (int64_t)c[CNT_CUT_SIGN];
    st->n_fp64_filter = (int64_t)c[CNT_FP64];
    st->n_exact = (int64_t)c[CNT_EXACT];
    st->n_stack_overflow = (int64_t)c[CNT_STACK_OVERFLOW];
    st->n_tri_tests = (int64_t)(c[CNT_TRI_TESTS] + c[CNT_ROOTS]);
    st->n_deferred_traverse = (int64_t)c[CNT_DEFER_TRAV];
    st->n_deferred_boundary = (int64_t)c[CNT_DEFER_BTERM];
    st->n_root_iters = (int64_t)c[CNT_NEWTON];
    st->n_cert = (int64_t)c[CNT_CERT];
    st->n_cert_fixed = (int64_t)c[CNT_CERT_FIX];
    float a = 0, b = 0, t = 0, p = 0;
    cudaEventElapsedTime(&a, ctx->ev[1], ctx->ev[2]);
    cudaEventElapsedTime(&b, ctx->ev[2], ctx->ev[3]);
    cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[3]);
    if (prepared) cudaEventElapsedTime(&p, ctx->ev[0], ctx->ev[1]);
    st->ms_prepare = p;
    st->ms_traverse = a;
    st->ms_boundary = b;
    st->ms_total = t;
    return GWN_OK;
}

}  // namespace gwn

extern "C" {

static gwn_status eval_impl(gwn_geom *g, const gwn_queries *q, const float *d, void *w_out, int32_t *chi_out,
                            void *b_out, uint8_t *inside_out, gwn_stats *stats) {
    if (!g) { set_error("gwn_eval: NULL geometry"); return GWN_E_INVALID; }
    gwn_ctx *ctx = g->ctx;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (g->kind == GWN_GEOM_MESH) {
        gwn_status s = check_queries(q, 3);
        if (s != GWN_OK) return s;
        if (q->kind == GWN_QUERY_POINTS && q->dtype != GWN_F32) { set_error("gwn_eval: mesh queries are float32"); return GWN_E_INVALID; }
        if (!d) { set_error("gwn_eval: mesh evaluation needs a direction"); return GWN_E_INVALID; }
        int64_t nq = query_count(q);
        if (nq > 0 && !w_out && !chi_out && !b_out && !inside_out) {
            set_error("gwn_eval: no output requested");
            return GWN_E_INVALID;
        }
        if (stats) {
            CK(cudaMemsetAsync(ctx->d_cnt, 0, sizeof(unsigned long long) * CNT_NUM, ctx->stream), "clear counters");
            CK(cudaEventRecord(ctx->ev[0], ctx->stream), "event");
        }
        bool prepared = !(g->bvh.valid && memcmp(g->bvh.dkey, d, sizeof(float) * 3) == 0);
        s = gwn_mesh_prepare(g, d);
        if (s != GWN_OK) return s;
        QuerySrc src;
        s = make_query_src(ctx, q, GWN_F32, src);
        if (s != GWN_OK) return s;
        if (nq == 0) return read_stats(ctx, stats, 0, 0, prepared);
        int32_t *chi = chi_out;
        cudaError_t e;
        if (!chi) {
            chi = (int32_t *)arena_get(ctx, 0, sizeof(int32_t) * nq, &e);
            if (!chi) return cuda_fail(e, "chi buffer");
        }
        int32_t *defer = (int32_t *)arena_get(ctx, 4, sizeof(int32_t) * nq, &e);
        if (!defer) return cuda_fail(e, "deferred-query list");
        int32_t *lines = nullptr;
        size_t lbytes = traverse_lines_bytes(g->bvh, src);
        if (lbytes) {
            lines = (int32_t *)arena_get(ctx, 5, lbytes, &e);
            if (!lines) return cuda_fail(e, "per-line crossing lists");
        } else if (g->crossing_index == GWN_INDEX_AUTO && !g->bvh.bins_tried &&
                   (g->bvh.queries_seen += nq) >= 4 * g->nf) {
            // enough queries per triangle, over the evaluations of this
            // (mesh, d), for the 2D bins to repay their build
            prepared = true;                 // ms_prepare covers the bin build
            e = bins_build(g, ctx->stream);
            if (e == cudaErrorMemoryAllocation) cudaGetLastError();   // no room for the bins: the tree serves
            else if (e != cudaSuccess) return cuda_fail(e, "crossing bins");
        }
        if (stats) CK(cudaEventRecord(ctx->ev[1], ctx->stream), "event");
        e = launch_traverse(g->bvh, src, chi, defer, ctx->d_defer_count, ctx->d_tpairs, ctx->d_tpair_count, lines,
                            stats ? ctx->d_cnt : nullptr, ctx->d_status, ctx->sm_count, ctx->stream,
                            g->crossing_index != GWN_INDEX_TREE);
        if (e != cudaSuccess) return cuda_fail(e, "crossing traversal");
        if (stats) CK(cudaEventRecord(ctx->ev[2], ctx->stream), "event");
        e = launch_bterm3d(g->bseq, g->bvh.bframe, g->n_bseq, g->bvh.frame, make_frame64(d), src, chi, (float *)w_out,
                           (float *)b_out, defer, ctx->d_defer_count, stats ? ctx->d_cnt : nullptr, ctx->d_status,
                           ctx->sm_count, ctx->stream, inside_out);
        if (e != cudaSuccess) return cuda_fail(e, "boundary term");
        if (stats) CK(cudaEventRecord(ctx->ev[3], ctx->stream), "event");
        int64_t edges = (int64_t)g->loop_vid.size();
        return read_stats(ctx, stats, nq, nq * edges, prepared);
    }
    if (g->kind == GWN_GEOM_PATCHES) {
        gwn_status s = check_queries(q, 3);
        if (s != GWN_OK) return s;
        if (q->kind == GWN_QUERY_POINTS && q->dtype != GWN_F32) { set_error("gwn_eval: patch queries are float32"); return GWN_E_INVALID; }
        if (!d) { set_error("gwn_eval: patch evaluation needs a direction"); return GWN_E_INVALID; }
        int64_t nq = query_count(q);
        if (nq > 0 && !w_out && !chi_out && !b_out && !inside_out) {
            set_error("gwn_eval: no output requested");
            return GWN_E_INVALID;
        }
        if (stats) {
            CK(cudaMemsetAsync(ctx->d_cnt, 0, sizeof(unsigned long long) * CNT_NUM, ctx->stream), "clear counters");
            CK(cudaEventRecord(ctx->ev[0], ctx->stream), "event");
        }
        bool prepared = !(g->ps.valid && memcmp(g->ps.dkey, d, sizeof(float) * 3) == 0);
        s = patches_prepare(g, d);
        if (s != GWN_OK) return s;
        QuerySrc src;
        s = make_query_src(ctx, q, GWN_F32, src);
        if (s != GWN_OK) return s;
        if (nq == 0) return read_stats(ctx, stats, 0, 0, prepared);
        int32_t *chi = chi_out;
        cudaError_t e;
        if (!chi) {
            chi = (int32_t *)arena_get(ctx, 0, sizeof(int32_t) * nq, &e);
            if (!chi) return cuda_fail(e, "chi buffer");
        }
        int32_t *defer = (int32_t *)arena_get(ctx, 4, sizeof(int32_t) * nq, &e);
        if (!defer) return cuda_fail(e, "deferred-query list");
        if (stats) CK(cudaEventRecord(ctx->ev[1], ctx->stream), "event");
        // the long (ray, patch) pairs go to a list settled by a second kernel
        // (scratch slot 7: counter, then PATCH_DEFER_CAP pairs)
        char *dbuf = (char *)arena_get(ctx, 7, 16 + sizeof(int2) * (size_t)PATCH_DEFER_CAP, &e);
        if (!dbuf) return cuda_fail(e, "deferred patch pairs");
        e = launch_chi_patches(g->ps, src, chi, stats ? ctx->d_cnt : nullptr, ctx->d_status, ctx->stream,
                               (int2 *)(dbuf + 16), (int32_t *)dbuf, PATCH_DEFER_CAP, ctx->sm_count);
        if (e != cudaSuccess) return cuda_fail(e, "patch crossings");
        if (stats) CK(cudaEventRecord(ctx->ev[2], ctx->stream), "event");
        e = launch_bterm3d(g->bseq, g->ps.bframe, g->n_bseq, g->ps.frame, make_frame64(d), src, chi, (float *)w_out,
                           (float *)b_out, defer, ctx->d_defer_count, stats ? ctx->d_cnt : nullptr, ctx->d_status,
                           ctx->sm_count, ctx->stream, inside_out);
        if (e != cudaSuccess) return cuda_fail(e, "boundary term");
        if (stats) CK(cudaEventRecord(ctx->ev[3], ctx->stream), "event");
        return read_stats(ctx, stats, nq, nq * (int64_t)g->loop_vid.size(), prepared);
    }
    if (g->kind == GWN_GEOM_BEZIER2D) {
        gwn_status s = check_queries(q, 2);
        if (s != GWN_OK) return s;
        if (d && !(d[0] > 0.f && d[1] == 0.f)) { set_error("gwn_eval: 2D chains use the +x ray only"); return GWN_E_UNSUPPORTED; }
        int64_t nq = query_count(q);
        if (nq > 0 && !w_out && !chi_out && !b_out) { set_error("gwn_eval: no output requested"); return GWN_E_INVALID; }
        QuerySrc src;
        s = make_query_src(ctx, q, g->dtype, src);
        if (s != GWN_OK) return s;
        if (q->kind == GWN_QUERY_POINTS) {                 // one ray per query
            if (stats) {
                CK(cudaMemsetAsync(ctx->d_cnt, 0, sizeof(unsigned long long) * CNT_NUM, ctx->stream), "clear counters");
                for (int k = 0; k < 3; k++) CK(cudaEventRecord(ctx->ev[k], ctx->stream), "event");
            }
            int32_t *order = nullptr;
            const size_t ob = eval2d_points_order_bytes(g->cs, src.n);
            if (ob > 0) {
                cudaError_t ae = cudaSuccess;
                order = (int32_t *)arena_get(ctx, 8, ob, &ae);
                if (!order) return cuda_fail(ae, "2D point order scratch");
            }
            CK(launch_eval2d_points(g->cs, src, w_out, chi_out, b_out, stats ? ctx->d_cnt : nullptr, ctx->d_status,
                                    ctx->stream, ctx->d_cert, ctx->d_cert_count, order, ctx->sm_count),
               "2D point evaluation");
            if (stats) CK(cudaEventRecord(ctx->ev[3], ctx->stream), "event");
            return read_stats(ctx, stats, nq, 0, false);
        }
        if (stats) {
            CK(cudaMemsetAsync(ctx->d_cnt, 0, sizeof(unsigned long long) * CNT_NUM, ctx->stream), "clear counters");
            CK(cudaEventRecord(ctx->ev[0], ctx->stream), "event");
            CK(cudaEventRecord(ctx->ev[1], ctx->stream), "event");
            CK(cudaEventRecord(ctx->ev[2], ctx->stream), "event");
        }
        s = eval2d_single(g, src, w_out, chi_out, b_out, stats ? ctx->d_cnt : nullptr);
        if (s != GWN_OK) return s;
        if (stats) CK(cudaEventRecord(ctx->ev[3], ctx->stream), "event");
        return read_stats(ctx, stats, nq, q->dims[1] * g->cs.n_pieces, false);
    }
    set_error("gwn_eval: unknown geometry kind");
    return GWN_E_INVALID;
}

GWN_API gwn_status gwn_eval(gwn_geom *g, const gwn_queries *q, const float *d, void *w_out, int32_t *chi_out,
                            void *b_out, gwn_stats *stats) {
    return eval_impl(g, q, d, w_out, chi_out, b_out, nullptr, stats);
}

GWN_API gwn_status gwn_eval_inside(gwn_geom *g, const gwn_queries *q, const float *d, uint8_t *inside_out) {
    if (!g || !q) { set_error("gwn_eval_inside: NULL argument"); return GWN_E_INVALID; }
    if (g->kind != GWN_GEOM_MESH && g->kind != GWN_GEOM_PATCHES) {
        set_error("gwn_eval_inside: meshes and patch surfaces only");
        return GWN_E_UNSUPPORTED;
    }
    if (query_count(q) > 0 && !inside_out) { set_error("gwn_eval_inside: NULL output"); return GWN_E_INVALID; }
    return eval_impl(g, q, d, nullptr, nullptr, nullptr, inside_out, nullptr);
}

GWN_API gwn_status gwn_eval_host(gwn_geom *g, const gwn_queries *q, const float *d, void *w_host) {
    if (!g || !q || !w_host) { set_error("gwn_eval_host: NULL argument"); return GWN_E_INVALID; }
    gwn_ctx *ctx = g->ctx;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    int64_t nq = query_count(q);
    size_t esz = (g->kind == GWN_GEOM_BEZIER2D && g->dtype == GWN_F64) ? 8 : 4;
    cudaError_t e;
    // A page-locked output buffer is written by the boundary-term kernels
    // themselves (on Grace-Blackwell over the coherent CPU-GPU link, while the
    // kernel runs); other memory gets a device buffer and one copy.  The mesh
    // and patch paths only ever store to w, one plain store per query.
    void *w = nullptr;
    bool direct = false;
    if (nq > 0 && (g->kind == GWN_GEOM_MESH || g->kind == GWN_GEOM_PATCHES)) {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, w_host) == cudaSuccess) {
            if (pa.type == cudaMemoryTypeHost && pa.devicePointer) {
                w = pa.devicePointer;
                direct = true;
            }
        } else {
            cudaGetLastError();
        }
    }
    if (!direct) {
        w = arena_get(ctx, 3, esz * (nq > 0 ? nq : 1), &e);
        if (!w) return cuda_fail(e, "gwn_eval_host output");
    }
    gwn_queries qq = *q;
    if (q->kind == GWN_QUERY_POINTS) qq.mem_kind = GWN_MEM_HOST;   // staged by make_query_src
    gwn_status s = gwn_eval(g, &qq, d, w, nullptr, nullptr, nullptr);
    if (s != GWN_OK) return s;
    if (nq > 0 && !direct) CK(cudaMemcpyAsync(w_host, w, esz * nq, cudaMemcpyDeviceToHost, ctx->stream), "copy w");
    CK(cudaStreamSynchronize(ctx->stream), "sync");
    return GWN_OK;
}

GWN_API gwn_status gwn_eval_bruteforce(gwn_geom *g, const gwn_queries *q, void *w_out) {
    if (!g || !w_out) { set_error("gwn_eval_bruteforce: NULL argument"); return GWN_E_INVALID; }
    if (g->kind == GWN_GEOM_PATCHES) { set_error("gwn_eval_bruteforce: not provided for patches"); return GWN_E_UNSUPPORTED; }
    gwn_ctx *ctx = g->ctx;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (g->kind == GWN_GEOM_MESH) {
        gwn_status s = check_queries(q, 3);
        if (s != GWN_OK) return s;
        QuerySrc src;
        s = make_query_src(ctx, q, GWN_F32, src);
        if (s != GWN_OK) return s;
        cudaError_t e = launch_bruteforce3d(g->dV, g->dF, g->nf, src, (float *)w_out, ctx->sm_count, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(e, "brute force");
        return GWN_OK;
    }
    gwn_status s = check_queries(q, 2);
    if (s != GWN_OK) return s;
    QuerySrc src;
    s = make_query_src(ctx, q, g->dtype, src);
    if (s != GWN_OK) return s;
    cudaError_t e = launch_bruteforce2d(g->cs, src, w_out, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "brute force 2D");
    return GWN_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------
namespace gwn {
// boundary vertex -> records lists for the deterministic gradient scatter
static gwn_status ensure_vertex_lists(gwn_geom *g) {
    if (g->d_bvert || g->n_bseq == 0) return GWN_OK;
    std::vector<int32_t> rv(g->n_bseq);
    CK(cudaMemcpy(rv.data(), g->bseq_vid, sizeof(int32_t) * g->n_bseq, cudaMemcpyDeviceToHost), "records");
    std::vector<std::pair<int32_t, int32_t>> vr;
    for (int64_t k = 0; k < g->n_bseq; k++) vr.emplace_back(rv[k], (int32_t)k);
    std::sort(vr.begin(), vr.end());
    std::vector<int32_t> bv, recs;
    std::vector<int64_t> off(1, 0);
    for (size_t i = 0; i < vr.size(); i++) {
        if (i == 0 || vr[i].first != vr[i - 1].first) {
            if (i) off.push_back((int64_t)recs.size());
            bv.push_back(vr[i].first);
        }
        recs.push_back(vr[i].second);
    }
    off.push_back((int64_t)recs.size());
    // edge i of loop j ends at record i + j + 1 (each loop's first record
    // ends no edge)
    std::vector<int32_t> er(g->loop_vid.size());
    for (size_t j = 0; j + 1 < g->loop_off.size(); j++)
        for (int64_t i = g->loop_off[j]; i < g->loop_off[j + 1]; i++) er[i] = (int32_t)(i + (int64_t)j + 1);
    if (!er.empty()) {
        CK(cudaMalloc(&g->d_edge_rec, sizeof(int32_t) * er.size()), "edge records");
        CK(cudaMemcpy(g->d_edge_rec, er.data(), sizeof(int32_t) * er.size(), cudaMemcpyHostToDevice), "edge records");
    }
    g->n_bvert = (int64_t)bv.size();
    CK(cudaMalloc(&g->d_bvert, sizeof(int32_t) * bv.size()), "vertex lists");
    CK(cudaMalloc(&g->d_brec_off, sizeof(int64_t) * off.size()), "vertex lists");
    CK(cudaMalloc(&g->d_brecs, sizeof(int32_t) * recs.size()), "vertex lists");
    CK(cudaMemcpy(g->d_bvert, bv.data(), sizeof(int32_t) * bv.size(), cudaMemcpyHostToDevice), "vertex lists");
    CK(cudaMemcpy(g->d_brec_off, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice), "vertex lists");
    CK(cudaMemcpy(g->d_brecs, recs.data(), sizeof(int32_t) * recs.size(), cudaMemcpyHostToDevice), "vertex lists");
    return GWN_OK;
}
}  // namespace gwn

extern "C" GWN_API gwn_status gwn_backward(gwn_geom *g, const gwn_queries *q, const float *d, const float *grad_w,
                                           float *grad_p, float *grad_V) {
    (void)d;
    if (!g || g->kind != GWN_GEOM_MESH) { set_error("gwn_backward: needs a mesh"); return GWN_E_INVALID; }
    gwn_status s = check_queries(q, 3);
    if (s != GWN_OK) return s;
    int64_t nq = query_count(q);
    if (nq > 0 && !grad_w) { set_error("gwn_backward: grad_w is NULL"); return GWN_E_INVALID; }
    gwn_ctx *ctx = g->ctx;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    QuerySrc src;
    s = make_query_src(ctx, q, GWN_F32, src);
    if (s != GWN_OK) return s;
    if (grad_p && grad_V && nq > 0 && g->n_bseq > 0) {
        // both: one pass over the (query, edge) pairs
        CK(cudaMemsetAsync(grad_V, 0, sizeof(float) * 3 * g->nv, ctx->stream), "clear grad_V");
        s = ensure_vertex_lists(g);
        if (s != GWN_OK) return s;
        const int64_t ne = (int64_t)g->loop_vid.size();
        int chunks = grad_pv_chunks(nq, ne, ctx->sm_count);
        size_t part = (sizeof(float) * 8 * (size_t)chunks * g->n_bseq + 255) & ~(size_t)255;
        size_t partp = (grad_pv_partial_p_bytes(nq, ne) + 255) & ~(size_t)255;
        size_t recb = sizeof(float) * 3 * g->n_bseq;
        cudaError_t e;
        char *buf = (char *)arena_get(ctx, 0, part + partp + recb, &e);
        if (!buf) return cuda_fail(e, "gradient workspace");
        e = launch_grad_pv(g->bseq, g->n_bseq, g->d_edge_rec, ne, src, grad_w, chunks, (float *)buf,
                           (float *)(buf + part), (float *)(buf + part + partp), g->d_bvert, g->d_brec_off,
                           g->d_brecs, g->n_bvert, grad_p, grad_V, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(e, "gradients");
        return GWN_OK;
    }
    if (grad_p) {
        cudaError_t e = launch_grad_p(g->bseq, g->n_bseq, src, grad_w, grad_p, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(e, "grad_p");
    }
    if (grad_V) {
        CK(cudaMemsetAsync(grad_V, 0, sizeof(float) * 3 * g->nv, ctx->stream), "clear grad_V");
        s = ensure_vertex_lists(g);
        if (s != GWN_OK) return s;
        if (nq > 0 && g->n_bseq > 0) {
            int chunks = grad_v_chunks(nq, g->n_bseq, ctx->sm_count);
            size_t part = sizeof(float) * 8 * (size_t)chunks * g->n_bseq;
            size_t recb = sizeof(float) * 3 * g->n_bseq;
            cudaError_t e;
            char *buf = (char *)arena_get(ctx, 0, part + recb + 256, &e);
            if (!buf) return cuda_fail(e, "gradient workspace");
            float *partial = (float *)buf;
            float *rec = (float *)(buf + ((part + 255) & ~(size_t)255));
            e = launch_grad_v(g->bseq, g->n_bseq, src, grad_w, chunks, partial, rec, g->d_bvert, g->d_brec_off,
                              g->d_brecs, g->n_bvert, grad_V, ctx->stream);
            if (e != cudaSuccess) return cuda_fail(e, "grad_V");
        }
    }
    return GWN_OK;
}
