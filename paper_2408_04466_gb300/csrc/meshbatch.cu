// meshbatch.cu -- many meshes of uneven sizes, each with its own queries,
// evaluated by one persistent launch (gwn_eval_meshes).
//
// Work items are (mesh, run of query tiles); a tile is the 1024 queries one
// boundary-term block takes (256 threads, two query pairs each).  Items are
// ordered by cost (boundary records per query, largest meshes first) and
// claimed from an atomic counter, so meshes of 1e3 and 1e6 triangles, with
// a few hundred or millions of queries, share one launch without idle SMs.
// For its tile a block first counts crossings (the 2D bins when the mesh has
// them, else one LBVH traversal per thread) and then runs the boundary
// term's main pass, writing B_d into the caller's output; the two are
// independent, so no barrier separates them.  Small list-driven kernels then
// settle the unsettled (query, triangle) pairs, recount deferred queries, take
// the careful boundary term of deferred queries, and form w = B_d + chi.
// Every step uses the same device code as gwn_eval (traverse.cuh,
// bterm.cuh), so each query gets the same bits as from gwn_eval on its mesh.
//
// Nothing in a call synchronises the host after the first: the first call
// with a given (meshes, queries, outputs, d) uploads the plan, picks the
// tile run length by timing the candidates, and captures the launch sequence
// in a CUDA graph; later calls replay it.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <new>
#include <vector>

#include "bterm.cuh"
#include "traverse.cuh"

namespace gwn {

constexpr int MB_THREADS = 256;
constexpr int MB_KP = 2;                                  // query pairs per thread in the boundary term
constexpr int MB_TILE = MB_THREADS * 2 * MB_KP;           // queries per tile

struct MeshDesc {
    // crossing search
    const BvhNode *nodes;
    const float4 *tris;
    int root;
    int use_bins;
    TravParams tp;
    const int32_t *bin_start;
    const float2 *bin_zt;
    const float4 *bin_box;
    BinParams bp;
    Frame fr;
    Frame64 f64;
    // boundary term
    const float4 *bframe;
    const float4 *bseq;
    int nb;
    // queries and output
    QuerySrc q;
    int64_t qofs;          // first batch-wide query index of this mesh
    int64_t n_tiles;
    float *w_out;
};

// the mesh holding batch-wide query index g: qofs is non-decreasing
__device__ __forceinline__ int mesh_of(const int64_t *__restrict__ qofs, int n, int64_t g) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (qofs[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int MINB>
__global__ void __launch_bounds__(MB_THREADS, MINB) mesh_batch_kernel(
    const MeshDesc *__restrict__ md, const int2 *__restrict__ items, int64_t n_items, int tiles_per_item,
    unsigned long long *counter, const __grid_constant__ PackedConsts K, int32_t *__restrict__ chi,
    int32_t *tdefer, int32_t *tdefer_count, int2 *tpairs, int32_t *tpair_count, int32_t *bdefer,
    int32_t *bdefer_count, int *status) {
    __shared__ long long s_item;
    for (int64_t guard = 0; guard <= n_items; guard++) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        const int2 it = items[item];
        const MeshDesc &D = md[it.x];
        const QuerySrc q = D.q;
        int64_t t1 = (int64_t)it.y + tiles_per_item;
        if (t1 > D.n_tiles) t1 = D.n_tiles;
        for (int64_t t = it.y; t < t1; t++) {
            const int64_t qbase = t * MB_TILE;
            // crossing counts of the tile's queries, 256 at a time
            for (int s = 0; s < MB_TILE / MB_THREADS; s++) {
                const int64_t idx = qbase + s * MB_THREADS + threadIdx.x;
                if (D.use_bins) {
                    chi_bins_block(D.bin_start, D.bin_zt, D.bin_box, D.bp, D.tris, D.fr, D.tp, q,
                                   idx < q.n ? idx : -1, D.qofs, chi, tdefer, tdefer_count, tpairs, tpair_count,
                                   nullptr);
                } else if (idx < q.n) {
                    int acc, ntests = 0;
                    bool unsure = false;
                    const bool ok = traverse_ray<true>(D.nodes, D.tris, D.root, D.fr, D.tp, query_point3(q, idx),
                                                       D.qofs + idx, acc, unsure, tpairs, tpair_count, ntests,
                                                       nullptr, status);
                    if (ok && unsure) defer_query(tdefer, tdefer_count, D.qofs + idx);
                    else chi[D.qofs + idx] = ok ? acc : INT32_MIN;
                }
            }
            // boundary term: B_d into the output (w is formed once chi is final)
            bterm_block<MB_KP>(D.bframe, D.nb, D.fr, K, q, qbase + threadIdx.x, D.qofs, nullptr, D.w_out, nullptr,
                               nullptr, bdefer, bdefer_count);
        }
    }
}

// unsettled pairs of the float32 passes (as traverse_pairs_kernel)
__global__ void __launch_bounds__(128) mesh_batch_pairs_kernel(const MeshDesc *__restrict__ md,
                                                               const int64_t *__restrict__ qofs, int n_mesh,
                                                               int32_t *chi, const int2 *__restrict__ pairs,
                                                               const int32_t *pair_count, int64_t n_total,
                                                               int *status) {
    int64_t n = *pair_count;
    if (n > GWN_TPAIR_CAP) n = GWN_TPAIR_CAP;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int2 pr = pairs[i];
        if (pr.x < 0 || pr.x >= n_total) { atomicOr(status, ST_BAD_INPUT); continue; }
        if (chi[pr.x] == INT32_MIN) continue;
        const MeshDesc &D = md[mesh_of(qofs, n_mesh, pr.x)];
        const float3 p = query_point3(D.q, pr.x - D.qofs);
        const float3 dd = make_float3(D.fr.d[0], D.fr.d[1], D.fr.d[2]);
        const float4 a = __ldg(&D.tris[3 * pr.y]), b = __ldg(&D.tris[3 * pr.y + 1]), c = __ldg(&D.tris[3 * pr.y + 2]);
        const int r = tri_crossing(make_float3(a.x, a.y, a.z), make_float3(b.x, b.y, b.z), make_float3(c.x, c.y, c.z),
                                   p, dd, nullptr, status);
        if (r) atomicAdd(&chi[pr.x], r);
    }
}

// deferred queries of the crossing search: full predicates (as
// traverse_careful_kernel)
__global__ void __launch_bounds__(128) mesh_batch_trav_careful_kernel(const MeshDesc *__restrict__ md,
                                                                      const int64_t *__restrict__ qofs, int n_mesh,
                                                                      int32_t *chi, const int32_t *__restrict__ defer,
                                                                      const int32_t *defer_count, int64_t n_total,
                                                                      int *status) {
    int64_t n = *defer_count;
    if (n > n_total) n = n_total;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = defer[i];
        if (g < 0 || g >= n_total) { atomicOr(status, ST_BAD_INPUT); continue; }
        const MeshDesc &D = md[mesh_of(qofs, n_mesh, g)];
        int acc, ntests = 0;
        bool unsure = false;
        const bool ok = traverse_ray<false>(D.nodes, D.tris, D.root, D.fr, D.tp, query_point3(D.q, g - D.qofs), g,
                                            acc, unsure, nullptr, nullptr, ntests, nullptr, status);
        chi[g] = ok ? acc : INT32_MIN;
    }
}

// deferred queries of the boundary term: the careful pass, B_d into the
// output (as bterm3d_careful_kernel)
__global__ void __launch_bounds__(128) mesh_batch_bterm_careful_kernel(const MeshDesc *__restrict__ md,
                                                                       const int64_t *__restrict__ qofs, int n_mesh,
                                                                       const int32_t *__restrict__ defer,
                                                                       const int32_t *defer_count, int64_t n_total,
                                                                       int *status) {
    int64_t n = *defer_count;
    if (n > n_total) n = n_total;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {       // block-uniform loop
        const int64_t g = defer[i];
        if (g < 0 || g >= n_total) {
            if (threadIdx.x == 0) atomicOr(status, ST_BAD_INPUT);
            continue;
        }
        const MeshDesc &D = md[mesh_of(qofs, n_mesh, g)];
        const float Bv = careful_block_B(D.bseq, D.nb, D.fr, D.f64, query_point3(D.q, g - D.qofs), nullptr, status);
        if (threadIdx.x == 0) D.w_out[g - D.qofs] = Bv;
        __syncthreads();
    }
}

// w = B_d + chi for every query of the batch (the boundary-term kernels'
// own final sum)
__global__ void __launch_bounds__(256) mesh_batch_combine_kernel(const MeshDesc *__restrict__ md,
                                                                 const int64_t *__restrict__ qofs, int n_mesh,
                                                                 const int32_t *__restrict__ chi, int64_t n_total) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const MeshDesc &D = md[mesh_of(qofs, n_mesh, g)];
        float *w = D.w_out + (g - D.qofs);
        *w = __fadd_rn(*w, (float)chi[g]);
    }
}

// ---- host ---------------------------------------------------------------------
struct MeshBatchPlan {
    std::vector<uint64_t> key;
    int n = 0;
    int64_t n_total = 0, n_items = 0;
    int tiles_per_item = 1, minb = 2, blocks = 0;
    void *dev = nullptr;                 // descriptors, offsets, items, axis tables, lists, counters
    MeshDesc *d_md = nullptr;
    int64_t *d_qofs = nullptr;
    int2 *d_items = nullptr;
    int32_t *d_chi = nullptr, *d_tdefer = nullptr, *d_bdefer = nullptr, *d_counts = nullptr;
    int2 *d_pairs = nullptr;
    unsigned long long *d_counter = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t stream = nullptr;
    float tuned_ms = 0.f;
};

struct MeshBatchCache {
    std::vector<MeshBatchPlan *> plans;
};

void mesh_batch_cache_free(void *p) {
    MeshBatchCache *c = (MeshBatchCache *)p;
    for (MeshBatchPlan *b : c->plans) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        if (b->dev) cudaFree(b->dev);
        delete b;
    }
    delete c;
}

static cudaError_t mesh_batch_launch(const MeshBatchPlan *P, int tiles_per_item, int minb, int blocks,
                                     int *status, int sm_count, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(P->d_counter, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->d_counts, 0, sizeof(int32_t) * 4, st);
    if (e != cudaSuccess) return e;
    const PackedConsts K = bterm_consts();
    int32_t *tdefer_count = P->d_counts, *tpair_count = P->d_counts + 1, *bdefer_count = P->d_counts + 2;
    if (minb == 1)
        mesh_batch_kernel<1><<<(unsigned)blocks, MB_THREADS, 0, st>>>(
            P->d_md, P->d_items, P->n_items, tiles_per_item, P->d_counter, K, P->d_chi, P->d_tdefer, tdefer_count,
            P->d_pairs, tpair_count, P->d_bdefer, bdefer_count, status);
    else
        mesh_batch_kernel<2><<<(unsigned)blocks, MB_THREADS, 0, st>>>(
            P->d_md, P->d_items, P->n_items, tiles_per_item, P->d_counter, K, P->d_chi, P->d_tdefer, tdefer_count,
            P->d_pairs, tpair_count, P->d_bdefer, bdefer_count, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int cblocks = (sm_count > 0 ? sm_count : 152) * 4;
    // pairs first (they add to chi), then the whole recounts (they overwrite it)
    mesh_batch_pairs_kernel<<<cblocks, 128, 0, st>>>(P->d_md, P->d_qofs, P->n, P->d_chi, P->d_pairs, tpair_count,
                                                     P->n_total, status);
    mesh_batch_trav_careful_kernel<<<cblocks, 128, 0, st>>>(P->d_md, P->d_qofs, P->n, P->d_chi, P->d_tdefer,
                                                            tdefer_count, P->n_total, status);
    mesh_batch_bterm_careful_kernel<<<cblocks, 128, 0, st>>>(P->d_md, P->d_qofs, P->n, P->d_bdefer, bdefer_count,
                                                             P->n_total, status);
    int64_t wb = (P->n_total + 255) / 256;
    int64_t cap = (int64_t)(sm_count > 0 ? sm_count : 152) * 16;
    mesh_batch_combine_kernel<<<(unsigned)(wb < cap ? wb : cap), 256, 0, st>>>(P->d_md, P->d_qofs, P->n, P->d_chi,
                                                                              P->n_total);
    return cudaGetLastError();
}

static int mesh_batch_blocks(int minb, int sm_count) {
    int per_sm = 0;
    cudaError_t e = minb == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mesh_batch_kernel<1>,
                                                                              MB_THREADS, 0)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mesh_batch_kernel<2>,
                                                                              MB_THREADS, 0);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    return (sm_count > 0 ? sm_count : 152) * per_sm;
}

}  // namespace gwn

using namespace gwn;

#define CK(call, what)                                     \
    do {                                                   \
        cudaError_t ck_e = (call);                         \
        if (ck_e != cudaSuccess) return cuda_fail(ck_e, what); \
    } while (0)

namespace {

// per mesh: a grid's axis tables are copied into the plan (the context's
// table cache may drop them); points stay the caller's
struct MeshIn {
    gwn_geom *g;
    gwn_queries q;
    float *w;
    int64_t nq;
    size_t axis_off;
};

void key_push(std::vector<uint64_t> &k, const void *p, size_t bytes) {
    const unsigned char *c = (const unsigned char *)p;
    for (size_t i = 0; i < bytes; i += 8) {
        uint64_t v = 0;
        memcpy(&v, c + i, bytes - i < 8 ? bytes - i : 8);
        k.push_back(v);
    }
}

}  // namespace

extern "C" GWN_API gwn_status gwn_eval_meshes(gwn_ctx *ctx, gwn_geom *const *meshes, const gwn_queries *qs,
                                              int64_t n, const float d[3], float *const *w_outs,
                                              const gwn_plan *plan, gwn_stats *stats) {
    if (!ctx || !meshes || !qs || !d || !w_outs || n < 1 || n > (1 << 20)) {
        set_error("gwn_eval_meshes: bad arguments");
        return GWN_E_INVALID;
    }
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    std::vector<MeshIn> in((size_t)n);
    int64_t n_total = 0;
    size_t axis_bytes = 0;
    for (int64_t i = 0; i < n; i++) {
        gwn_geom *g = meshes[i];
        const gwn_queries *q = &qs[i];
        if (!g || g->kind != GWN_GEOM_MESH || g->ctx != ctx) {
            set_error("gwn_eval_meshes: every geometry must be a mesh of this context");
            return GWN_E_INVALID;
        }
        if (!g->bvh.valid || memcmp(g->bvh.dkey, d, sizeof(float) * 3) != 0 || g->bvh.n <= 1) {
            set_error("gwn_eval_meshes: every mesh must be prepared for d (gwn_mesh_prepare) and have at least "
                      "two triangles");
            return GWN_E_INVALID;
        }
        if (q->dim != 3 || (q->kind != GWN_QUERY_GRID && q->kind != GWN_QUERY_POINTS)) {
            set_error("gwn_eval_meshes: queries must be 3D grids or points");
            return GWN_E_INVALID;
        }
        if (q->kind == GWN_QUERY_POINTS && (q->dtype != GWN_F32 || q->mem_kind != GWN_MEM_DEVICE || (q->n > 0 && !q->pts))) {
            set_error("gwn_eval_meshes: point queries must be float32 in device memory");
            return GWN_E_INVALID;
        }
        int64_t nq = q->kind == GWN_QUERY_GRID ? q->dims[0] * q->dims[1] * q->dims[2] : q->n;
        if (q->kind == GWN_QUERY_GRID)
            for (int k = 0; k < 3; k++)
                if (q->dims[k] < 1) { set_error("gwn_eval_meshes: grid dims must be >= 1"); return GWN_E_INVALID; }
        if (nq < 0 || (nq > 0 && !w_outs[i])) { set_error("gwn_eval_meshes: missing output"); return GWN_E_INVALID; }
        in[i] = MeshIn{g, *q, w_outs[i], nq, axis_bytes};
        if (q->kind == GWN_QUERY_GRID) axis_bytes += sizeof(float) * (size_t)(q->dims[0] + q->dims[1] + q->dims[2]);
        n_total += nq;
    }
    if (n_total > 0x7fffffff) { set_error("gwn_eval_meshes: more than 2^31 - 1 queries in one batch"); return GWN_E_INVALID; }
    if (n_total == 0) return GWN_OK;
    // plan key: meshes and their device structures, queries, outputs, d, plan
    std::vector<uint64_t> key;
    key_push(key, d, sizeof(float) * 3);
    for (const MeshIn &m : in) {
        key_push(key, &m.g, sizeof(m.g));
        key_push(key, &m.g->bvh.block, sizeof(void *));
        key_push(key, &m.g->bvh.bin_block, sizeof(void *));
        key_push(key, &m.g->bvh.n_bin_entries, sizeof(int64_t));
        key_push(key, &m.q, sizeof(gwn_queries));
        key_push(key, &m.w, sizeof(m.w));
    }
    gwn_plan pl;
    memset(&pl, 0, sizeof(pl));
    if (plan) pl = *plan;
    key_push(key, &pl, sizeof(pl));
    key_push(key, &ctx->stream, sizeof(ctx->stream));
    if (!ctx->mesh_batch_cache) ctx->mesh_batch_cache = new (std::nothrow) MeshBatchCache();
    MeshBatchCache *C = (MeshBatchCache *)ctx->mesh_batch_cache;
    if (!C) { set_error("gwn_eval_meshes: out of host memory"); return GWN_E_OOM; }
    MeshBatchPlan *P = nullptr;
    for (MeshBatchPlan *b : C->plans)
        if (b->key == key) { P = b; break; }
    cudaEvent_t e0 = ctx->ev[0], e1 = ctx->ev[3];
    if (stats) CK(cudaEventRecord(e0, ctx->stream), "event");
    if (!P) {
        P = new (std::nothrow) MeshBatchPlan();
        if (!P) { set_error("gwn_eval_meshes: out of host memory"); return GWN_E_OOM; }
        P->key = key;
        P->n = (int)n;
        P->n_total = n_total;
        // mesh order for the items: most boundary records first (cost per query)
        std::vector<int> order((size_t)n);
        for (int i = 0; i < (int)n; i++) order[i] = i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return in[a].g->n_bseq > in[b].g->n_bseq; });
        std::vector<MeshDesc> md((size_t)n);
        std::vector<int64_t> qofs((size_t)n + 1, 0);
        for (int i = 0; i < (int)n; i++) qofs[i + 1] = qofs[i] + in[i].nq;
        // device layout: md | qofs | axis tables | chi | tdefer | bdefer | pairs | counts | counter | items
        std::vector<int2> items;
        auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
        size_t o_md = 0, o_qofs = al(o_md + sizeof(MeshDesc) * n), o_ax = al(o_qofs + sizeof(int64_t) * (n + 1));
        size_t o_chi = al(o_ax + axis_bytes), o_td = al(o_chi + sizeof(int32_t) * n_total);
        size_t o_bd = al(o_td + sizeof(int32_t) * n_total), o_pr = al(o_bd + sizeof(int32_t) * n_total);
        size_t o_cnt = al(o_pr + sizeof(int2) * GWN_TPAIR_CAP), o_ctr = al(o_cnt + sizeof(int32_t) * 4);
        size_t o_items = al(o_ctr + sizeof(unsigned long long));
        // items of every tile (tiles_per_item chosen below; one tile each here)
        int64_t n_tiles_total = 0;
        for (int i = 0; i < (int)n; i++) n_tiles_total += (in[i].nq + MB_TILE - 1) / MB_TILE;
        size_t bytes = al(o_items + sizeof(int2) * (size_t)n_tiles_total);
        cudaError_t e = cudaMalloc(&P->dev, bytes);
        if (e != cudaSuccess) {
            delete P;
            return cuda_fail(e, "gwn_eval_meshes: plan memory");
        }
        char *base = (char *)P->dev;
        P->d_md = (MeshDesc *)(base + o_md);
        P->d_qofs = (int64_t *)(base + o_qofs);
        P->d_chi = (int32_t *)(base + o_chi);
        P->d_tdefer = (int32_t *)(base + o_td);
        P->d_bdefer = (int32_t *)(base + o_bd);
        P->d_pairs = (int2 *)(base + o_pr);
        P->d_counts = (int32_t *)(base + o_cnt);
        P->d_counter = (unsigned long long *)(base + o_ctr);
        P->d_items = (int2 *)(base + o_items);
        std::vector<float> axes(axis_bytes / sizeof(float));
        for (int i = 0; i < (int)n; i++) {
            MeshIn &m = in[i];
            gwn_geom *g = m.g;
            const MeshBvh &b = g->bvh;
            MeshDesc &D = md[i];
            memset(&D, 0, sizeof(D));
            D.nodes = b.nodes;
            D.tris = b.tris;
            D.root = b.root;
            D.use_bins = g->crossing_index != GWN_INDEX_TREE && b.n_bin_entries > 0 && b.n < (int64_t(1) << 26);
            D.tp = trav_params(b);
            D.bin_start = b.bin_start;
            D.bin_zt = b.bin_zt;
            D.bin_box = b.bin_box;
            D.bp = b.bins;
            D.fr = b.frame;
            D.f64 = make_frame64(d);
            D.bframe = b.bframe;
            D.bseq = g->bseq;
            D.nb = (int)g->n_bseq;
            memset(&D.q, 0, sizeof(D.q));
            D.q.kind = m.q.kind;
            D.q.dim = 3;
            D.q.n = m.nq;
            if (m.q.kind == GWN_QUERY_GRID) {
                for (int k = 0; k < 3; k++) D.q.dims[k] = m.q.dims[k];
                size_t off = m.axis_off;
                for (int k = 0; k < 3; k++) {
                    std::vector<double> ax;
                    axis_table(m.q.lo[k], m.q.hi[k], m.q.dims[k], ax);
                    for (int64_t j = 0; j < m.q.dims[k]; j++) axes[off / sizeof(float) + j] = (float)ax[j];
                    D.q.ax[k] = (const float *)(base + o_ax + off);
                    off += sizeof(float) * m.q.dims[k];
                }
            } else {
                D.q.pts = (const float *)m.q.pts;
            }
            D.qofs = qofs[i];
            D.n_tiles = (m.nq + MB_TILE - 1) / MB_TILE;
            D.w_out = m.w;
        }
        e = cudaMemcpy(P->d_md, md.data(), sizeof(MeshDesc) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(P->d_qofs, qofs.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && axis_bytes)
            e = cudaMemcpy(base + o_ax, axes.data(), axis_bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(P->dev);
            delete P;
            return cuda_fail(e, "gwn_eval_meshes: plan upload");
        }
        // candidates: tiles per item x blocks per SM, each timed once after a
        // warm-up (or the caller's plan: rows_per_item = tiles per item,
        // threads_per_block = blocks per SM)
        std::vector<std::pair<int, int>> cand;
        if (pl.rows_per_item > 0 || pl.threads_per_block > 0)
            cand.push_back({pl.rows_per_item > 0 ? pl.rows_per_item : 1, pl.threads_per_block == 1 ? 1 : 2});
        else
            cand = {{1, 2}, {4, 2}, {16, 2}, {1, 1}, {4, 1}};
        float best = 1e30f;
        for (auto cd : cand) {
            items.clear();
            for (int oi : order) {
                int64_t nt = md[oi].n_tiles;
                for (int64_t t = 0; t < nt; t += cd.first) items.push_back(make_int2(oi, (int)t));
            }
            e = cudaMemcpy(P->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) break;
            P->n_items = (int64_t)items.size();
            int blocks = mesh_batch_blocks(cd.second, ctx->sm_count);
            float ms = 0.f;
            if (cand.size() > 1) {
                e = mesh_batch_launch(P, cd.first, cd.second, blocks, ctx->d_status, ctx->sm_count, ctx->stream);
                cudaEvent_t a = ctx->ev[4], z = ctx->ev[5];
                if (e == cudaSuccess) e = cudaEventRecord(a, ctx->stream);
                if (e == cudaSuccess)
                    e = mesh_batch_launch(P, cd.first, cd.second, blocks, ctx->d_status, ctx->sm_count, ctx->stream);
                if (e == cudaSuccess) e = cudaEventRecord(z, ctx->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(z);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, z);
                if (e != cudaSuccess) break;
            }
            if (ms < best) {
                best = ms;
                P->tiles_per_item = cd.first;
                P->minb = cd.second;
                P->blocks = blocks;
            }
        }
        if (e == cudaSuccess) {          // final item list of the chosen run length
            items.clear();
            for (int oi : order) {
                int64_t nt = md[oi].n_tiles;
                for (int64_t t = 0; t < nt; t += P->tiles_per_item) items.push_back(make_int2(oi, (int)t));
            }
            e = cudaMemcpy(P->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice);
            P->n_items = (int64_t)items.size();
        }
        P->tuned_ms = best < 1e29f ? best : 0.f;
        if (e == cudaSuccess && (plan ? pl.use_graph : 1)) {   // capture the launch sequence once
            cudaStream_t cap = ctx->stream;
            bool own = false;
            if (cap == nullptr) {    // the legacy stream cannot be captured: a private one for the capture
                e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
                own = e == cudaSuccess;
            }
            if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t le = mesh_batch_launch(P, P->tiles_per_item, P->minb, P->blocks, ctx->d_status,
                                                   ctx->sm_count, cap);
                e = cudaStreamEndCapture(cap, &P->graph);
                if (le != cudaSuccess) e = le;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&P->exec, P->graph, 0);
            if (own) cudaStreamDestroy(cap);
            P->stream = ctx->stream;
        }
        if (e != cudaSuccess) {
            if (P->exec) cudaGraphExecDestroy(P->exec);
            if (P->graph) cudaGraphDestroy(P->graph);
            cudaFree(P->dev);
            delete P;
            return cuda_fail(e, "gwn_eval_meshes: plan");
        }
        C->plans.push_back(P);
    }
    cudaError_t e;
    if (P->exec) e = cudaGraphLaunch(P->exec, ctx->stream);
    else e = mesh_batch_launch(P, P->tiles_per_item, P->minb, P->blocks, ctx->d_status, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "gwn_eval_meshes: launch");
    if (stats) {
        CK(cudaEventRecord(e1, ctx->stream), "event");
        CK(cudaEventSynchronize(e1), "event");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        memset(stats, 0, sizeof(*stats));
        stats->n_queries = n_total;
        stats->ms_total = ms;
        stats->ms_boundary = ms;
        stats->ms_prepare = P->tuned_ms;
        int32_t c[4] = {0, 0, 0, 0};
        CK(cudaMemcpy(c, P->d_counts, sizeof(c), cudaMemcpyDeviceToHost), "counters");
        stats->n_deferred_traverse = c[0] + c[1];
        stats->n_deferred_boundary = c[2];
    }
    return GWN_OK;
}

extern "C" GWN_API gwn_status gwn_meshes_plan_get(gwn_ctx *ctx, int32_t *tiles_per_item, int32_t *blocks_per_sm) {
    if (!ctx || !ctx->mesh_batch_cache || ((MeshBatchCache *)ctx->mesh_batch_cache)->plans.empty()) {
        set_error("gwn_meshes_plan_get: no batched mesh plan yet");
        return GWN_E_INVALID;
    }
    const MeshBatchPlan *P = ((MeshBatchCache *)ctx->mesh_batch_cache)->plans.back();
    if (tiles_per_item) *tiles_per_item = P->tiles_per_item;
    if (blocks_per_sm) *blocks_per_sm = P->minb;
    return GWN_OK;
}
