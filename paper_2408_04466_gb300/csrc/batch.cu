// batch.cu -- host side of the 2D evaluation: one chain set on one grid
// (gwn_eval), and many independent chains each on its own grid in one
// persistent launch (gwn_eval_batch) with an autotuned work-item shape and a
// CUDA graph replayed on later calls.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <new>
#include <vector>

#include "gwn_internal.h"

namespace gwn {




static const int64_t MAX_NX = 16384;

// axis value i of a grid axis, as the axis tables hold it (float64 formula,
// rounded to the chain's precision)
static double axis_value(double lo, double hi, int64_t n, int64_t i, int dtype) {
    double v = n == 1 ? lo : lo + (double)i * ((hi - lo) / (double)(n - 1));
    return dtype == GWN_F64 ? v : (double)(float)v;
}

// items (set, row block, first piece, end piece), most expensive sets first.
// A set's pieces are ordered by their lowest y; a piece can cross a row of
// the block only if its lowest y is <= the block's last row and its highest
// y > the block's first row, so the run [first, end) skips the pieces whose
// lowest y lies above the block and the prefix whose running maximum of the
// highest y stays at or below it (the same comparisons the kernel makes, in
// the same precision).
static void make_items(const std::vector<Set2D> &sets, const gwn_queries *qs, const ChainSet &cs, int rows_per_item,
                       std::vector<int4> &items) {
    std::vector<std::pair<double, int>> order;
    for (size_t s = 0; s < sets.size(); s++)
        order.emplace_back(-(double)(sets[s].p_hi - sets[s].p_lo + 1) * (double)sets[s].nx, (int)s);
    std::stable_sort(order.begin(), order.end());
    items.clear();
    const double *lo_t = cs.h_piece_lo.data(), *hmax_t = cs.h_piece_hmax.data();
    for (auto &o : order) {
        const Set2D &S = sets[o.second];
        const gwn_queries &q = qs[o.second];
        int64_t nb = (S.ny + rows_per_item - 1) / rows_per_item;
        for (int64_t b = 0; b < nb; b++) {
            int64_t r0 = b * rows_per_item, r1 = std::min<int64_t>(r0 + rows_per_item, S.ny);
            double y_first = axis_value(q.lo[1], q.hi[1], S.ny, r0, cs.dtype);
            double y_last = axis_value(q.lo[1], q.hi[1], S.ny, r1 - 1, cs.dtype);
            // first piece with hmax > y_first; first piece with lo > y_last
            int64_t pa = std::upper_bound(hmax_t + S.p_lo, hmax_t + S.p_hi, y_first) - hmax_t;
            int64_t pb = std::upper_bound(lo_t + S.p_lo, lo_t + S.p_hi, y_last) - lo_t;
            if (pb < pa) pb = pa;
            items.push_back(make_int4(o.second, (int)b, (int)pa, (int)pb));
        }
    }
}

static void axis_fill(double lo, double hi, int64_t n, int dtype, char *dst) {
    double step = n > 1 ? (hi - lo) / (double)(n - 1) : 0.0;
    for (int64_t i = 0; i < n; i++) {
        double v = n == 1 ? lo : lo + (double)i * step;
        if (dtype == GWN_F64) ((double *)dst)[i] = v;
        else ((float *)dst)[i] = (float)v;
    }
}

gwn_status eval2d_single(gwn_geom *g, const QuerySrc &src, void *w_out, int32_t *chi_out, void *b_out,
                         unsigned long long *cnt) {
    gwn_ctx *ctx = g->ctx;
    const ChainSet &cs = g->cs;
    if (src.dims[0] > MAX_NX) { set_error("gwn_eval: 2D grids are limited to 16384 columns"); return GWN_E_UNSUPPORTED; }
    Set2D S;
    S.c_lo = 0;
    S.c_hi = cs.n_chains;
    S.p_lo = 0;
    S.p_hi = cs.n_pieces;
    S.nx = src.dims[0];
    S.ny = src.dims[1];
    S.ax = cs.dtype == GWN_F64 ? (const void *)src.ax64[0] : (const void *)src.ax[0];
    S.ay = cs.dtype == GWN_F64 ? (const void *)src.ax64[1] : (const void *)src.ax[1];
    S.out_off = 0;
    // rows per work item: enough items to fill the device twice, at most 32,
    // and at most 64 KB of difference cells per block.  One set, passed by
    // value; its items are its row blocks (no work list to upload, no host
    // synchronisation).
    int64_t rows64 = S.ny / (2 * (int64_t)(ctx->sm_count > 0 ? ctx->sm_count : 152));
    const int rows0 = (int)(rows64 < 1 ? 1 : (rows64 > 32 ? 32 : rows64));
    const int cap_rows = (int)std::max<int64_t>(1, 16384 / (((int64_t)S.nx + 255) & ~(int64_t)255));
    const int rows = std::min(rows0, cap_rows);
    int64_t n_items = (S.ny + rows - 1) / rows;
    const int threads = 128;
    cudaError_t e = launch_eval2d_items(cs, nullptr, nullptr, &S, n_items, ctx->d_work_counter, rows, threads, S.nx,
                                        w_out, chi_out, b_out, cnt, ctx->d_status, ctx->sm_count, ctx->stream,
                                        ctx->d_cert, ctx->d_cert_count);
    if (e != cudaSuccess) return cuda_fail(e, "2D evaluation");
    return GWN_OK;
}

// ---- batched evaluation ------------------------------------------------------
struct BatchPlan {
    std::vector<double> key;         // grids + offsets fingerprint
    int threads = 128, rows = 4;
    void *dev = nullptr;             // axis tables + sets + items + counter
    size_t dev_bytes = 0;
    Set2D *d_sets = nullptr;
    int4 *d_items = nullptr;
    unsigned long long *d_counter = nullptr;
    int64_t n_items = 0, max_nx = 0;
    void *w_out = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t stream = nullptr;
    float tuned_ms = 0.f;
};

struct BatchCache {
    std::vector<BatchPlan *> plans;
};

void batch_cache_free(void *p) {
    BatchCache *c = (BatchCache *)p;
    for (BatchPlan *b : c->plans) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        if (b->dev) cudaFree(b->dev);
        delete b;
    }
    delete c;
}

static gwn_status plan_upload(gwn_geom *g, const gwn_queries *qs, int64_t n, const int64_t *out_off,
                              BatchPlan *P, int rows) {
    const ChainSet &cs = g->cs;
    size_t esz = cs.dtype == GWN_F64 ? 8 : 4;
    std::vector<Set2D> sets(n);
    size_t axis_bytes = 0;
    for (int64_t c = 0; c < n; c++) axis_bytes += esz * (qs[c].dims[0] + qs[c].dims[1]);
    axis_bytes = (axis_bytes + 255) & ~(size_t)255;
    std::vector<int4> items;
    int64_t max_nx = 0;
    for (int64_t c = 0; c < n; c++) {
        sets[c].nx = qs[c].dims[0];
        sets[c].ny = qs[c].dims[1];
        sets[c].c_lo = c;
        sets[c].c_hi = c + 1;
        sets[c].p_lo = cs.h_chain_piece_off[c];
        sets[c].p_hi = cs.h_chain_piece_off[c + 1];
        sets[c].out_off = out_off[c];
        max_nx = std::max(max_nx, sets[c].nx);
    }
    make_items(sets, qs, cs, rows, items);
    size_t sets_off = axis_bytes, items_off = (sets_off + sizeof(Set2D) * n + 15) & ~(size_t)15;
    size_t ctr_off = (items_off + sizeof(int4) * items.size() + 15) & ~(size_t)15;
    size_t total = ctr_off + 16;
    if (P->dev) { cudaFree(P->dev); P->dev = nullptr; }
    cudaError_t e = cudaMalloc(&P->dev, total);
    if (e != cudaSuccess) return cuda_fail(e, "batch plan");
    std::vector<char> host(total, 0);
    size_t off = 0;
    for (int64_t c = 0; c < n; c++) {
        axis_fill(qs[c].lo[0], qs[c].hi[0], qs[c].dims[0], cs.dtype, host.data() + off);
        sets[c].ax = (char *)P->dev + off;
        off += esz * qs[c].dims[0];
        axis_fill(qs[c].lo[1], qs[c].hi[1], qs[c].dims[1], cs.dtype, host.data() + off);
        sets[c].ay = (char *)P->dev + off;
        off += esz * qs[c].dims[1];
    }
    memcpy(host.data() + sets_off, sets.data(), sizeof(Set2D) * n);
    memcpy(host.data() + items_off, items.data(), sizeof(int4) * items.size());
    e = cudaMemcpy(P->dev, host.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "batch plan upload");
    P->dev_bytes = total;
    P->d_sets = (Set2D *)((char *)P->dev + sets_off);
    P->d_items = (int4 *)((char *)P->dev + items_off);
    P->d_counter = (unsigned long long *)((char *)P->dev + ctr_off);
    P->n_items = (int64_t)items.size();
    P->max_nx = max_nx;
    P->rows = rows;
    return GWN_OK;
}

}  // namespace gwn

using namespace gwn;

extern "C" GWN_API gwn_status gwn_eval_batch(gwn_geom *g, const gwn_queries *queries, int64_t n_chains,
                                             const int64_t *out_offsets, void *w_out, const gwn_plan *plan,
                                             gwn_stats *stats) {
    if (!g || g->kind != GWN_GEOM_BEZIER2D || !queries || !out_offsets || !w_out) {
        set_error("gwn_eval_batch: bad arguments");
        return GWN_E_INVALID;
    }
    if (n_chains != g->cs.n_chains) { set_error("gwn_eval_batch: one query grid per chain is required"); return GWN_E_INVALID; }
    if (g->cs.n_pieces > 0x7fffffff) { set_error("gwn_eval_batch: more than 2^31 - 1 monotone pieces"); return GWN_E_UNSUPPORTED; }
    for (int64_t c = 0; c < n_chains; c++) {
        const gwn_queries &q = queries[c];
        if (q.kind != GWN_QUERY_GRID || q.dim != 2 || q.dims[0] < 1 || q.dims[1] < 1 || q.dims[0] > MAX_NX ||
            q.dims[1] > (1 << 24) || out_offsets[c] < 0) {
            set_error("gwn_eval_batch: every chain needs a 2D grid (at most 16384 columns)");
            return GWN_E_INVALID;
        }
    }
    gwn_ctx *ctx = g->ctx;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    if (!g->batch_cache) g->batch_cache = new (std::nothrow) BatchCache();
    if (!g->batch_cache) { set_error("gwn_eval_batch: out of host memory"); return GWN_E_OOM; }
    BatchCache *C = (BatchCache *)g->batch_cache;
    // fingerprint of the request
    std::vector<double> key;
    key.reserve(6 * n_chains + 4);
    for (int64_t c = 0; c < n_chains; c++) {
        key.push_back(queries[c].lo[0]); key.push_back(queries[c].lo[1]);
        key.push_back(queries[c].hi[0]); key.push_back(queries[c].hi[1]);
        key.push_back((double)queries[c].dims[0]); key.push_back((double)queries[c].dims[1]);
        key.push_back((double)out_offsets[c]);
    }
    int want_threads = plan && plan->threads_per_block > 0 ? plan->threads_per_block : 0;
    int want_rows = plan && plan->rows_per_item > 0 ? plan->rows_per_item : 0;
    if (want_rows > 256 || (plan && (plan->threads_per_block < 0 || plan->threads_per_block > 256 ||
                                     plan->threads_per_block % 32 != 0))) {
        set_error("gwn_eval_batch: plan rows_per_item must be 0..256 and threads_per_block 0 or a multiple of 32 up "
                  "to 256");
        return GWN_E_INVALID;
    }
    int use_graph = plan ? plan->use_graph : 1;
    key.push_back((double)want_threads);
    key.push_back((double)want_rows);
    BatchPlan *P = nullptr;
    for (BatchPlan *b : C->plans)
        if (b->key == key) P = b;
    if (!P) {
        P = new (std::nothrow) BatchPlan();
        if (!P) { set_error("gwn_eval_batch: out of host memory"); return GWN_E_OOM; }
        P->key = key;
        // autotune: time each candidate shape (best of three after a warm-up) on the
        // real work list and keep the fastest
        std::vector<std::pair<int, int>> cands;
        if (want_threads && want_rows) cands.emplace_back(want_threads, want_rows);
        else {
            int ts[2] = {128, 256};
            int rs[5] = {4, 8, 16, 32, 64};
            for (int t : ts)
                for (int r : rs)
                    if ((!want_threads || t == want_threads) && (!want_rows || r == want_rows)) cands.emplace_back(t, r);
        }
        // shapes whose difference cells do not fit are dropped; wide grids get
        // as many rows per item as fit
        int64_t mx = 0;
        for (int64_t c = 0; c < n_chains; c++) mx = std::max<int64_t>(mx, queries[c].dims[0]);
        std::vector<std::pair<int, int>> fit;
        for (auto &cd : cands)
            if (eval2d_smem(g->cs.dtype, mx, cd.second) <= EVAL2D_SMEM_MAX) fit.push_back(cd);
        if (fit.empty()) {
            if (want_rows) {
                set_error("gwn_eval_batch: rows_per_item too large for the grid width (shared memory)");
                delete P;
                return GWN_E_INVALID;
            }
            int r = 64;
            while (r > 1 && eval2d_smem(g->cs.dtype, mx, r) > EVAL2D_SMEM_MAX) r--;
            for (auto &cd : cands) fit.emplace_back(cd.first, r);
            std::sort(fit.begin(), fit.end());
            fit.erase(std::unique(fit.begin(), fit.end()), fit.end());
        }
        cands = fit;
        float best = 1e30f;
        int bt = cands[0].first, br = cands[0].second;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (auto &cd : cands) {
            gwn_status s = plan_upload(g, queries, n_chains, out_offsets, P, cd.second);
            if (s != GWN_OK) { delete P; cudaEventDestroy(e0); cudaEventDestroy(e1); return s; }
            // one warm-up launch, then the fastest of three
            float ms = 1e30f;
            for (int rep = 0; rep < 4; rep++) {
                cudaEventRecord(e0, ctx->stream);
                e = launch_eval2d_items(g->cs, P->d_sets, P->d_items, nullptr, P->n_items, P->d_counter, cd.second, cd.first,
                                        P->max_nx, w_out, nullptr, nullptr, nullptr, ctx->d_status, ctx->sm_count,
                                        ctx->stream, ctx->d_cert, ctx->d_cert_count);
                cudaEventRecord(e1, ctx->stream);
                if (e != cudaSuccess) break;
                cudaEventSynchronize(e1);
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0 && t < ms) ms = t;
            }
            if (e != cudaSuccess) { delete P; cudaEventDestroy(e0); cudaEventDestroy(e1); return cuda_fail(e, "autotune"); }
            if (ms < best) { best = ms; bt = cd.first; br = cd.second; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        gwn_status s = plan_upload(g, queries, n_chains, out_offsets, P, br);
        if (s != GWN_OK) { delete P; return s; }
        P->threads = bt;
        P->tuned_ms = best;
        C->plans.push_back(P);
    }
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        cudaEventRecord(ctx->ev[0], ctx->stream);
    }
    bool graph_ok = use_graph && P->w_out == w_out && P->stream == ctx->stream && P->exec;
    if (use_graph && !graph_ok) {
        if (P->exec) { cudaGraphExecDestroy(P->exec); P->exec = nullptr; }
        if (P->graph) { cudaGraphDestroy(P->graph); P->graph = nullptr; }
        cudaStream_t cap = ctx->stream;
        bool own = false;
        if (cap == nullptr) {    // the legacy stream cannot be captured
            e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "capture stream");
            own = true;
        }
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = launch_eval2d_items(g->cs, P->d_sets, P->d_items, nullptr, P->n_items, P->d_counter, P->rows,
                                                 P->threads, P->max_nx, w_out, nullptr, nullptr, nullptr,
                                                 ctx->d_status, ctx->sm_count, cap, ctx->d_cert, ctx->d_cert_count);
            e = cudaStreamEndCapture(cap, &P->graph);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&P->exec, P->graph, 0);
        if (own) cudaStreamDestroy(cap);
        if (e != cudaSuccess) return cuda_fail(e, "graph capture");
        P->w_out = w_out;
        P->stream = ctx->stream;
    }
    if (use_graph) e = cudaGraphLaunch(P->exec, ctx->stream);
    else
        e = launch_eval2d_items(g->cs, P->d_sets, P->d_items, nullptr, P->n_items, P->d_counter, P->rows, P->threads, P->max_nx,
                                w_out, nullptr, nullptr, nullptr, ctx->d_status, ctx->sm_count, ctx->stream,
                                ctx->d_cert, ctx->d_cert_count);
    if (e != cudaSuccess) return cuda_fail(e, "batched launch");
    if (stats) {
        cudaEventRecord(ctx->ev[3], ctx->stream);
        e = cudaEventSynchronize(ctx->ev[3]);
        if (e != cudaSuccess) return cuda_fail(e, "sync");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[3]);
        int64_t nq = 0;
        for (int64_t c = 0; c < n_chains; c++) nq += queries[c].dims[0] * queries[c].dims[1];
        stats->n_queries = nq;
        stats->n_pairs = g->cs.n_pieces;
        stats->ms_boundary = ms;
        stats->ms_total = ms;
        stats->ms_prepare = P->tuned_ms;
        // one more launch, outside the timing, with the root counters on
        e = cudaMemsetAsync(ctx->d_cnt, 0, sizeof(unsigned long long) * CNT_NUM, ctx->stream);
        if (e == cudaSuccess)
            e = launch_eval2d_items(g->cs, P->d_sets, P->d_items, nullptr, P->n_items, P->d_counter, P->rows,
                                    P->threads, P->max_nx, w_out, nullptr, nullptr, ctx->d_cnt, ctx->d_status,
                                    ctx->sm_count, ctx->stream, ctx->d_cert, ctx->d_cert_count);
        unsigned long long c[CNT_NUM];
        if (e == cudaSuccess) e = cudaMemcpyAsync(c, ctx->d_cnt, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(e, "batched counters");
        stats->n_tri_tests = (int64_t)c[CNT_ROOTS];
        stats->n_root_iters = (int64_t)c[CNT_NEWTON];
        stats->n_cert = (int64_t)c[CNT_CERT];
        stats->n_cert_fixed = (int64_t)c[CNT_CERT_FIX];
    }
    return GWN_OK;
}

extern "C" GWN_API gwn_status gwn_batch_plan_get(gwn_geom *g, int32_t *threads, int32_t *rows) {
    if (!g || !g->batch_cache) { set_error("gwn_batch_plan_get: no batched plan yet"); return GWN_E_INVALID; }
    BatchCache *C = (BatchCache *)g->batch_cache;
    if (C->plans.empty()) { set_error("gwn_batch_plan_get: no batched plan yet"); return GWN_E_INVALID; }
    if (threads) *threads = C->plans.back()->threads;
    if (rows) *rows = C->plans.back()->rows;
    return GWN_OK;
}
