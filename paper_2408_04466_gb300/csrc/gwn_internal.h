// gwn_internal.h -- structures shared by the host library and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gwn.h"

namespace gwn {

// device counter slots (unsigned long long array of CNT_NUM)
enum {
    CNT_CUT_SIGN = 0,
    CNT_FP64 = 1,
    CNT_EXACT = 2,
    CNT_STACK_OVERFLOW = 3,
    CNT_TRI_TESTS = 4,
    CNT_PAIRS = 5,
    CNT_ROOTS = 6,
    CNT_TIMEOUT = 7,
    CNT_DEFER_TRAV = 8,
    CNT_DEFER_BTERM = 9,
    CNT_NEWTON = 10,         // 2D: root iterations (Newton or bisection steps)
    CNT_CERT = 11,           // 2D: crossings (or extremum rows) handed to the float64 certification
    CNT_CERT_FIX = 12,       // 2D: query counts the certification changed
    CNT_NUM = 16
};

// device status bits (int32)
enum {
    ST_STACK_OVERFLOW = 1,
    ST_TIMEOUT = 2,
    ST_EXPANSION_OVERFLOW = 4,
    ST_BAD_INPUT = 8,
    ST_CERT_OVERFLOW = 16    // 2D: more uncertain crossings than the certification list holds
};

// Orthonormal frame of the ray direction: n = -d/|d| (pole of the boundary
// term), e1, e2 span the plane orthogonal to d, dh = d/|d| (depth axis of the
// crossing hierarchy).  d keeps the caller's float32 bits for the exact
// predicates.
struct Frame {
    float e1[3], e2[3], n[3], dh[3];
    float d[3];
};

// The same frame in float64 plus the symbolic-perturbation direction dp: the
// first of e_x, e_y, e_z not parallel to d, minus its component along d.
struct Frame64 {
    double e1[3], e2[3], n[3], dh[3], dp[3];
};

// Grid or point query source (device side view).
struct QuerySrc {
    int kind;             // GWN_QUERY_POINTS / GWN_QUERY_GRID
    int dim;
    const float *pts;     // POINTS, float32 (3D)
    const double *pts64;  // POINTS, float64 (2D f64)
    const float *ax[3];   // GRID: per-axis float32 coordinate tables
    const double *ax64[3];
    int64_t dims[3];
    int64_t n;
};

struct BvhNode {          // internal node: boxes of both children in the d-frame
    float4 lo;            // child0: x0, x1, y0, y1
    float4 hi;            // child1: x0, x1, y0, y1
    float4 z;             // child0 zmax, child1 zmax, child0 ref (int bits), child1 ref (int bits)
};
// child ref: >= 0 internal node index; < 0 leaf ~(sorted triangle index)

// Bin grid of the projection plane (frame of d): the bin of a coordinate v
// along x is clamp(floor((v - x0) * invx), 0, nbx - 1), likewise along y;
// [x0, x1] x [y0, y1] bounds every padded triangle box.
struct BinParams {
    float x0 = 0.f, y0 = 0.f, x1 = 0.f, y1 = 0.f, invx = 0.f, invy = 0.f;
    int nbx = 0, nby = 0;   // 0: no bins
};

struct MeshBvh {
    bool valid = false;
    float dkey[3] = {0, 0, 0};
    int64_t n = 0;             // triangles
    BvhNode *nodes = nullptr;  // n - 1
    void *block = nullptr;     // one allocation holding bframe, tris, tbox and nodes
    float4 *tris = nullptr;    // 3 float4 per sorted triangle (xyz of v0, v1, v2)
    float4 *tbox = nullptr;    // 2 float4 per sorted triangle: (x0, x1, y0, y1), (zmax, 0, 0, 0)
    int root = 0;              // ref of the root
    float scene_radius = 0.f;  // max |v|_2 over the mesh vertices
    Frame frame;
    float4 *bframe = nullptr;  // 2 float4 per boundary record: A.(e1, e2, n) hi (+ w), lo
    float box_bounds[4] = {0, 0, 0, 0};   // min x0, max x1, min y0, max y1 of the padded boxes
    // bins, built on demand by bins_build (n_bin_entries = 0: none, the tree
    // is used): bin b = j * nbx + i lists entries [bin_start[b],
    // bin_start[b + 1]) by decreasing zmax
    bool bins_tried = false;
    int64_t queries_seen = 0;       // queries evaluated since this (mesh, d) was prepared
    void *bin_block = nullptr;      // one allocation holding the three bin arrays
    BinParams bins;
    int64_t n_bin_entries = 0;
    int64_t bin_maxlen = 0;
    int32_t *bin_start = nullptr;   // nbx * nby + 1
    float2 *bin_zt = nullptr;       // (zmax, sorted triangle index as int bits) per entry
    float4 *bin_box = nullptr;      // padded box (x0, x1, y0, y1) per entry
};

// Bicubic Bezier patches (parametric surfaces): control nets, and per ray
// direction their projection into the frame of d with a 2D bin grid over the
// projected boxes (all rays share d, so a ray is a point of the plane).
struct PatchSet {
    int64_t n = 0;                   // patches
    std::vector<float> h_ctrl;       // host [n][4][4][3]
    int segments = 0;                // polyline segments per boundary curve
    bool valid = false;
    float dkey[3] = {0, 0, 0};
    Frame frame;
    float4 *bframe = nullptr;        // 2 float4 per boundary record (as MeshBvh::bframe)
    float4 *qnet = nullptr;          // [n][16]: (e1.P, e2.P, dh.P, 0) per control point
    float4 *box = nullptr;           // [n]: (xmin, xmax, ymin, ymax) of the projected net
    float *zmax = nullptr;           // [n]: max dh.P
    int32_t *bin_off = nullptr;      // [nbx * nby + 1]
    int32_t *bin_idx = nullptr;
    int nbx = 0, nby = 0;
    float bx0 = 0.f, by0 = 0.f, binv = 0.f;   // cell (i, j) = [bx0 + i / binv, ...) x [by0 + j / binv, ...)
    // boundary curves (patch edge curves of nonzero net multiplicity), each
    // sampled at segments + 1 vertices in its canonical orientation
    int64_t n_bcurves = 0;
    std::vector<int32_t> h_bedge;    // [n][4]: curve << 1 | (edge runs against the canonical order), or -1
    std::vector<float4> h_pl_xyz;    // [n_bcurves * (segments + 1)]: sample vertices (float32, w = 0)
    std::vector<float> h_pl_dev;     // [n_bcurves * segments]: bound on the distance between arc and chord
    int32_t *bedge = nullptr;        // device copies
    float4 *pl_xyz = nullptr;
    float *pl_dev = nullptr;
    float4 *pl_proj = nullptr;       // per direction: (e1.v, e2.v, dh.v, 0) of the sample vertices
};

// Boundary loops as vertex sequences: loop j is vid[off[j] .. off[j+1]-1],
// closing back to its first vertex.
struct BoundaryLoops {
    std::vector<int64_t> off;   // n_loops + 1, in edges
    std::vector<int32_t> vid;   // loop vertex ids
};

// Chain unit directed edges (every vertex with equal in- and out-degree)
// into closed loops.
gwn_status chain_unit_edges(std::vector<std::pair<int32_t, int32_t>> &bedges, int64_t nv, BoundaryLoops &out);

// Device pointers of one 2D chain set.
struct ChainSet {
    int dtype = GWN_F32;
    int64_t n_chains = 0, n_ctrl = 0, n_seg = 0, n_pieces = 0;
    void *ctrl = nullptr;          // [n_ctrl][2] of dtype
    int64_t *chain_off = nullptr;  // device [n_chains + 1] control point offsets
    // y-monotone pieces (ordered by their lowest y within each chain): y at
    // the ends of the piece's parameter interval
    double *piece_y = nullptr;     // [n_pieces][2] (y at u0, y at u1)
    void *piece_yT = nullptr;      // piece_y in the chain dtype (aliases piece_y for float64)
    // point queries: the pieces' conservative x ranges (control hull of their
    // segment, chain dtype, [n_pieces][2]) and a y-bucket index of the pieces
    void *piece_xT = nullptr;
    // per piece, in the chain dtype: the piece in local power form (see
    // bezier2d.cu) -- one contiguous 16-byte aligned record per piece
    void *piece_rec = nullptr;
    // per piece, for the float64 certification of uncertain crossings: the
    // index of its segment's first control point, its parameter interval
    // [u0, u1] on the segment, the pieces sharing its ends when an end is an
    // interior extremum of y (else -1), and per end the bound on the
    // difference between the stored end value (piece_yT) and the curve's
    // value there (0 at control points; chain dtype)
    int64_t *piece_seg = nullptr;
    double2 *piece_u = nullptr;
    // every end bound is below 8u (|y_a| + |y_b|) + eps_abs (u the unit
    // roundoff of the chain dtype, y_a, y_b the piece's end values): a test
    // that needs no table read rules out almost every row first
    double eps_abs = 0.0;
    int2 *piece_part = nullptr;
    void *piece_eps = nullptr;
    int32_t *bucket_off = nullptr;     // [n_buckets + 1]
    int32_t *bucket_idx = nullptr;     // piece indices, bucket by bucket
    int32_t n_buckets = 0;
    double bucket_y0 = 0.0, bucket_inv_h = 0.0;   // bucket(y) = floor((y - y0) * inv_h), in the chain dtype
    std::vector<int64_t> h_chain_off, h_chain_piece_off;
    // host, per piece (pieces of a chain ordered by their lowest y): that
    // lowest y and the running maximum of the highest y over the chain's
    // pieces so far, both rounded to the chain's precision
    std::vector<double> h_piece_lo, h_piece_hmax;
};

// One 2D evaluation set: chains [c_lo, c_hi) (their pieces [p_lo, p_hi)) on
// one nx x ny grid written at out_off.
struct Set2D {
    int64_t c_lo, c_hi;
    int64_t p_lo, p_hi;
    int64_t nx, ny;
    const void *ax, *ay;      // device axis tables (chain dtype)
    int64_t out_off;
};

struct Arena {            // grow-only scratch owned by a context
    void *ptr = nullptr;
    size_t bytes = 0;
};

// Device coordinate tables of one query grid (per context, reused while the
// same grid is evaluated again).
struct AxisCache {
    double lo[3], hi[3];
    int64_t dims[3];
    int dim, dtype;
    void *dev = nullptr;
    size_t bytes = 0;
};

}  // namespace gwn

struct gwn_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    int *d_status = nullptr;                  // device status bits
    unsigned long long *d_cnt = nullptr;      // device counters [CNT_NUM]
    int32_t *d_defer_count = nullptr;         // length of the deferred-query list
    int2 *d_tpairs = nullptr;                 // traversal: unsettled (query, triangle) pairs [GWN_TPAIR_CAP]
    unsigned long long *d_work_counter = nullptr;   // 2D work-item counter
    void *mesh_batch_cache = nullptr;         // plans of gwn_eval_meshes (meshbatch.cu)
    int4 *d_cert = nullptr;                   // 2D certification list [2 * GWN_CERT_CAP] (two int4 per entry)
    int32_t *d_cert_count = nullptr;
    int32_t *d_tpair_count = nullptr;
    gwn::Arena scratch[9];                    // 0 chi, 1 staged points, 2 2D batch, 3 host-eval w, 4 deferred list,
                                              // 5 per-line crossing lists, 6 mesh intake and LBVH build, 7 bin sort,
                                              // 8 2D point order
    // (slot 7 also holds the deferred (ray, patch) pairs of the patch path)
    std::vector<gwn::AxisCache> axis_cache;   // most recent grids, at most 64
    cudaEvent_t ev[8];
    bool events = false;
    // lifetime: geometries keep their context alive; gwn_ctx_destroy releases
    // it once no geometry refers to it (guarded by a library-wide mutex)
    int64_t geom_refs = 0;
    bool destroy_requested = false;
};

struct gwn_geom {
    gwn_ctx *ctx = nullptr;
    int kind = 0;
    int dtype = GWN_F32;
    // mesh
    int64_t nv = 0, nf = 0;
    int crossing_index = GWN_INDEX_AUTO;   // GWN_INDEX_TREE: never the bins
    float *dV = nullptr;
    int32_t *dF = nullptr;
    std::vector<int64_t> loop_off;     // host, n_loops + 1 (in edges)
    std::vector<int32_t> loop_vid;     // host, n_edges vertex ids
    float4 *bseq = nullptr;            // device loop sequence (n_edges + n_loops records)
    int32_t *bseq_vid = nullptr;       // device vertex id per record
    int64_t n_bseq = 0;
    // boundary vertex -> records lists (gradient scatter), built on demand
    int32_t *d_edge_rec = nullptr;     // device: record index ending each boundary edge, in edge order
    int32_t *d_bvert = nullptr;
    int64_t *d_brec_off = nullptr;
    int32_t *d_brecs = nullptr;
    int64_t n_bvert = 0;
    gwn::MeshBvh bvh;
    // 2D
    gwn::ChainSet cs;
    // parametric patches
    gwn::PatchSet ps;
    // batched launch cache
    void *batch_cache = nullptr;
};

namespace gwn {

// ---- helpers implemented in api.cpp -------------------------------------
void set_error(const std::string &msg);
gwn_status cuda_fail(cudaError_t e, const char *what);
void *arena_get(gwn_ctx *ctx, int slot, size_t bytes, cudaError_t *err);
Frame make_frame(const float d[3]);
void ctx_add_geometry(gwn_ctx *ctx);      // a geometry now refers to ctx (released by gwn_geom_destroy)
Frame64 make_frame64(const float d[3]);

// ---- launchers (return the first CUDA error) -------------------------------
cudaError_t bvh_build(gwn_geom *g, const Frame &fr, cudaStream_t st);
void bvh_free(MeshBvh &b);
// Builds the 2D bin index of a built tree once (a later call returns at
// once); keeps it when it is compact, else leaves n_bin_entries = 0.
// Synchronises the stream.
cudaError_t bins_build(gwn_geom *g, cudaStream_t st);
// Mesh intake on the device (V: nv x 3 float32, F: nf x 3 int32, both on the
// device): fails with GWN_E_INVALID on a non-finite coordinate or a face index
// outside [0, nv); otherwise returns the boundary unit edges (each undirected
// edge with net multiplicity m over the faces' directed edges, as |m| copies
// in the direction of m's sign), in no fixed order.  Synchronises the stream.
gwn_status mesh_intake_device(gwn_ctx *ctx, const float *dV, int64_t nv, const int32_t *dF, int64_t nf,
                              std::vector<std::pair<int32_t, int32_t>> &bedges);
// bseq[i] = (V[v], w), bseq_vid[i] = v for code[i] = v (w = 1) or ~v (w = 0,
// the first record of a loop).
cudaError_t launch_bseq(const float *dV, const int32_t *code, int64_t n, float4 *bseq, int32_t *bseq_vid,
                        cudaStream_t st);

// Crossing counts chi[q.n].  defer / defer_count: the same deferred-list
// scratch as launch_bterm3d (used and emptied before it returns in stream
// order, so the two may share it); pairs / pair_count: GWN_TPAIR_CAP
// unsettled (query, triangle) pairs; lines: scratch of
// traverse_lines_bytes(b, q) bytes for grid queries with d parallel to a grid
// axis (one traversal per grid line), or NULL to traverse every query.
#define GWN_TPAIR_CAP 65536
size_t traverse_lines_bytes(const MeshBvh &b, const QuerySrc &q);
cudaError_t launch_traverse(const MeshBvh &b, const QuerySrc &q, int32_t *chi, int32_t *defer,
                            int32_t *defer_count, int2 *pairs, int32_t *pair_count, int32_t *lines,
                            unsigned long long *cnt, int *status, int sm_count, cudaStream_t st, bool use_bins = true);

// Boundary term + epilogue (w = chi + B; inside_out, when given, gets
// w >= 0.5 as one byte per query).  defer: int32 scratch of q.n entries for
// the deferred-query list; defer_count: one device int32.
cudaError_t launch_bterm3d(const float4 *bseq, const float4 *bframe, int64_t n_bseq, const Frame &fr,
                           const Frame64 &f64, const QuerySrc &q, const int32_t *chi, float *w_out, float *b_out,
                           int32_t *defer, int32_t *defer_count, unsigned long long *cnt, int *status, int sm_count,
                           cudaStream_t st, uint8_t *inside_out = nullptr);
// Boundary records in the frame of d (double-float), 2 float4 per record.
cudaError_t launch_bframe(const float4 *bseq, int64_t n, const Frame &fr, float4 *out, cudaStream_t st);

cudaError_t launch_grad_p(const float4 *bseq, int64_t nb, const QuerySrc &q, const float *grad_w, float *grad_p,
                          cudaStream_t st);
int grad_v_chunks(int64_t nq, int64_t nb, int sm_count);
// both gradients from one pass over the (query, edge) pairs, two edges per
// thread (edge_rec: the record ending each edge); partial_p holds
// grad_pv_partial_p_bytes(nq, n_edges) bytes, partial 8 floats per (chunk,
// record); grad_pv_chunks gives the number of query chunks
size_t grad_pv_partial_p_bytes(int64_t nq, int64_t n_edges);
int grad_pv_chunks(int64_t nq, int64_t n_edges, int sm_count);
cudaError_t launch_grad_pv(const float4 *bseq, int64_t nb, const int32_t *edge_rec, int64_t n_edges,
                           const QuerySrc &q, const float *grad_w, int n_chunks, float *partial, float *partial_p,
                           float *rec_grad, const int32_t *bvert, const int64_t *rec_off, const int32_t *recs,
                           int64_t n_bvert, float *grad_p, float *grad_V, cudaStream_t st);
cudaError_t launch_grad_v(const float4 *bseq, int64_t nb, const QuerySrc &q, const float *grad_w, int n_chunks,
                          float *partial, float *rec_grad, const int32_t *bvert, const int64_t *rec_off,
                          const int32_t *recs, int64_t n_bvert, float *grad_V, cudaStream_t st);

cudaError_t launch_bruteforce3d(const float *V, const int32_t *F, int64_t nf, const QuerySrc &q, float *w_out,
                                int sm_count, cudaStream_t st);

// 2D
// 2D evaluation at point queries (one +x ray per query, y-bucket index).
// Parametric patches: prepare the per-direction tables of g->ps (host and
// device), and the signed crossing counts chi[q.n] of the rays p + t d.
gwn_status patches_prepare(gwn_geom *g, const float d[3]);
// dpairs: optional list (dcap int2 entries, counter dcount) of the long
// (ray, patch) pairs, settled by a second kernel; without it every pair is
// settled in place.  Results are the same.
constexpr int PATCH_DEFER_CAP = 1 << 21;
cudaError_t launch_chi_patches(const PatchSet &ps, const QuerySrc &q, int32_t *chi, unsigned long long *cnt,
                               int *status, cudaStream_t st, int2 *dpairs, int32_t *dcount, int dcap,
                               int sm_count);
void patches_free(PatchSet &ps);

// Point queries of a chain set (one +x ray each).  order_buf (optional):
// eval2d_points_order_bytes(cs, q.n) bytes of device scratch; when given and
// that size is nonzero, the queries are evaluated in the order of their
// y-buckets (a counting sort per call) so that the warps walk the same
// bucket lists.  Results do not depend on it.
constexpr int64_t EVAL2D_POINTS_ORDER_MIN = 65536;            // fewer queries: as given
constexpr int64_t EVAL2D_POINTS_ORDER_MAX_BUCKETS = 1 << 16;  // more buckets: as given (one-block scan)
size_t eval2d_points_order_bytes(const ChainSet &cs, int64_t n);
cudaError_t launch_eval2d_points(const ChainSet &cs, const QuerySrc &q, void *w_out, int32_t *chi_out, void *b_out,
                                 unsigned long long *cnt, int *status, cudaStream_t st, int4 *cert,
                                 int32_t *cert_count, int32_t *order_buf, int sm_count);
// 2D evaluation over work items: either a device work list (d_sets, d_items)
// or one set passed by value (single, items = its row blocks).
// shared memory of eval2d_kernel for work items of `rows` grid rows on grids
// up to max_nx columns (one int difference cell per row and column, the
// width rounded up to 256), and the most one block may take (sm_103a opt-in
// limit).  Blocks have at most 256 threads.
size_t eval2d_smem(int dtype, int64_t max_nx, int rows);
constexpr size_t EVAL2D_SMEM_MAX = 227 * 1024;
// The launch is followed by the certification pass: crossings whose float
// position lies within its error bound of a query column (and rows within
// rounding of an interior extremum of y) were listed in cert by the main
// kernel; each listed (piece, row, column) is decided again in float64 from
// the control points and the count of a query corrected where it differs.
// cert holds 2 * GWN_CERT_CAP int4; cert_count is reset by the launch.
#define GWN_CERT_CAP (1 << 18)
cudaError_t launch_eval2d_items(const ChainSet &cs, const Set2D *d_sets, const int4 *d_items, const Set2D *single,
                                int64_t n_items,
                                unsigned long long *d_counter, int rows_per_item, int threads, int64_t max_nx,
                                void *w_out, int32_t *chi_out, void *b_out, unsigned long long *cnt, int *status,
                                int sm_count, cudaStream_t st, int4 *cert, int32_t *cert_count);
gwn_status eval2d_single(gwn_geom *g, const QuerySrc &src, void *w_out, int32_t *chi_out, void *b_out,
                         unsigned long long *cnt);
void batch_cache_free(void *p);
void mesh_batch_cache_free(void *p);
// coordinate table of a grid axis: lo + i ((hi - lo) / (n - 1)) in float64
void axis_table(double lo, double hi, int64_t n, std::vector<double> &out);

cudaError_t launch_bruteforce2d(const ChainSet &cs, const QuerySrc &q, void *w_out, int sm_count,
                                cudaStream_t st);

}  // namespace gwn
