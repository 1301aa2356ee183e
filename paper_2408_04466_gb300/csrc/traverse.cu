// traverse.cu -- signed crossing count chi_d(p) of the ray p + t d (Eq. chi).
//
// All rays share the direction d, so the hierarchy is built in the frame
// (e1, e2, dh) of d: a ray is a point (p.e1, p.e2) of the projection plane
// plus the half-line of depths > p.dh.  A child box (x0, x1, y0, y1, zmax)
// can hold a crossing only if the projected point lies in [x0,x1]x[y0,y1] and
// zmax >= p.dh: five comparisons per child instead of a slab test.  Boxes
// and the query point are padded by bounds on their float32 rounding and on
// the residual non-orthogonality of the rounded frame, so culling never drops
// a crossing; every surviving triangle is decided by exact predicates.
//
// The signed crossings are accumulated per query with float32-filtered
// predicates; a query one of whose signs the float32 filter cannot settle is
// appended to a deferred list and recounted by a second kernel with the full
// predicates (float64 filter, then exact expansions), so the hot loop holds
// no call.  The traversal stack holds at most the tree depth, bounded by GWN_STACK;
// overflow or the iteration limit sets a status bit and a counter and marks
// the query result as invalid (INT32_MIN).
#include <stdlib.h>

#include "gwn_internal.h"
#include "traverse.cuh"

namespace gwn {

// Scattered points: one ray per thread, float32 predicates; unsettled
// queries are deferred.
__global__ void __launch_bounds__(256) traverse_kernel(const BvhNode *__restrict__ nodes,
                                                       const float4 *__restrict__ tris, int root, Frame fr,
                                                       TravParams tp, QuerySrc q, int32_t *__restrict__ chi,
                                                       int32_t *defer, int32_t *defer_count, int2 *pairs,
                                                       int32_t *pair_count, unsigned long long *cnt, int *status) {
    int64_t idx = q.kind == GWN_QUERY_GRID ? grid_tile_query(q) : (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < 0 || idx >= q.n) return;
    int acc, ntests = 0;
    bool unsure = false;
    bool ok = traverse_ray<true>(nodes, tris, root, fr, tp, query_point3(q, idx), idx, acc, unsure, pairs,
                                 pair_count, ntests, cnt, status);
    if (cnt) {                                   // statistics: one atomic per warp
        unsigned m = __activemask();
        int tot = __reduce_add_sync(m, ntests);
        if ((threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(&cnt[CNT_TRI_TESTS], (unsigned long long)tot);
    }
    if (ok && unsure)
        defer_query(defer, defer_count, idx);
    else
        chi[idx] = ok ? acc : INT32_MIN;
}

// Deferred queries (a float32 predicate could not settle a sign): the same
// traversal with the full predicates, persistent grid over the list.
__global__ void __launch_bounds__(128) traverse_careful_kernel(const BvhNode *__restrict__ nodes,
                                                               const float4 *__restrict__ tris, int root, Frame fr,
                                                               TravParams tp, QuerySrc q,
                                                               int32_t *__restrict__ chi,
                                                               const int32_t *__restrict__ defer,
                                                               const int32_t *defer_count, unsigned long long *cnt,
                                                               int *status) {
    int64_t n = *defer_count;
    if (n > q.n) n = q.n;
    if (cnt && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&cnt[CNT_DEFER_TRAV], (unsigned long long)n);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t idx = defer[i];
        if (idx < 0 || idx >= q.n) { atomicOr(status, ST_BAD_INPUT); continue; }
        int acc, ntests = 0;
        bool unsure = false;
        bool ok = traverse_ray<false>(nodes, tris, root, fr, tp, query_point3(q, idx), idx, acc, unsure, nullptr,
                                      nullptr, ntests, cnt, status);
        if (cnt) atomicAdd(&cnt[CNT_TRI_TESTS], (unsigned long long)ntests);
        chi[idx] = ok ? acc : INT32_MIN;
    }
}

// Unsettled (query, triangle) pairs of the float32 passes: one thread per
// pair, full predicates, the signed crossing added to the query's count
// (left alone when the query's traversal failed and its count is invalid).
__global__ void __launch_bounds__(128) traverse_pairs_kernel(const float4 *__restrict__ tris, Frame fr, QuerySrc q,
                                                             int32_t *chi, const int2 *__restrict__ pairs,
                                                             const int32_t *pair_count, unsigned long long *cnt,
                                                             int *status) {
    int64_t n = *pair_count;
    if (n > GWN_TPAIR_CAP) n = GWN_TPAIR_CAP;
    if (cnt && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&cnt[CNT_DEFER_TRAV], (unsigned long long)n);
    float3 D = make_float3(fr.d[0], fr.d[1], fr.d[2]);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int2 pr = pairs[i];
        if (pr.x < 0 || pr.x >= q.n) { atomicOr(status, ST_BAD_INPUT); continue; }
        if (chi[pr.x] == INT32_MIN) continue;
        float3 p = query_point3(q, pr.x);
        float4 a = __ldg(&tris[3 * pr.y]), b = __ldg(&tris[3 * pr.y + 1]), c = __ldg(&tris[3 * pr.y + 2]);
        int r = tri_crossing(make_float3(a.x, a.y, a.z), make_float3(b.x, b.y, b.z), make_float3(c.x, c.y, c.z), p,
                             D, cnt, status);
        if (r) atomicAdd(&chi[pr.x], r);
    }
}

// Warp-packet traversal for grid queries: the 32 rays of a warp (a 4x4x2
// grid tile, neighbours in the projection plane) walk the tree together.
// The traversal order is warp-uniform: at a node each lane tests its own ray
// against both child boxes and the warp descends into a child if any lane's
// ray hits it; the stack lives in shared memory (one per warp).  Node loads
// are warp-uniform (one broadcast per warp).
//
// Leaves are compacted: a leaf hit by the ray boxes of a few lanes appends
// one (triangle, lane) pair per such lane to a per-warp buffer, and whenever
// 32 pairs are pending every lane tests one pair (the float32 crossing test,
// for the query of the pair's lane, whose point it fetches with a shuffle)
// and adds the result to that lane's count in shared memory.  So a triangle
// test costs one lane-slot instead of a warp-wide pass per visited leaf.
// A query with an unsettled float32 sign is deferred to
// traverse_careful_kernel.  Lanes outside the grid take part with an empty
// box.  Requires fewer than 2^26 triangles (pair = triangle << 5 | lane).
__global__ void __launch_bounds__(256) traverse_packet_kernel(const BvhNode *__restrict__ nodes,
                                                              const float4 *__restrict__ tris,
                                                              const float4 *__restrict__ tbox, int root, Frame fr,
                                                              TravParams tp, QuerySrc q, int32_t *__restrict__ chi,
                                                              int32_t *defer, int32_t *defer_count, int2 *tpairs,
                                                              int32_t *tpair_count, unsigned long long *cnt,
                                                              int *status) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t idx = grid_tile_query(q);
    bool valid = idx >= 0 && idx < q.n;
    float3 p = valid ? query_point3(q, idx) : make_float3(0.f, 0.f, 0.f);
    float3 D = make_float3(fr.d[0], fr.d[1], fr.d[2]);
    float p1 = fmaf(p.z, fr.e1[2], fmaf(p.y, fr.e1[1], p.x * fr.e1[0]));
    float p2 = fmaf(p.z, fr.e2[2], fmaf(p.y, fr.e2[1], p.x * fr.e2[0]));
    float p3 = fmaf(p.z, fr.dh[2], fmaf(p.y, fr.dh[1], p.x * fr.dh[0]));
    float pad = fmaf(tp.pad_rel, fabsf(p.x) + fabsf(p.y) + fabsf(p.z), tp.pad_abs);
    float xlo = p1 - pad, xhi = p1 + pad, ylo = p2 - pad, yhi = p2 + pad, zlo = p3 - pad;
    if (!valid) { xlo = 3.4e38f; xhi = -3.4e38f; }     // never hits
    __shared__ int s_stack[256 / 32][GWN_STACK];
    __shared__ int s_pair[256 / 32][64];
    __shared__ int s_acc[256 / 32][32];
    __shared__ unsigned s_uns[256 / 32];
    int *stack = s_stack[w];
    int *pairs = s_pair[w];
    s_acc[w][lane] = 0;
    if (lane == 0) s_uns[w] = 0u;
    __syncwarp();
    int ntests = 0;
    int npairs = 0;                               // warp-uniform
    // test the first min(npairs, 32) pending pairs, one per lane, and move
    // the rest to the front; returns the number still pending (< 32)
    auto flush = [&](int n) -> int {
        int m = n < 32 ? n : 32;
        int pr = lane < m ? pairs[lane] : -1;
        int ql = pr >= 0 ? (pr & 31) : lane;
        float qx = __shfl_sync(FULL, p.x, ql), qy = __shfl_sync(FULL, p.y, ql), qz = __shfl_sync(FULL, p.z, ql);
        int qi = __shfl_sync(FULL, (int)idx, ql);
        if (pr >= 0) {
            int t = pr >> 5;
            float4 a = __ldg(&tris[3 * t]), b = __ldg(&tris[3 * t + 1]), c = __ldg(&tris[3 * t + 2]);
            bool uns = false;
            int r = tri_crossing_fast(make_float3(a.x, a.y, a.z), make_float3(b.x, b.y, b.z),
                                      make_float3(c.x, c.y, c.z), make_float3(qx, qy, qz), D, uns);
            if (r) atomicAdd(&s_acc[w][ql], r);
            if (uns) {
                bool whole = false;
                defer_pair(tpairs, tpair_count, qi, t, whole);
                if (whole) atomicOr(&s_uns[w], 1u << ql);
            }
        }
        int rem = n - m;
        __syncwarp();
        int moved = lane < rem ? pairs[m + lane] : 0;
        __syncwarp();
        if (lane < rem) pairs[lane] = moved;
        __syncwarp();
        return rem;
    };
    int sp = 0;
    int node = root;
    bool bad = false;
    for (int64_t iter = 0;; iter++) {
        if (iter > tp.max_iter) {
            if (lane == 0) {
                atomicOr(status, ST_TIMEOUT);
                if (cnt) atomicAdd(&cnt[CNT_TIMEOUT], 1ull);
            }
            bad = true;
            break;
        }
        if (node >= tp.n_internal || ~node >= tp.n_leaves) {   // corrupt reference: report, never read
            atomicOr(status, ST_BAD_INPUT);
            bad = true;
            break;
        }
        if (node < 0) {
            int t = ~node;
            float4 bx = __ldg(&tbox[2 * t]), bz = __ldg(&tbox[2 * t + 1]);
            bool hit = box_hit(bx.x, bx.y, bx.z, bx.w, bz.x, xlo, xhi, ylo, yhi, zlo);
            unsigned m = __ballot_sync(FULL, hit);
            if (m) {
                if (hit) pairs[npairs + __popc(m & ((1u << lane) - 1u))] = (t << 5) | lane;
                npairs += __popc(m);
                ntests += hit;
                __syncwarp();
                if (npairs >= 32) npairs = flush(npairs);
            }
            if (sp == 0) break;
            node = stack[--sp];
            continue;
        }
        const BvhNode nd = nodes[node];
        bool h0 = box_hit(nd.lo.x, nd.lo.y, nd.lo.z, nd.lo.w, nd.z.x, xlo, xhi, ylo, yhi, zlo);
        bool h1 = box_hit(nd.hi.x, nd.hi.y, nd.hi.z, nd.hi.w, nd.z.y, xlo, xhi, ylo, yhi, zlo);
        bool a0 = __any_sync(FULL, h0), a1 = __any_sync(FULL, h1);
        int c0 = __float_as_int(nd.z.z), c1 = __float_as_int(nd.z.w);
        if (a0 && a1) {
            if (sp >= GWN_STACK) {
                if (lane == 0) {
                    atomicOr(status, ST_STACK_OVERFLOW);
                    if (cnt) atomicAdd(&cnt[CNT_STACK_OVERFLOW], 1ull);
                }
                bad = true;
                break;
            }
            stack[sp++] = c1;
            __syncwarp();
            node = c0;
        } else if (a0) {
            node = c0;
        } else if (a1) {
            node = c1;
        } else {
            if (sp == 0) break;
            node = stack[--sp];
        }
    }
    if (!bad)
        while (npairs > 0) npairs = flush(npairs);
    __syncwarp();
    int acc = s_acc[w][lane];
    bool unsure = (s_uns[w] >> lane) & 1u;
    if (valid) {
        if (!bad && unsure)
            defer_query(defer, defer_count, idx);
        else
            chi[idx] = bad ? INT32_MIN : acc;
    }
    if (cnt) {                                   // statistics: one atomic per block
        __shared__ unsigned s_tests;
        if (threadIdx.x == 0) s_tests = 0;
        __syncthreads();
        atomicAdd(&s_tests, (unsigned)ntests);
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(&cnt[CNT_TRI_TESTS], (unsigned long long)s_tests);
    }
}

// Crossing count from the 2D bins (bvh.cu): the query's padded ray box
// [xlo, xhi] x [ylo, yhi] covers bins [bin(xlo), bin(xhi)] x [bin(ylo),
// bin(yhi)] (usually one).  A triangle box overlapping the ray box shares
// with it the point (max(x0, xlo), max(y0, ylo)), whose bin, by the
// monotonicity of bin_of, is (max(bin(x0), bin(xlo)), max(bin(y0), bin(ylo)))
// and lies in both bin ranges: the pair is tested in that bin only, so every
// triangle that passes the tree's leaf test (the same box_hit) is tested
// exactly once, and the count equals the tree traversal's.  A bin's list runs
// by decreasing zmax, so its scan stops at the first box behind the query.
// The leaf tests go through the same per-warp (triangle, lane) compaction as
// traverse_packet_kernel.  GRID: warp tiles of the grid; otherwise one point
// per thread.  Requires fewer than 2^26 triangles.
// Crossing counts from the 2D bins: see chi_bins_block.  GRID: warp tiles of
// the grid; otherwise one point per thread.
template <bool GRID>
__global__ void __launch_bounds__(256, 5) chi_bins_kernel(const int32_t *__restrict__ bin_start,
                                                       const float2 *__restrict__ bin_zt,
                                                       const float4 *__restrict__ bin_box, BinParams bp,
                                                       const float4 *__restrict__ tris, Frame fr, TravParams tp,
                                                       QuerySrc q, int32_t *__restrict__ chi, int32_t *defer,
                                                       int32_t *defer_count, int2 *tpairs, int32_t *tpair_count,
                                                       unsigned long long *cnt) {
    const int64_t idx = GRID ? grid_tile_query(q) : (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    chi_bins_block(bin_start, bin_zt, bin_box, bp, tris, fr, tp, q, idx, 0, chi, defer, defer_count, tpairs,
                   tpair_count, cnt);
}

// Ray reuse for grid queries when d is parallel to grid axis k: every
// query on a grid line along k shares the ray line (the "Optimization" of
// the one-shot algorithm, in 3D).  For an edge AB,
//   det[A-p, B-p, d] = d_k ((A x B)_k + ((B-A) x p)_k)
// does not depend on p_k, so the edge signs, hence which triangles the line
// crosses and with which sign, are the same for every query on the line.
// traverse_lines_kernel: one thread per line traverses once from the line's
// first query (the one farthest back along d) and stores the crossed
// triangles, GWN_LINE_MAX per line: the crossing's coordinate along axis k
// (float64 plane intersection, stored as float) with a conservative band,
// and (triangle << 2 | code), code 0: +1, 1: -1, 2: an exactly zero edge
// determinant (the perturbed tie-break depends on p_k, so each query settles
// that pair on its own); a count of -1 marks a line with more crossings, -2 a
// failed traversal.
// lines_count_kernel: one thread per query counts the stored crossings in
// front of it: a query outside a crossing's band compares coordinates; one
// inside it takes the orientation of the query against the triangle (float32
// filter on edge vectors, then float64 and exact).
#define GWN_LINE_MAX 24
#define GWN_LINE_REC (1 + 3 * GWN_LINE_MAX)   // ints per line record
__global__ void __launch_bounds__(128) traverse_lines_kernel(const BvhNode *__restrict__ nodes,
                                                             const float4 *__restrict__ tris, int root, Frame fr,
                                                             TravParams tp, QuerySrc q, int k,
                                                             int32_t *__restrict__ lines, unsigned long long *cnt,
                                                             int *status) {
    const int ia = k == 0 ? 1 : 0, ib = k == 2 ? 1 : 2;           // the other two axes
    const int64_t na = q.dims[ia], nb = q.dims[ib], nk = q.dims[k];
    const int64_t line = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= na * nb) return;
    const int64_t stride[3] = {1, q.dims[0], q.dims[0] * q.dims[1]};
    const int64_t base = (line % na) * stride[ia] + (line / na) * stride[ib];
    const float3 D = make_float3(fr.d[0], fr.d[1], fr.d[2]);
    const int64_t m_first = comp(D, k) > 0.f ? 0 : nk - 1;      // farthest back along d
    const float3 p = query_point3(q, base + m_first * stride[k]);
    float p1 = fmaf(p.z, fr.e1[2], fmaf(p.y, fr.e1[1], p.x * fr.e1[0]));
    float p2 = fmaf(p.z, fr.e2[2], fmaf(p.y, fr.e2[1], p.x * fr.e2[0]));
    float p3 = fmaf(p.z, fr.dh[2], fmaf(p.y, fr.dh[1], p.x * fr.dh[0]));
    float pad = fmaf(tp.pad_rel, fabsf(p.x) + fabsf(p.y) + fabsf(p.z), tp.pad_abs);
    float xlo = p1 - pad, xhi = p1 + pad, ylo = p2 - pad, yhi = p2 + pad, zlo = p3 - pad;
    int32_t *out = lines + line * GWN_LINE_REC;
    int n = 0, ntests = 0;
    bool overflow = false, bad = false;
    int stack[GWN_STACK];
    int sp = 0, node = root;
    for (int64_t iter = 0;; iter++) {
        if (iter > tp.max_iter) {
            atomicOr(status, ST_TIMEOUT);
            if (cnt) atomicAdd(&cnt[CNT_TIMEOUT], 1ull);
            bad = true;
            break;
        }
        if (node >= tp.n_internal || ~node >= tp.n_leaves) {
            atomicOr(status, ST_BAD_INPUT);
            bad = true;
            break;
        }
        if (node < 0) {
            const int t = ~node;
            float4 a4 = __ldg(&tris[3 * t]), b4 = __ldg(&tris[3 * t + 1]), c4 = __ldg(&tris[3 * t + 2]);
            const float3 V[3] = {make_float3(a4.x, a4.y, a4.z), make_float3(b4.x, b4.y, b4.z),
                                 make_float3(c4.x, c4.y, c4.z)};
            ntests++;
            int sg[3];                                  // the line's three edge signs, exact
#pragma unroll
            for (int e = 0; e < 3; e++) {
                float3 A = V[e], B = V[(e + 1) % 3];
                float3 a = make_float3(A.x - p.x, A.y - p.y, A.z - p.z);
                float3 E = make_float3(B.x - A.x, B.y - A.y, B.z - A.z);
                sg[e] = edge_sign_f32(a, E, D);
                if (sg[e] == 0) sg[e] = det_abd_sign_f64(A, B, p, D, cnt, status);
            }
            const bool differ = sg[0] * sg[1] < 0 || sg[1] * sg[2] < 0 || sg[0] * sg[2] < 0;
            if (!differ) {
                int code = (sg[0] == 0 || sg[1] == 0 || sg[2] == 0) ? 2 : (sg[0] > 0 ? 0 : 1);
                float cT = 0.f, band = 0.f;
                if (code != 2) {
                    // plane of the triangle met by the line: c_T = p_k - nrm.(p - v0) / nrm_k, in float64
                    // (differences and products of float32 values are exact there); the band covers that
                    // rounding by a wide margin plus the rounding of c_T to float32
                    double e1[3] = {(double)V[1].x - V[0].x, (double)V[1].y - V[0].y, (double)V[1].z - V[0].z};
                    double e2[3] = {(double)V[2].x - V[0].x, (double)V[2].y - V[0].y, (double)V[2].z - V[0].z};
                    double nr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                                    e1[0] * e2[1] - e1[1] * e2[0]};
                    double w[3] = {(double)p.x - V[0].x, (double)p.y - V[0].y, (double)p.z - V[0].z};
                    double nk = nr[k];
                    double num = nr[0] * w[0] + nr[1] * w[1] + nr[2] * w[2];
                    double ct = (double)comp(p, k) - num / nk;
                    double scale = (fabs(nr[0] * w[0]) + fabs(nr[1] * w[1]) + fabs(nr[2] * w[2])) / fabs(nk);
                    cT = (float)ct;
                    band = (float)(1e-6 * (fabs(ct) + scale) + 1e-30);
                    if (!(fabs(nk) > 0.0) || !isfinite(ct)) band = INFINITY;   // no usable coordinate: exact test
                }
                if (n < GWN_LINE_MAX) {
                    out[1 + 3 * n] = __float_as_int(cT);
                    out[2 + 3 * n] = __float_as_int(band);
                    out[3 + 3 * n] = (t << 2) | code;
                    n++;
                } else {
                    overflow = true;
                }
            }
            if (sp == 0) break;
            node = stack[--sp];
            continue;
        }
        const BvhNode nd = nodes[node];
        bool h0 = box_hit(nd.lo.x, nd.lo.y, nd.lo.z, nd.lo.w, nd.z.x, xlo, xhi, ylo, yhi, zlo);
        bool h1 = box_hit(nd.hi.x, nd.hi.y, nd.hi.z, nd.hi.w, nd.z.y, xlo, xhi, ylo, yhi, zlo);
        int c0 = __float_as_int(nd.z.z), c1 = __float_as_int(nd.z.w);
        if (h0 && h1) {
            if (sp >= GWN_STACK) {
                atomicOr(status, ST_STACK_OVERFLOW);
                if (cnt) atomicAdd(&cnt[CNT_STACK_OVERFLOW], 1ull);
                bad = true;
                break;
            }
            stack[sp++] = c1;
            node = c0;
        } else if (h0) {
            node = c0;
        } else if (h1) {
            node = c1;
        } else {
            if (sp == 0) break;
            node = stack[--sp];
        }
    }
    out[0] = bad ? -2 : (overflow ? -1 : n);
    if (cnt) atomicAdd(&cnt[CNT_TRI_TESTS], (unsigned long long)ntests);
}

__global__ void __launch_bounds__(256) lines_count_kernel(const float4 *__restrict__ tris, Frame fr, QuerySrc q,
                                                          int k, const int32_t *__restrict__ lines,
                                                          int32_t *__restrict__ chi, int32_t *defer,
                                                          int32_t *defer_count, int2 *pairs, int32_t *pair_count,
                                                          unsigned long long *cnt, int *status) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= q.n) return;
    const int ia = k == 0 ? 1 : 0, ib = k == 2 ? 1 : 2;
    // grid coordinates in 32-bit arithmetic (q.n < 2^31)
    const unsigned nx = (unsigned)q.dims[0], ny = (unsigned)q.dims[1], ui = (unsigned)idx;
    const unsigned t = ui / nx;
    const unsigned c[3] = {ui - t * nx, t % ny, t / ny};
    const int64_t line = (int64_t)c[ia] + q.dims[ia] * (int64_t)c[ib];
    const int32_t *L = lines + line * GWN_LINE_REC;
    const int n = L[0];
    if (n == -2) { chi[idx] = INT32_MIN; return; }
    if (n < 0) { defer_query(defer, defer_count, idx); return; }
    const float3 pm = query_point3(q, idx);
    const float cm = comp(pm, k);
    const bool fwd = fr.d[k] > 0.f;
    int acc = 0;
    bool whole = false;
    for (int j = 0; j < n; j++) {
        const int e = L[3 + 3 * j], t = e >> 2, code = e & 3;
        if (code == 2) { defer_pair(pairs, pair_count, idx, t, whole); continue; }
        const int s0 = code == 0 ? 1 : -1;
        const float cT = __int_as_float(L[1 + 3 * j]), band = __int_as_float(L[2 + 3 * j]);
        // ahead of the query along d: counted; behind: not; inside the band: orientation
        if (fwd ? cm < cT - band : cm > cT + band) { acc += s0; continue; }
        if (fwd ? cm > cT + band : cm < cT - band) continue;
        float4 a4 = __ldg(&tris[3 * t]), b4 = __ldg(&tris[3 * t + 1]), c4 = __ldg(&tris[3 * t + 2]);
        float3 v0 = make_float3(a4.x, a4.y, a4.z), v1 = make_float3(b4.x, b4.y, b4.z);
        float3 v2 = make_float3(c4.x, c4.y, c4.z);
        float3 a = make_float3(v0.x - pm.x, v0.y - pm.y, v0.z - pm.z);
        float3 e0 = make_float3(v1.x - v0.x, v1.y - v0.y, v1.z - v0.z);
        float3 e2 = make_float3(v0.x - v2.x, v0.y - v2.y, v0.z - v2.z);
        int o = -det3_sign_f32(a, e0, e2);                   // orientation det[v0-p, v1-p, v2-p]
        if (o == 0) o = orient_sign_f64(v0, v1, v2, pm, cnt, status);
        if (o == s0) acc += s0;
    }
    if (whole) defer_query(defer, defer_count, idx);
    else chi[idx] = acc;
}

// Root is a single leaf (one triangle) or the mesh is empty.
__global__ void traverse_single_kernel(const float4 *__restrict__ tris, int ntri, Frame fr, QuerySrc q,
                                       int32_t *__restrict__ chi, unsigned long long *cnt, int *status) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= q.n) return;
    int acc = 0;
    if (ntri == 1) {
        float3 p = query_point3(q, idx);
        float3 D = make_float3(fr.d[0], fr.d[1], fr.d[2]);
        float4 a = tris[0], b = tris[1], c = tris[2];
        acc = tri_crossing(make_float3(a.x, a.y, a.z), make_float3(b.x, b.y, b.z), make_float3(c.x, c.y, c.z),
                           p, D, cnt, status);
    }
    chi[idx] = acc;
}

// grid axis parallel to d (d has exactly one nonzero component), or -1
static int grid_axis_of(const Frame &fr) {
    int axis = -1, nzero = 0;
    for (int c = 0; c < 3; c++) {
        if (fr.d[c] == 0.f) nzero++;
        else axis = c;
    }
    return nzero == 2 ? axis : -1;
}

size_t traverse_lines_bytes(const MeshBvh &b, const QuerySrc &q) {
    if (q.kind != GWN_QUERY_GRID || b.n <= 1) return 0;
    int axis = grid_axis_of(b.frame);
    if (axis < 0 || q.dims[axis] < 2) return 0;
    return sizeof(int32_t) * GWN_LINE_REC * (size_t)(q.n / q.dims[axis]);
}

TravParams trav_params(const MeshBvh &b) {
    // frame non-orthogonality: |d_hat . e_i| for the rounded frame, times the
    // largest distance a crossing can lie from the query along the ray
    const Frame &fr = b.frame;
    double dn = sqrt((double)fr.d[0] * fr.d[0] + (double)fr.d[1] * fr.d[1] + (double)fr.d[2] * fr.d[2]);
    double c1 = fabs((fr.d[0] * (double)fr.e1[0] + fr.d[1] * (double)fr.e1[1] + fr.d[2] * (double)fr.e1[2]) / dn);
    double c2 = fabs((fr.d[0] * (double)fr.e2[0] + fr.d[1] * (double)fr.e2[1] + fr.d[2] * (double)fr.e2[2]) / dn);
    double perp = (c1 > c2 ? c1 : c2) * 1.01 + 1e-12;
    TravParams tp;
    // |p.e - fl(p.e)| <= 3u |p|_1 for unit-norm float32 frame rows; a crossing
    // at distance t|d| <= |p|_2 + R along the ray (R = largest vertex norm)
    // shifts its projection by at most perp * t|d|.
    tp.pad_rel = (float)(4e-7 + 2.0 * perp);
    tp.pad_abs = (float)(2.0 * perp * (double)b.scene_radius + 1e-30);
    tp.max_iter = 8 * b.n + 64;
    tp.n_internal = (int)(b.n - 1);
    tp.n_leaves = (int)b.n;
    return tp;
}

cudaError_t launch_traverse(const MeshBvh &b, const QuerySrc &q, int32_t *chi, int32_t *defer,
                            int32_t *defer_count, int2 *pairs, int32_t *pair_count, int32_t *lines,
                            unsigned long long *cnt, int *status, int sm_count, cudaStream_t st, bool use_bins) {
    if (q.n == 0) return cudaSuccess;
    if (q.n > 0x7fffffff) return cudaErrorInvalidValue;
    const int threads = 128;
    int64_t blocks = (q.n + threads - 1) / threads;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    if (b.n <= 1) {
        traverse_single_kernel<<<(unsigned)blocks, threads, 0, st>>>(b.tris, (int)b.n, b.frame, q, chi, cnt,
                                                                      status);
        return cudaGetLastError();
    }
    const Frame &fr = b.frame;
    const TravParams tp = trav_params(b);
    int64_t tblocks = q.kind == GWN_QUERY_GRID ? grid_tile_blocks(q) : (q.n + 255) / 256;
    if (tblocks > 0x7fffffff) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(defer_count, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(pair_count, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    // d parallel to a grid axis: one traversal per grid line along it
    const int axis = grid_axis_of(fr);
    // Grid queries come in spatially coherent warp tiles: one warp-uniform
    // stack per tile.  Scattered points take one stack per thread.
    if (lines && traverse_lines_bytes(b, q) > 0) {
        int64_t nlines = q.n / q.dims[axis];
        traverse_lines_kernel<<<(unsigned)((nlines + 127) / 128), 128, 0, st>>>(b.nodes, b.tris, b.root, b.frame,
                                                                                 tp, q, axis, lines, cnt, status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        lines_count_kernel<<<(unsigned)((q.n + 255) / 256), 256, 0, st>>>(b.tris, b.frame, q, axis, lines, chi,
                                                                           defer, defer_count, pairs, pair_count,
                                                                           cnt, status);
    } else if (use_bins && b.n_bin_entries > 0 && b.n < (int64_t(1) << 26)) {
        if (q.kind == GWN_QUERY_GRID)
            chi_bins_kernel<true><<<(unsigned)tblocks, 256, 0, st>>>(b.bin_start, b.bin_zt, b.bin_box, b.bins, b.tris,
                                                                     b.frame, tp, q, chi, defer, defer_count, pairs,
                                                                     pair_count, cnt);
        else
            chi_bins_kernel<false><<<(unsigned)tblocks, 256, 0, st>>>(b.bin_start, b.bin_zt, b.bin_box, b.bins,
                                                                      b.tris, b.frame, tp, q, chi, defer, defer_count,
                                                                      pairs, pair_count, cnt);
    } else if (q.kind == GWN_QUERY_GRID && b.tbox && b.n < (int64_t(1) << 26))
        traverse_packet_kernel<<<(unsigned)tblocks, 256, 0, st>>>(b.nodes, b.tris, b.tbox, b.root, b.frame, tp, q,
                                                                  chi, defer, defer_count, pairs, pair_count, cnt,
                                                                  status);
    else
        traverse_kernel<<<(unsigned)tblocks, 256, 0, st>>>(b.nodes, b.tris, b.root, b.frame, tp, q, chi, defer,
                                                           defer_count, pairs, pair_count, cnt, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // settle the unsettled pairs (adds to chi), then recount the queries whose
    // pairs did not fit in the list (overwrites chi): in this order
    int cblocks = (sm_count > 0 ? sm_count : 152) * 4;
    traverse_pairs_kernel<<<cblocks, 128, 0, st>>>(b.tris, b.frame, q, chi, pairs, pair_count, cnt, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    traverse_careful_kernel<<<cblocks, 128, 0, st>>>(b.nodes, b.tris, b.root, b.frame, tp, q, chi, defer,
                                                     defer_count, cnt, status);
    return cudaGetLastError();
}

}  // namespace gwn
