// traverse.cuh -- device parts of the crossing count shared by the
// per-geometry kernels (traverse.cu) and the batched mesh launch
// (meshbatch.cu): the ray/box tests, the one-ray traversal of the LBVH, the
// deferral of unsettled pairs and queries, and the 2D-bin crossing search of
// one block of queries.  See traverse.cu for the method.
#pragma once
#include "gwn_internal.h"
#include "predicates.cuh"
#include "query.cuh"

namespace gwn {

#define GWN_STACK 64

struct TravParams {
    float pad_rel;    // relative pad on |p|_1
    float pad_abs;    // absolute pad (frame non-orthogonality x scene radius)
    int64_t max_iter; // iteration limit per query
    int n_internal;   // valid internal refs are [0, n_internal)
    int n_leaves;     // valid leaf refs are ~[0, n_leaves)
};

// padding and limits of a mesh's traversal (host; traverse.cu)
TravParams trav_params(const MeshBvh &b);

__device__ __forceinline__ bool box_hit(float x0, float x1, float y0, float y1, float zm, float xlo, float xhi,
                                        float ylo, float yhi, float zlo) {
    return x0 <= xhi && xlo <= x1 && y0 <= yhi && ylo <= y1 && zm >= zlo;
}

// One ray per thread.  FAST: float32 predicates only, `unsure` set when one
// of them cannot settle a sign; otherwise the full predicates (float64 and
// exact fallbacks).  Returns false on stack overflow, iteration limit or a
// corrupt node reference (status bits set).
// Unsettled pair (query idx, triangle t) of a float32 pass: appended to the
// pair list when it has room (the pair is then settled by
// traverse_pairs_kernel and added to chi), otherwise the whole query is
// deferred.
__device__ __forceinline__ void defer_pair(int2 *pairs, int32_t *pair_count, int64_t idx, int t, bool &unsure) {
    int slot = atomicAdd(pair_count, 1);
    if (slot < GWN_TPAIR_CAP) pairs[slot] = make_int2((int)idx, t);
    else unsure = true;
}

// One ray per thread.  FAST: float32 predicates only; a pair they cannot
// settle goes through defer_pair; otherwise the full predicates (float64 and
// exact fallbacks).  Returns false on stack overflow, iteration limit or a
// corrupt node reference (status bits set).
template <bool FAST>
__device__ __forceinline__ bool traverse_ray(const BvhNode *__restrict__ nodes, const float4 *__restrict__ tris,
                                             int root, const Frame &fr, const TravParams &tp, float3 p, int64_t idx,
                                             int &acc, bool &unsure, int2 *pairs, int32_t *pair_count, int &ntests,
                                             unsigned long long *cnt, int *status) {
    float3 D = make_float3(fr.d[0], fr.d[1], fr.d[2]);
    float p1 = fmaf(p.z, fr.e1[2], fmaf(p.y, fr.e1[1], p.x * fr.e1[0]));
    float p2 = fmaf(p.z, fr.e2[2], fmaf(p.y, fr.e2[1], p.x * fr.e2[0]));
    float p3 = fmaf(p.z, fr.dh[2], fmaf(p.y, fr.dh[1], p.x * fr.dh[0]));
    float pad = fmaf(tp.pad_rel, fabsf(p.x) + fabsf(p.y) + fabsf(p.z), tp.pad_abs);
    float xlo = p1 - pad, xhi = p1 + pad, ylo = p2 - pad, yhi = p2 + pad, zlo = p3 - pad;
    acc = 0;
    int stack[GWN_STACK];
    int sp = 0;
    int node = root;
    int64_t iter = 0;
    while (true) {
        if (++iter > tp.max_iter) {
            atomicOr(status, ST_TIMEOUT);
            if (cnt) atomicAdd(&cnt[CNT_TIMEOUT], 1ull);
            return false;
        }
        if (node >= tp.n_internal || ~node >= tp.n_leaves) {   // corrupt reference: report, never read
            atomicOr(status, ST_BAD_INPUT);
            return false;
        }
        if (node < 0) {
            int t = ~node;
            float4 a = __ldg(&tris[3 * t]), b = __ldg(&tris[3 * t + 1]), c = __ldg(&tris[3 * t + 2]);
            ntests++;
            float3 v0 = make_float3(a.x, a.y, a.z), v1 = make_float3(b.x, b.y, b.z), v2 = make_float3(c.x, c.y, c.z);
            if (FAST) {
                bool u = false;
                acc += tri_crossing_fast(v0, v1, v2, p, D, u);
                if (u) defer_pair(pairs, pair_count, idx, t, unsure);
            } else
                acc += tri_crossing(v0, v1, v2, p, D, cnt, status);
            if (sp == 0) return true;
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
                return false;
            }
            stack[sp++] = c1;
            node = c0;
        } else if (h0) {
            node = c0;
        } else if (h1) {
            node = c1;
        } else {
            if (sp == 0) return true;
            node = stack[--sp];
        }
    }
}

// Append query idx to the deferred list (at most one entry per query, so the
// list never outgrows its q.n entries).
__device__ __forceinline__ void defer_query(int32_t *defer, int32_t *defer_count, int64_t idx) {
    int slot = atomicAdd(defer_count, 1);
    defer[slot] = (int32_t)idx;
}

// The body of chi_bins_kernel for a block of 256 threads: thread i takes query
// idx of q (idx outside [0, q.n): no query, the thread still takes part);
// counts, pairs and deferred queries are written at index gofs + idx.
__device__ __forceinline__ void chi_bins_block(const int32_t *__restrict__ bin_start, const float2 *__restrict__ bin_zt,
                                               const float4 *__restrict__ bin_box, const BinParams &bp,
                                               const float4 *__restrict__ tris, const Frame &fr, const TravParams &tp,
                                               const QuerySrc &q, int64_t idx, int64_t gofs,
                                               int32_t *__restrict__ chi, int32_t *defer, int32_t *defer_count,
                                               int2 *tpairs, int32_t *tpair_count, unsigned long long *cnt) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    bool valid = idx >= 0 && idx < q.n;
    float3 p = valid ? query_point3(q, idx) : make_float3(0.f, 0.f, 0.f);
    float3 D = make_float3(fr.d[0], fr.d[1], fr.d[2]);
    float p1 = fmaf(p.z, fr.e1[2], fmaf(p.y, fr.e1[1], p.x * fr.e1[0]));
    float p2 = fmaf(p.z, fr.e2[2], fmaf(p.y, fr.e2[1], p.x * fr.e2[0]));
    float p3 = fmaf(p.z, fr.dh[2], fmaf(p.y, fr.dh[1], p.x * fr.dh[0]));
    float pad = fmaf(tp.pad_rel, fabsf(p.x) + fabsf(p.y) + fabsf(p.z), tp.pad_abs);
    float xlo = p1 - pad, xhi = p1 + pad, ylo = p2 - pad, yhi = p2 + pad, zlo = p3 - pad;
    __shared__ int s_pair[256 / 32][64];
    __shared__ int s_acc[256 / 32][32];
    __shared__ unsigned s_uns[256 / 32];
    int *pairs = s_pair[w];
    s_acc[w][lane] = 0;
    if (lane == 0) s_uns[w] = 0u;
    __syncwarp();
    auto flush = [&](int n) -> int {            // as in traverse_packet_kernel
        int m = n < 32 ? n : 32;
        int pr = lane < m ? pairs[lane] : -1;
        int ql = pr >= 0 ? (pr & 31) : lane;
        float qx = __shfl_sync(FULL, p.x, ql), qy = __shfl_sync(FULL, p.y, ql), qz = __shfl_sync(FULL, p.z, ql);
        int qi = __shfl_sync(FULL, (int)(gofs + idx), ql);
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
    // the query's bin range; a ray box outside every triangle box has nothing to test
    bool live = valid && xlo <= bp.x1 && xhi >= bp.x0 && ylo <= bp.y1 && yhi >= bp.y0;
    const int qbx0 = bin_of(xlo, bp.x0, bp.invx, bp.nbx), qbx1 = bin_of(xhi, bp.x0, bp.invx, bp.nbx);
    const int qby0 = bin_of(ylo, bp.y0, bp.invy, bp.nby), qby1 = bin_of(yhi, bp.y0, bp.invy, bp.nby);
    const bool multi = qbx0 != qbx1 || qby0 != qby1;
    int bx = qbx0 - 1, by = qby0, i = 0, e = 0;
    auto settle = [&]() {                       // on to the next non-empty bin of the range
        while (live && i >= e) {
            if (++bx > qbx1) {
                bx = qbx0;
                if (++by > qby1) { live = false; break; }
            }
            int b = by * bp.nbx + bx;
            i = __ldg(&bin_start[b]);
            e = __ldg(&bin_start[b + 1]);
        }
    };
    settle();
    int ntests = 0, npairs = 0;                 // npairs: warp-uniform
    while (__any_sync(FULL, live)) {
        bool hit = false;
        int t = 0;
        if (live) {
            float2 zt = __ldg(&bin_zt[i]);
            if (zt.x < zlo) {
                i = e;                          // the rest of this bin lies behind the query
            } else {
                float4 bb = __ldg(&bin_box[i]);
                hit = box_hit(bb.x, bb.y, bb.z, bb.w, zt.x, xlo, xhi, ylo, yhi, zlo);
                if (hit && multi)
                    hit = max(bin_of(bb.x, bp.x0, bp.invx, bp.nbx), qbx0) == bx &&
                          max(bin_of(bb.z, bp.y0, bp.invy, bp.nby), qby0) == by;
                t = __float_as_int(zt.y);
                i++;
            }
            settle();
        }
        unsigned m = __ballot_sync(FULL, hit);
        if (m) {
            if (hit) pairs[npairs + __popc(m & ((1u << lane) - 1u))] = (t << 5) | lane;
            npairs += __popc(m);
            ntests += hit;
            __syncwarp();
            if (npairs >= 32) npairs = flush(npairs);
        }
    }
    while (npairs > 0) npairs = flush(npairs);
    __syncwarp();
    int acc = s_acc[w][lane];
    bool unsure = (s_uns[w] >> lane) & 1u;
    if (valid) {
        if (unsure) defer_query(defer, defer_count, gofs + idx);
        else chi[gofs + idx] = acc;
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


}  // namespace gwn
