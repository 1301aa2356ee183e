// backward.cu -- gradient of w with respect to the query points and the mesh
// vertices.  chi_d is piecewise constant, so dw = dB_d: only the boundary term
// contributes, and its derivative does not depend on d.
//
// Moving the boundary by delta x changes the solid angle by the flux of the
// swept strip; for a straight edge r(s) = a + s E (a = A - p, b = B - p,
// E = B - A, s in [0, 1]) with linearly interpolated motion this gives
//     dOmega/dA = -(a x E) J_A,   dOmega/dB = -(a x E) J_B,
//     dOmega/dp =  (a x E) (J_A + J_B)   (= -(dOmega/dA + dOmega/dB))
// with J_A = int_0^1 (1 - s) |r|^-3 ds and J_B = int_0^1 s |r|^-3 ds.  Their
// closed forms share one denominator Q = |a||b| + a.b:
//     J_A = 1 / (|a| Q),   J_B = 1 / (|b| Q),
// (from the antiderivatives (L s + c)/(D |r|) and -(c s + |a|^2)/(D |r|),
// L = |E|^2, c = a.E, D = |a x E|^2 = (|a||b| - a.b) Q).  Neither form
// subtracts nearly equal terms, so J_A and J_B keep a few ulps of relative
// accuracy at any distance; the earlier difference form of J_B, ((1/|a| -
// 1/|b|) - (a.E) I0) / |E|^2, lost a factor |a|/|E| to cancellation for
// queries far from short edges.  Q itself cancels only when a and b point
// nearly opposite ways (p close to the edge's interior); there it is taken
// as D / (|a||b| - a.b), with D = |a x E|^2 computed from E.
// The p-gradient sum over edges is the Biot-Savart line integral of the
// boundary; it is checked against finite differences and against the
// gradient of the per-triangle solid-angle sum.
//
// Kernels: when both gradients are asked for, (1) grad_pv_partial_kernel
// evaluates every (query, edge) pair once, two edges per thread, and writes
// per-query partial sums per block of 256 edges and per-edge partial sums per
// query chunk; grad_p_reduce_kernel adds the edge blocks in order,
// grad_v_record_kernel the chunks in a fixed order, and grad_v_scatter_kernel
// sums each vertex's records.  For one gradient alone: (2) grad_p_kernel, one
// thread per K queries looping over the boundary records (deterministic per
// query); (3) grad_v_partial_kernel, one thread per boundary record looping
// over a chunk of queries staged in shared memory, then the same record and
// scatter kernels.
#include "gwn_internal.h"
#include "query.cuh"

namespace gwn {

#define GWN_INV_4PI 0.07957747154594767f

struct EdgeGrad {
    float cx, cy, cz, ja, jb;
};

// MUFU reciprocal and reciprocal square root (rcp/rsqrt.approx, ~1-2 ulp):
// the gradient is needed to ~1e-4 relative, and these replace two IEEE
// square roots and several divisions per (query, edge) pair.  Arguments are
// clamped to normal floats.
__device__ __forceinline__ float grcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float grsqrt(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ EdgeGrad edge_grad(float ax, float ay, float az, float bx, float by, float bz,
                                              float ex, float ey, float ez) {
    EdgeGrad g;
    g.cx = ay * ez - az * ey;
    g.cy = az * ex - ax * ez;
    g.cz = ax * ey - ay * ex;
    float del = fmaxf(g.cx * g.cx + g.cy * g.cy + g.cz * g.cz, 1e-37f);
    float ra2 = fmaxf(ax * ax + ay * ay + az * az, 1e-37f);
    float rb2 = fmaxf(bx * bx + by * by + bz * bz, 1e-37f);
    float ia = grsqrt(ra2), ib = grsqrt(rb2);
    float lab = (ra2 * ia) * (rb2 * ib);             // |a||b|
    float ab = ax * bx + ay * by + az * bz;
    float q = ab >= 0.f ? lab + ab : del * grcp(lab - ab);
    float iq = grcp(fmaxf(q, 1e-37f));
    g.ja = ia * iq;
    g.jb = ib * iq;
    return g;
}

template <int K>
__global__ void __launch_bounds__(256) grad_p_kernel(const float4 *__restrict__ bseq, int nb, QuerySrc q,
                                                     const float *__restrict__ grad_w, float *__restrict__ grad_p) {
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * K + threadIdx.x;
    float px[K], py[K], pz[K], gx[K], gy[K], gz[K];
#pragma unroll
    for (int j = 0; j < K; j++) {
        int64_t idx = base + (int64_t)j * blockDim.x;
        float3 p = idx < q.n ? query_point3(q, idx) : make_float3(0.f, 0.f, 0.f);
        px[j] = p.x; py[j] = p.y; pz[j] = p.z;
        gx[j] = gy[j] = gz[j] = 0.f;
    }
    for (int k = 1; k < nb; k++) {
        float4 A = __ldg(&bseq[k - 1]), B = __ldg(&bseq[k]);
        if (B.w == 0.f) continue;
        float ex = B.x - A.x, ey = B.y - A.y, ez = B.z - A.z;
#pragma unroll
        for (int j = 0; j < K; j++) {
            EdgeGrad g = edge_grad(A.x - px[j], A.y - py[j], A.z - pz[j], B.x - px[j], B.y - py[j], B.z - pz[j],
                                   ex, ey, ez);
            float w = (g.ja + g.jb) * B.w;
            gx[j] = fmaf(g.cx, w, gx[j]);
            gy[j] = fmaf(g.cy, w, gy[j]);
            gz[j] = fmaf(g.cz, w, gz[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < K; j++) {
        int64_t idx = base + (int64_t)j * blockDim.x;
        if (idx < q.n) {
            float s = grad_w[idx] * GWN_INV_4PI;
            grad_p[3 * idx] = gx[j] * s;
            grad_p[3 * idx + 1] = gy[j] * s;
            grad_p[3 * idx + 2] = gz[j] * s;
        }
    }
}

constexpr int GV_THREADS = 128;
constexpr int GV_QTILE = 256;

// partial[(chunk * nb + k) * 8 + {0..2}] = sum over the chunk of dw/dA of the
// edge ending at record k, {4..6} = dw/dB ({3} and {7} pad each half to a
// float4).  Rows are written only for records that end an edge.
__global__ void __launch_bounds__(GV_THREADS) grad_v_partial_kernel(const float4 *__restrict__ bseq, int nb,
                                                                    QuerySrc q, const float *__restrict__ grad_w,
                                                                    int64_t chunk_len, float *__restrict__ partial) {
    __shared__ float4 qs[GV_QTILE];
    int k = blockIdx.x * GV_THREADS + threadIdx.x;
    int chunk = blockIdx.y;
    int64_t q0 = (int64_t)chunk * chunk_len;
    int64_t q1 = q0 + chunk_len < q.n ? q0 + chunk_len : q.n;
    bool active = k >= 1 && k < nb;
    float4 A = active ? bseq[k - 1] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 B = active ? bseq[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    active = active && B.w != 0.f;
    float ex = B.x - A.x, ey = B.y - A.y, ez = B.z - A.z;
    float sA[3] = {0.f, 0.f, 0.f}, sB[3] = {0.f, 0.f, 0.f};
    for (int64_t t0 = q0; t0 < q1; t0 += GV_QTILE) {
        __syncthreads();
        for (int i = threadIdx.x; i < GV_QTILE; i += GV_THREADS) {
            int64_t qi = t0 + i;
            if (qi < q1) {
                float3 p = query_point3(q, qi);
                qs[i] = make_float4(p.x, p.y, p.z, grad_w[qi] * GWN_INV_4PI);
            } else {
                qs[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        __syncthreads();
        if (active) {
            int cnt = (int)(q1 - t0 < GV_QTILE ? q1 - t0 : GV_QTILE);
            for (int i = 0; i < cnt; i++) {
                float4 p = qs[i];
                EdgeGrad g = edge_grad(A.x - p.x, A.y - p.y, A.z - p.z, B.x - p.x, B.y - p.y, B.z - p.z, ex, ey, ez);
                float wa = -g.ja * p.w, wb = -g.jb * p.w;
                sA[0] = fmaf(g.cx, wa, sA[0]); sA[1] = fmaf(g.cy, wa, sA[1]); sA[2] = fmaf(g.cz, wa, sA[2]);
                sB[0] = fmaf(g.cx, wb, sB[0]); sB[1] = fmaf(g.cy, wb, sB[1]); sB[2] = fmaf(g.cz, wb, sB[2]);
            }
        }
    }
    if (k < nb) {
        float4 *o = reinterpret_cast<float4 *>(partial + ((int64_t)chunk * nb + k) * 8);
        o[0] = make_float4(sA[0], sA[1], sA[2], 0.f);
        o[1] = make_float4(sB[0], sB[1], sB[2], 0.f);
    }
}

// Both gradients from one evaluation per (query, edge): the per-edge sums as
// in grad_v_partial_kernel, and per query the sum of its dw/dp contributions
// over the block's edges.
//
// A block holds GPV_EDGES = 256 edges, two per thread (edges t and t + 128 of
// the block) as one packed f32x2 lane pair, so every packed operand of the
// edge geometry is a register pair of two different edges and the query
// enters as a duplicated pair (x, x) read straight from shared memory.  A warp
// takes its 64 edges against the tile's queries 32 at a time: in step s lane l
// evaluates both its edges against query base + (l ^ s), adds the two
// contributions to the three accumulators it holds and hands them to lane
// l ^ s ^ (s + 1), the lane that takes that query in step s + 1, so after 32
// steps lane l holds the sums over the warp's edges of query base + (l ^ 31)
// (3 shuffles per 2 pairs, a fixed order).  The warps are added in order in
// shared memory, one value per (edge block, query, component) goes to
// partial_p[(eb * 3 + c) * nq + q], and grad_p_reduce_kernel sums the edge
// blocks in order.
//
// Per (query, edge), with a = A - p, b = B - p: c = a x E, the clamped squares
// |a|^2, |b|^2 (a tiny constant added, so a query on a vertex gives finite
// weights), 1/|a|, 1/|b| by MUFU rsqrt, and 1/Q by one MUFU reciprocal.  When
// a.b >= 0 for every pair of the warp's step (the query outside the sphere on
// each edge as diameter: nearly always), 1/Q = (1/|a||b|) / (1 + a.b/|a||b|),
// with no cancellation; otherwise the whole warp takes 1/Q = num / den with
// (num, den) = (1, |a||b| + a.b) when a.b >= 0 and (|a||b| - a.b, |c|^2 + tiny)
// when a.b < 0.  The per-edge sums collect c J_A g and c J_B g
// (g = dL/dw / 4 pi) and are negated once at the end.  A block whose
// edge slots are not all valid takes the instantiation that zeroes the
// invalid slots' query contributions by a select; their edge sums are not
// written.  Queries past the tile's end sit far from the geometry with weight
// zero.
constexpr int GPV_EDGES = 2 * GV_THREADS;

typedef float2 f2;
__device__ __forceinline__ f2 mk2(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }

struct EdgePair {
    f2 ax, ay, az, bx, by, bz;          // A and B of the two edges
    f2 ex, ey, ez, nex, ney, nez;       // E = B - A and -E
};

template <bool MASK>
__device__ __forceinline__ void gpv_group(const float4 *__restrict__ qxy, const float4 *__restrict__ qzw, int lb,
                                          const EdgePair &G, bool m0, bool m1, f2 (&sA)[3], f2 (&sB)[3],
                                          float (&acc)[3]) {
    const unsigned FULL = 0xffffffffu;
    const f2 TINY = mk2(1e-37f), MONE = mk2(-1.f), ONE = mk2(1.f);
    for (int o = 0; o < 32; o += 16) {
        const int lo = lb ^ o;
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const int j = lo ^ i;
            const float4 u = qxy[j], v = qzw[j];
            const f2 px = make_float2(u.x, u.y), py = make_float2(u.z, u.w), pz = make_float2(v.x, v.y);
            const f2 pw = make_float2(v.z, v.w);
            // the tile holds -p
            const f2 ax = add2(G.ax, px), ay = add2(G.ay, py), az = add2(G.az, pz);
            const f2 bx = add2(G.bx, px), by = add2(G.by, py), bz = add2(G.bz, pz);
            const f2 cx = fma2(ay, G.ez, mul2(az, G.ney));
            const f2 cy = fma2(az, G.ex, mul2(ax, G.nez));
            const f2 cz = fma2(ax, G.ey, mul2(ay, G.nex));
            const f2 ra2 = fma2(ax, ax, fma2(ay, ay, fma2(az, az, TINY)));
            const f2 rb2 = fma2(bx, bx, fma2(by, by, fma2(bz, bz, TINY)));
            const f2 ab = fma2(ax, bx, fma2(ay, by, mul2(az, bz)));
            const f2 ia = make_float2(grsqrt(ra2.x), grsqrt(ra2.y)), ib = make_float2(grsqrt(rb2.x), grsqrt(rb2.y));
            f2 s;
            if (__any_sync(FULL, ab.x < 0.f || ab.y < 0.f)) {
                const f2 lab = mul2(mul2(ra2, ia), mul2(rb2, ib));
                const f2 del = fma2(cx, cx, fma2(cy, cy, fma2(cz, cz, TINY)));
                const f2 qp = add2(lab, ab), qm = fma2(ab, MONE, lab);
                const f2 num = make_float2(ab.x >= 0.f ? 1.f : qm.x, ab.y >= 0.f ? 1.f : qm.y);
                const f2 den = make_float2(ab.x >= 0.f ? qp.x : del.x, ab.y >= 0.f ? qp.y : del.y);
                s = mul2(mul2(num, make_float2(grcp(den.x), grcp(den.y))), pw);
            } else {
                // 1/Q = (1/|a||b|) / (1 + a.b / |a||b|), no cancellation for a.b >= 0
                const f2 iab = mul2(ia, ib), t = fma2(ab, iab, ONE);
                s = mul2(mul2(iab, make_float2(grcp(t.x), grcp(t.y))), pw);
            }
            const f2 ta = mul2(ia, s), tb = mul2(ib, s);
            f2 tp = add2(ta, tb);
            if (MASK) tp = make_float2(m0 ? tp.x : 0.f, m1 ? tp.y : 0.f);
            sA[0] = fma2(cx, ta, sA[0]); sA[1] = fma2(cy, ta, sA[1]); sA[2] = fma2(cz, ta, sA[2]);
            sB[0] = fma2(cx, tb, sB[0]); sB[1] = fma2(cy, tb, sB[1]); sB[2] = fma2(cz, tb, sB[2]);
            acc[0] = fmaf(cx.y, tp.y, fmaf(cx.x, tp.x, acc[0]));
            acc[1] = fmaf(cy.y, tp.y, fmaf(cy.x, tp.x, acc[1]));
            acc[2] = fmaf(cz.y, tp.y, fmaf(cz.x, tp.x, acc[2]));
            // the query of this lane in step s + 1 is the one lane l ^ s ^ (s + 1) took now
            if (o + i < 31) {
                const int m = (o + i) ^ (o + i + 1);
                acc[0] = __shfl_xor_sync(FULL, acc[0], m);
                acc[1] = __shfl_xor_sync(FULL, acc[1], m);
                acc[2] = __shfl_xor_sync(FULL, acc[2], m);
            }
        }
    }
}

__global__ void __launch_bounds__(GV_THREADS, 7) grad_pv_partial_kernel(const float4 *__restrict__ bseq, int nb,
                                                                        const int32_t *__restrict__ edge_rec,
                                                                        int n_edges, QuerySrc q,
                                                                        const float *__restrict__ grad_w,
                                                                        int64_t chunk_len, float *__restrict__ partial,
                                                                        float *__restrict__ partial_p) {
    __shared__ float4 qs[2][GV_QTILE];                  // (-x, -x, -y, -y), (-z, -z, g, g)
    __shared__ float accp[GV_THREADS / 32][3][GV_QTILE];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the thread's two edges end at records edge_rec[e0] and edge_rec[e1]
    // (the records that start a loop end no edge, so every slot of a full
    // block is valid)
    const int e0 = blockIdx.x * GPV_EDGES + threadIdx.x, e1 = e0 + GV_THREADS;
    const int chunk = blockIdx.y;
    const int64_t q0 = (int64_t)chunk * chunk_len;
    const int64_t q1 = q0 + chunk_len < q.n ? q0 + chunk_len : q.n;
    const int k0 = e0 < n_edges ? __ldg(&edge_rec[e0]) : 0, k1 = e1 < n_edges ? __ldg(&edge_rec[e1]) : 0;
    const float4 Z = make_float4(0.f, 0.f, 0.f, 0.f), X = make_float4(1.f, 0.f, 0.f, 1.f);
    float4 A0 = Z, B0 = X, A1 = Z, B1 = X;            // invalid slots: a unit edge, masked
    bool m0 = k0 >= 1 && k0 < nb, m1 = k1 >= 1 && k1 < nb;
    if (m0) { A0 = bseq[k0 - 1]; B0 = bseq[k0]; m0 = B0.w != 0.f; }
    if (m1) { A1 = bseq[k1 - 1]; B1 = bseq[k1]; m1 = B1.w != 0.f; }
    const bool full = __syncthreads_and(m0 && m1) != 0;
    EdgePair G;
    G.ax = make_float2(A0.x, A1.x); G.ay = make_float2(A0.y, A1.y); G.az = make_float2(A0.z, A1.z);
    G.bx = make_float2(B0.x, B1.x); G.by = make_float2(B0.y, B1.y); G.bz = make_float2(B0.z, B1.z);
    G.ex = make_float2(B0.x - A0.x, B1.x - A1.x); G.ey = make_float2(B0.y - A0.y, B1.y - A1.y);
    G.ez = make_float2(B0.z - A0.z, B1.z - A1.z);
    G.nex = make_float2(-G.ex.x, -G.ex.y); G.ney = make_float2(-G.ey.x, -G.ey.y); G.nez = make_float2(-G.ez.x, -G.ez.y);
    f2 sA[3] = {mk2(0.f), mk2(0.f), mk2(0.f)}, sB[3] = {mk2(0.f), mk2(0.f), mk2(0.f)};
    for (int64_t t0 = q0; t0 < q1; t0 += GV_QTILE) {
        __syncthreads();
        for (int i = threadIdx.x; i < GV_QTILE; i += GV_THREADS) {
            const int64_t qi = t0 + i;
            float3 p = make_float3(1e6f, 1e6f, 1e6f);     // far from the geometry, weight zero
            float g = 0.f;
            if (qi < q1) {
                p = query_point3(q, qi);
                g = grad_w[qi] * GWN_INV_4PI;
            }
            qs[0][i] = make_float4(-p.x, -p.x, -p.y, -p.y);
            qs[1][i] = make_float4(-p.z, -p.z, g, g);
        }
        __syncthreads();
        const int cnt = (int)(q1 - t0 < GV_QTILE ? q1 - t0 : GV_QTILE);
        for (int base = 0; base < cnt; base += 32) {
            float acc[3] = {0.f, 0.f, 0.f};
            if (full)
                gpv_group<false>(qs[0], qs[1], base + lane, G, m0, m1, sA, sB, acc);
            else
                gpv_group<true>(qs[0], qs[1], base + lane, G, m0, m1, sA, sB, acc);
            // after 32 steps lane l holds query base + (l ^ 31)
            accp[warp][0][base + (lane ^ 31)] = acc[0];
            accp[warp][1][base + (lane ^ 31)] = acc[1];
            accp[warp][2][base + (lane ^ 31)] = acc[2];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += GV_THREADS)
            for (int c = 0; c < 3; c++) {
                float v = 0.f;
                for (int w = 0; w < GV_THREADS / 32; w++) v += accp[w][c][i];
                partial_p[((int64_t)blockIdx.x * 3 + c) * q.n + t0 + i] = v;
            }
    }
    if (m0) {
        float4 *o = reinterpret_cast<float4 *>(partial + ((int64_t)chunk * nb + k0) * 8);
        o[0] = make_float4(-sA[0].x, -sA[1].x, -sA[2].x, 0.f);
        o[1] = make_float4(-sB[0].x, -sB[1].x, -sB[2].x, 0.f);
    }
    if (m1) {
        float4 *o = reinterpret_cast<float4 *>(partial + ((int64_t)chunk * nb + k1) * 8);
        o[0] = make_float4(-sA[0].y, -sA[1].y, -sA[2].y, 0.f);
        o[1] = make_float4(-sB[0].y, -sB[1].y, -sB[2].y, 0.f);
    }
}

// grad_p[q] = sum over the edge blocks, in order, of partial_p
__global__ void grad_p_reduce_kernel(const float *__restrict__ partial_p, int n_eb, int64_t nq,
                                     float *__restrict__ grad_p) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    for (int c = 0; c < 3; c++) {
        float v = 0.f;
        for (int eb = 0; eb < n_eb; eb++) v += partial_p[((int64_t)eb * 3 + c) * nq + q];
        grad_p[3 * q + c] = v;
    }
}

// per record: total gradient of its vertex from the edge ending there (as B)
// and the edge starting there (as A of record k+1), summed over the chunks.  A
// block takes 32 consecutive records, one per lane, so that a warp's loads of
// one chunk cover 32 consecutive rows; warp w adds chunks w, w + 32, ... in
// order, and the 32 warp sums are added in order (the order depends on
// n_chunks only).
constexpr int GV_REC_WARPS = 32;
__global__ void __launch_bounds__(GV_REC_WARPS * 32) grad_v_record_kernel(const float *__restrict__ partial,
                                                                          int n_chunks, int nb,
                                                                          const float4 *__restrict__ bseq,
                                                                          float *__restrict__ rec_grad) {
    __shared__ float red[GV_REC_WARPS][3][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = blockIdx.x * 32 + lane;
    const bool asB = k < nb && bseq[k].w != 0.f;
    const bool asA = k + 1 < nb && bseq[k + 1].w != 0.f;
    float g[3] = {0.f, 0.f, 0.f};
    for (int c = warp; c < n_chunks; c += GV_REC_WARPS) {
        const float4 *pk = reinterpret_cast<const float4 *>(partial + ((int64_t)c * nb + k) * 8);
        if (asB) { const float4 b = pk[1]; g[0] += b.x; g[1] += b.y; g[2] += b.z; }
        if (asA) { const float4 a = pk[2]; g[0] += a.x; g[1] += a.y; g[2] += a.z; }   // record k + 1, its A part
    }
    for (int i = 0; i < 3; i++) red[warp][i][lane] = g[i];
    __syncthreads();
    if (warp == 0 && k < nb) {
        for (int i = 0; i < 3; i++) {
            float v = 0.f;
            for (int w = 0; w < GV_REC_WARPS; w++) v += red[w][i][lane];
            rec_grad[3 * k + i] = v;
        }
    }
}

// per boundary vertex: sum its records in list order
__global__ void grad_v_scatter_kernel(const float *__restrict__ rec_grad, const int32_t *__restrict__ bvert,
                                      const int64_t *__restrict__ rec_off, const int32_t *__restrict__ recs,
                                      int64_t n_bvert, float *__restrict__ grad_V) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_bvert) return;
    float g[3] = {0.f, 0.f, 0.f};
    for (int64_t r = rec_off[i]; r < rec_off[i + 1]; r++) {
        int k = recs[r];
        g[0] += rec_grad[3 * k]; g[1] += rec_grad[3 * k + 1]; g[2] += rec_grad[3 * k + 2];
    }
    int64_t v = bvert[i];
    grad_V[3 * v] = g[0];
    grad_V[3 * v + 1] = g[1];
    grad_V[3 * v + 2] = g[2];
}

cudaError_t launch_grad_p(const float4 *bseq, int64_t nb, const QuerySrc &q, const float *grad_w, float *grad_p,
                          cudaStream_t st) {
    if (q.n == 0) return cudaSuccess;
    constexpr int K = 2;
    int64_t blocks = (q.n + 256 * K - 1) / (256 * K);
    grad_p_kernel<K><<<(unsigned)blocks, 256, 0, st>>>(bseq, (int)nb, q, grad_w, grad_p);
    return cudaGetLastError();
}

int grad_v_chunks(int64_t nq, int64_t nb, int sm_count) {
    int64_t eblocks = (nb + GV_THREADS - 1) / GV_THREADS;
    int64_t want = (int64_t)sm_count * 8 / (eblocks > 0 ? eblocks : 1);
    if (want < 1) want = 1;
    int64_t maxc = (nq + GV_QTILE - 1) / GV_QTILE;
    if (want > maxc) want = maxc;
    if (want > 4096) want = 4096;
    return (int)(want > 0 ? want : 1);
}

cudaError_t launch_grad_v(const float4 *bseq, int64_t nb, const QuerySrc &q, const float *grad_w, int n_chunks,
                          float *partial, float *rec_grad, const int32_t *bvert, const int64_t *rec_off,
                          const int32_t *recs, int64_t n_bvert, float *grad_V, cudaStream_t st) {
    if (nb == 0 || n_bvert == 0) return cudaSuccess;
    int64_t chunk_len = (q.n + n_chunks - 1) / n_chunks;
    dim3 grid((unsigned)((nb + GV_THREADS - 1) / GV_THREADS), (unsigned)n_chunks);
    grad_v_partial_kernel<<<grid, GV_THREADS, 0, st>>>(bseq, (int)nb, q, grad_w, chunk_len, partial);
    grad_v_record_kernel<<<(unsigned)((nb + 31) / 32), GV_REC_WARPS * 32, 0, st>>>(partial, n_chunks, (int)nb,
                                                                                   bseq, rec_grad);
    grad_v_scatter_kernel<<<(unsigned)((n_bvert + 255) / 256), 256, 0, st>>>(rec_grad, bvert, rec_off, recs, n_bvert,
                                                                              grad_V);
    return cudaGetLastError();
}

size_t grad_pv_partial_p_bytes(int64_t nq, int64_t n_edges) {
    return sizeof(float) * 3 * (size_t)((n_edges + GPV_EDGES - 1) / GPV_EDGES) * (size_t)nq;
}

// Query chunks for the fused pass: n_eb edge blocks x chunks blocks, sized to
// whole waves of the blocks that fit on the GPU at once (every block does the
// same work), at least GPV_MIN_WAVES waves: with one wave the blocks that the
// warp schedulers favour finish early and the rest of each SM's work runs at
// low occupancy, while each further chunk adds a partial row per record; the
// fewest waves from there that come within 3% of full, at least 256 queries
// per chunk.
constexpr int GPV_MIN_WAVES = 8;
int grad_pv_chunks(int64_t nq, int64_t n_edges, int sm_count) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, grad_pv_partial_kernel, GV_THREADS, 0) != cudaSuccess ||
            b < 1) {
            cudaGetLastError();
            b = 1;
        }
        per_sm = b;
    }
    const int64_t n_eb = (n_edges + GPV_EDGES - 1) / GPV_EDGES;
    const int64_t cap = (int64_t)(sm_count > 0 ? sm_count : 152) * per_sm;
    int64_t maxc = (nq + GV_QTILE - 1) / GV_QTILE;
    if (maxc > 4096) maxc = 4096;
    if (maxc < 1) maxc = 1;
    int64_t best = 1;
    double best_fill = 0.0;
    for (int64_t w = GPV_MIN_WAVES; w <= 4 * GPV_MIN_WAVES; w++) {
        int64_t c = w * cap / (n_eb > 0 ? n_eb : 1);
        if (c < 1) c = 1;
        if (c > maxc) c = maxc;
        int64_t blocks = c * n_eb, waves = (blocks + cap - 1) / cap;
        double fill = (double)blocks / (double)(waves * cap);
        if (fill > best_fill + 1e-9) { best_fill = fill; best = c; }
        if (fill >= 0.97 || c == maxc) break;
    }
    return (int)best;
}

cudaError_t launch_grad_pv(const float4 *bseq, int64_t nb, const int32_t *edge_rec, int64_t n_edges,
                           const QuerySrc &q, const float *grad_w, int n_chunks, float *partial, float *partial_p,
                           float *rec_grad, const int32_t *bvert, const int64_t *rec_off, const int32_t *recs,
                           int64_t n_bvert, float *grad_p, float *grad_V, cudaStream_t st) {
    if (nb == 0 || n_edges == 0 || q.n == 0) return cudaSuccess;
    // whole groups of 32 queries per chunk: only the last chunk has a ragged
    // group (trailing chunks may be empty and write zero partial rows)
    const int64_t chunk_len = ((q.n + n_chunks - 1) / n_chunks + 31) & ~(int64_t)31;
    const int n_eb = (int)((n_edges + GPV_EDGES - 1) / GPV_EDGES);
    dim3 grid((unsigned)n_eb, (unsigned)n_chunks);
    grad_pv_partial_kernel<<<grid, GV_THREADS, 0, st>>>(bseq, (int)nb, edge_rec, (int)n_edges, q, grad_w, chunk_len,
                                                        partial, partial_p);
    grad_p_reduce_kernel<<<(unsigned)((q.n + 255) / 256), 256, 0, st>>>(partial_p, n_eb, q.n, grad_p);
    if (n_bvert > 0) {
        grad_v_record_kernel<<<(unsigned)((nb + 31) / 32), GV_REC_WARPS * 32, 0, st>>>(partial, n_chunks, (int)nb,
                                                                                   bseq, rec_grad);
        grad_v_scatter_kernel<<<(unsigned)((n_bvert + 255) / 256), 256, 0, st>>>(rec_grad, bvert, rec_off, recs,
                                                                                  n_bvert, grad_V);
    }
    return cudaGetLastError();
}

}  // namespace gwn
