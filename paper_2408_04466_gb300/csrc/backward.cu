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
// Kernels: (1) grad_p, one thread per K queries looping over the boundary
// records (deterministic per query); (2) grad_V partials, one thread per
// boundary record looping over a chunk of queries staged in shared memory,
// one partial per (chunk, record); (3) a fixed-order reduction over chunks
// and a scatter to vertices through a per-vertex record list.
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

// edge_grad for two queries at once (packed f32x2 add/mul/fma, MUFU per
// element); the same formulas and clamps
typedef float2 f2;
struct EdgeGrad2 {
    f2 cx, cy, cz, ja, jb;
};
__device__ __forceinline__ f2 mk2(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 mx2(f2 a, float lo) { return make_float2(fmaxf(a.x, lo), fmaxf(a.y, lo)); }
__device__ __forceinline__ EdgeGrad2 edge_grad2(f2 ax, f2 ay, f2 az, f2 bx, f2 by, f2 bz, float ex, float ey,
                                                float ez) {
    EdgeGrad2 g;
    const f2 EX = mk2(ex), EY = mk2(ey), EZ = mk2(ez);
    g.cx = __ffma2_rn(ay, EZ, __fmul2_rn(az, mk2(-ey)));
    g.cy = __ffma2_rn(az, EX, __fmul2_rn(ax, mk2(-ez)));
    g.cz = __ffma2_rn(ax, EY, __fmul2_rn(ay, mk2(-ex)));
    const f2 del = mx2(__ffma2_rn(g.cx, g.cx, __ffma2_rn(g.cy, g.cy, __fmul2_rn(g.cz, g.cz))), 1e-37f);
    const f2 ra2 = mx2(__ffma2_rn(ax, ax, __ffma2_rn(ay, ay, __fmul2_rn(az, az))), 1e-37f);
    const f2 rb2 = mx2(__ffma2_rn(bx, bx, __ffma2_rn(by, by, __fmul2_rn(bz, bz))), 1e-37f);
    const f2 ia = make_float2(grsqrt(ra2.x), grsqrt(ra2.y)), ib = make_float2(grsqrt(rb2.x), grsqrt(rb2.y));
    const f2 lab = __fmul2_rn(__fmul2_rn(ra2, ia), __fmul2_rn(rb2, ib));
    const f2 ab = __ffma2_rn(ax, bx, __ffma2_rn(ay, by, __fmul2_rn(az, bz)));
    const f2 qp = __fadd2_rn(lab, ab), qm = __fadd2_rn(lab, make_float2(-ab.x, -ab.y));
    const float q0 = ab.x >= 0.f ? qp.x : del.x * grcp(qm.x);
    const float q1 = ab.y >= 0.f ? qp.y : del.y * grcp(qm.y);
    const f2 iq = make_float2(grcp(fmaxf(q0, 1e-37f)), grcp(fmaxf(q1, 1e-37f)));
    g.ja = __fmul2_rn(ia, iq);
    g.jb = __fmul2_rn(ib, iq);
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

// partial[(chunk * nb + k) * 6 + {0..2}] = sum over the chunk of dw/dA of the
// edge ending at record k, {3..5} = dw/dB.
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
        float *o = partial + ((int64_t)chunk * nb + k) * 6;
        o[0] = sA[0]; o[1] = sA[1]; o[2] = sA[2];
        o[3] = sB[0]; o[4] = sB[1]; o[5] = sB[2];
    }
}

// Both gradients from one evaluation per (query, edge): the per-edge sums as
// in grad_v_partial_kernel, and per query the sum of its dw/dp contributions
// over the block's edges.  A warp takes its 32 edges against the tile's
// queries 64 at a time, two per lane in packed f32x2 arithmetic: in step s
// lane l evaluates its edge against queries base + (l + s) mod 32 and
// base + 32 + (l + s) mod 32, adds the contributions to the accumulators it
// holds and passes them one lane down, so after 32 steps lane l holds the
// sums over the warp's edges of queries base + l and base + 32 + l (3
// shuffles per pair, a fixed order).  The warps are added in order in shared
// memory, one value per (edge block, query, component) goes to
// partial_p[(eb * 3 + c) * nq + q], and grad_p_reduce_kernel sums the edge
// blocks in order.  Lanes without an edge contribute nothing; queries past
// the tile's end sit far from the geometry with weight zero.
__global__ void __launch_bounds__(GV_THREADS) grad_pv_partial_kernel(const float4 *__restrict__ bseq, int nb,
                                                                     const int32_t *__restrict__ edge_rec,
                                                                     int n_edges, QuerySrc q,
                                                                     const float *__restrict__ grad_w,
                                                                     int64_t chunk_len, float *__restrict__ partial,
                                                                     float *__restrict__ partial_p) {
    __shared__ float4 qs[GV_QTILE];
    __shared__ float accp[GV_THREADS / 32][3][GV_QTILE];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // thread t takes edge t, the edge ending at record edge_rec[t] (the
    // records that start a loop end no edge, so every thread of a full block
    // has one)
    const int t = blockIdx.x * GV_THREADS + threadIdx.x;
    int chunk = blockIdx.y;
    int64_t q0 = (int64_t)chunk * chunk_len;
    int64_t q1 = q0 + chunk_len < q.n ? q0 + chunk_len : q.n;
    const int k = t < n_edges ? __ldg(&edge_rec[t]) : 0;
    bool active = t < n_edges && k >= 1 && k < nb;
    float4 A = active ? bseq[k - 1] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 B = active ? bseq[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    active = active && B.w != 0.f;
    float ex = B.x - A.x, ey = B.y - A.y, ez = B.z - A.z;
    f2 sA2[3] = {mk2(0.f), mk2(0.f), mk2(0.f)}, sB2[3] = {mk2(0.f), mk2(0.f), mk2(0.f)};
    for (int64_t t0 = q0; t0 < q1; t0 += GV_QTILE) {
        __syncthreads();
        for (int i = threadIdx.x; i < GV_QTILE; i += GV_THREADS) {
            int64_t qi = t0 + i;
            if (qi < q1) {
                float3 p = query_point3(q, qi);
                qs[i] = make_float4(p.x, p.y, p.z, grad_w[qi] * GWN_INV_4PI);
            } else {
                qs[i] = make_float4(1e6f, 1e6f, 1e6f, 0.f);      // far from the geometry, weight zero
            }
        }
        __syncthreads();
        const int cnt = (int)(q1 - t0 < GV_QTILE ? q1 - t0 : GV_QTILE);
        // queries base + j and base + 32 + j as one packed pair per step
        for (int base = 0; base < cnt; base += 64) {
            f2 acx = mk2(0.f), acy = mk2(0.f), acz = mk2(0.f);
            for (int st = 0; st < 32; st++) {
                const int j = (lane + st) & 31;
                if (active) {
                    const float4 pa = qs[base + j], pb = qs[base + 32 + j];
                    const f2 pw = make_float2(pa.w, pb.w);
                    EdgeGrad2 g = edge_grad2(make_float2(A.x - pa.x, A.x - pb.x), make_float2(A.y - pa.y, A.y - pb.y),
                                             make_float2(A.z - pa.z, A.z - pb.z), make_float2(B.x - pa.x, B.x - pb.x),
                                             make_float2(B.y - pa.y, B.y - pb.y), make_float2(B.z - pa.z, B.z - pb.z),
                                             ex, ey, ez);
                    const f2 wa = __fmul2_rn(make_float2(-g.ja.x, -g.ja.y), pw);
                    const f2 wb = __fmul2_rn(make_float2(-g.jb.x, -g.jb.y), pw);
                    const f2 wp = __fmul2_rn(__fmul2_rn(__fadd2_rn(g.ja, g.jb), mk2(B.w)), pw);
                    sA2[0] = __ffma2_rn(g.cx, wa, sA2[0]); sA2[1] = __ffma2_rn(g.cy, wa, sA2[1]);
                    sA2[2] = __ffma2_rn(g.cz, wa, sA2[2]);
                    sB2[0] = __ffma2_rn(g.cx, wb, sB2[0]); sB2[1] = __ffma2_rn(g.cy, wb, sB2[1]);
                    sB2[2] = __ffma2_rn(g.cz, wb, sB2[2]);
                    acx = __ffma2_rn(g.cx, wp, acx); acy = __ffma2_rn(g.cy, wp, acy); acz = __ffma2_rn(g.cz, wp, acz);
                }
                // pass the accumulators one lane down
                const int src = (lane + 1) & 31;
                acx = make_float2(__shfl_sync(FULL, acx.x, src), __shfl_sync(FULL, acx.y, src));
                acy = make_float2(__shfl_sync(FULL, acy.x, src), __shfl_sync(FULL, acy.y, src));
                acz = make_float2(__shfl_sync(FULL, acz.x, src), __shfl_sync(FULL, acz.y, src));
            }
            // after 32 steps lane l holds queries base + l and base + 32 + l
            accp[warp][0][base + lane] = acx.x; accp[warp][0][base + 32 + lane] = acx.y;
            accp[warp][1][base + lane] = acy.x; accp[warp][1][base + 32 + lane] = acy.y;
            accp[warp][2][base + lane] = acz.x; accp[warp][2][base + 32 + lane] = acz.y;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += GV_THREADS)
            for (int c = 0; c < 3; c++) {
                float v = 0.f;
                for (int w = 0; w < GV_THREADS / 32; w++) v += accp[w][c][i];
                partial_p[((int64_t)blockIdx.x * 3 + c) * q.n + t0 + i] = v;
            }
    }
    if (active) {
        float *o = partial + ((int64_t)chunk * nb + k) * 6;
        for (int c = 0; c < 3; c++) {
            o[c] = sA2[c].x + sA2[c].y;
            o[3 + c] = sB2[c].x + sB2[c].y;
        }
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
// and the edge starting there (as A of record k+1), summed over chunks in
// chunk order.
__global__ void grad_v_record_kernel(const float *__restrict__ partial, int n_chunks, int nb,
                                     const float4 *__restrict__ bseq, float *__restrict__ rec_grad) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    float g[3] = {0.f, 0.f, 0.f};
    bool asB = bseq[k].w != 0.f;
    bool asA = k + 1 < nb && bseq[k + 1].w != 0.f;
    for (int c = 0; c < n_chunks; c++) {
        const float *pk = partial + ((int64_t)c * nb + k) * 6;
        if (asB) { g[0] += pk[3]; g[1] += pk[4]; g[2] += pk[5]; }
        if (asA) {
            const float *pn = partial + ((int64_t)c * nb + k + 1) * 6;
            g[0] += pn[0]; g[1] += pn[1]; g[2] += pn[2];
        }
    }
    rec_grad[3 * k] = g[0];
    rec_grad[3 * k + 1] = g[1];
    rec_grad[3 * k + 2] = g[2];
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
    grad_v_record_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(partial, n_chunks, (int)nb, bseq, rec_grad);
    grad_v_scatter_kernel<<<(unsigned)((n_bvert + 255) / 256), 256, 0, st>>>(rec_grad, bvert, rec_off, recs, n_bvert,
                                                                              grad_V);
    return cudaGetLastError();
}

size_t grad_pv_partial_p_bytes(int64_t nq, int64_t n_edges) {
    return sizeof(float) * 3 * (size_t)((n_edges + GV_THREADS - 1) / GV_THREADS) * (size_t)nq;
}

// Query chunks for the fused pass: n_eb edge blocks x chunks blocks, sized to
// whole waves of the blocks that fit on the GPU at once (every block of a
// chunk row does the same work), the fewest waves that come within 3% of
// full, at least 256 queries per chunk.
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
    const int64_t n_eb = (n_edges + GV_THREADS - 1) / GV_THREADS;
    const int64_t cap = (int64_t)(sm_count > 0 ? sm_count : 152) * per_sm;
    int64_t maxc = (nq + GV_QTILE - 1) / GV_QTILE;
    if (maxc > 4096) maxc = 4096;
    if (maxc < 1) maxc = 1;
    int64_t best = 1;
    double best_fill = 0.0;
    for (int64_t w = 1; w <= 8; w++) {
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
    int64_t chunk_len = (q.n + n_chunks - 1) / n_chunks;
    const int n_eb = (int)((n_edges + GV_THREADS - 1) / GV_THREADS);
    dim3 grid((unsigned)n_eb, (unsigned)n_chunks);
    grad_pv_partial_kernel<<<grid, GV_THREADS, 0, st>>>(bseq, (int)nb, edge_rec, (int)n_edges, q, grad_w, chunk_len,
                                                        partial, partial_p);
    grad_p_reduce_kernel<<<(unsigned)((q.n + 255) / 256), 256, 0, st>>>(partial_p, n_eb, q.n, grad_p);
    if (n_bvert > 0) {
        grad_v_record_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(partial, n_chunks, (int)nb, bseq, rec_grad);
        grad_v_scatter_kernel<<<(unsigned)((n_bvert + 255) / 256), 256, 0, st>>>(rec_grad, bvert, rec_off, recs,
                                                                                  n_bvert, grad_V);
    }
    return cudaGetLastError();
}

}  // namespace gwn
