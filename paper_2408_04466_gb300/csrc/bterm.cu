// bterm.cu -- boundary term of the one-shot winding number (3D meshes).
//
// Closing the surface M with the half-infinite curtain {x - s d : x in dM,
// s >= 0} yields a closed surface that the ray p + t d never meets through
// the curtain; its winding number is the crossing count chi_d(p) (Eq. chi,
// Lemma 1/2, closure as in the proof of Appendix A).  Hence
//     w(p) = chi_d(p) + B_d(p),
//     B_d(p) = (1/4pi) sum_{boundary edges A->B} Omega(A - p, B - p, n),
// with n = -d/|d| and Omega the signed solid angle of the spherical triangle
// (A-p, B-p, n).  tan(Omega/2) = num/den (Van Oosterom-Strackee); written in
// the orthonormal frame (e1, e2, n) with a = A - p, b = B - p:
//     num = a1 b2 - a2 b1
//     den = s_a s_b + a1 b1 + a2 b2,     s_x = |x| + x_n
// (the stereographic form: den = |a||b| + a.b + a_n|b| + b_n|a| regrouped).
// s_x cancels when x points along -n = d; there s_x = (x1^2 + x2^2)/(|x| - x_n)
// is used instead, so every factor is computed to a few ulps.  Each vertex's
// (a1, a2, s_a) is computed once per query and shared by its two edges.
//
// Where the ray p + t d crosses edge AB, num changes sign with den < 0 and
// Omega jumps by 4pi while chi_d jumps by -1.  Pairs with |Omega/2| within
// 0.01 of pi take the sign of num from the exact perturbed predicate
// -sign det[A-p, B-p, d_eps] (the same predicate the crossing count uses), so
// both jumps happen at exactly the same place.
//
// Layout: bseq holds the boundary loops as float4 records (x, y, z, w) in loop
// order; each loop is v0 (w = 0), v1 .. v_{n-1} (w = 1), v0 again (w = 1).
// w is the weight of the edge from the previous record.  All lanes of a warp
// read the same record (broadcast); every thread carries K queries.
#include <stdlib.h>

#include "gwn_internal.h"
#include "predicates.cuh"
#include "query.cuh"

namespace gwn {

#define GWN_CUT_THRESHOLD 3.1315926f   // pi - 0.01
#define GWN_INV_2PI 0.15915494309189535f

// Take the sign of num from the exact predicate (rare path).
static __device__ __noinline__ float cut_fix(float th, float4 va, float4 vb, float3 p, Frame fr,
                                      unsigned long long *cnt, int *status) {
    float3 A = make_float3(va.x, va.y, va.z), B = make_float3(vb.x, vb.y, vb.z);
    float3 D = make_float3(fr.d[0], fr.d[1], fr.d[2]);
    int s = edge_sign_slow(A, B, p, D, cnt, status);   // sign(num) = -s
    if (cnt) atomicAdd(&cnt[CNT_CUT_SIGN], 1ull);
    if (s > 0) return -fabsf(th);
    if (s < 0) return fabsf(th);
    return th;
}

struct VertexProj {
    float a1, a2, s;
};

__device__ __forceinline__ VertexProj project(float4 v, float px, float py, float pz, const Frame &fr) {
    float ax = v.x - px, ay = v.y - py, az = v.z - pz;
    VertexProj o;
    o.a1 = fmaf(az, fr.e1[2], fmaf(ay, fr.e1[1], ax * fr.e1[0]));
    o.a2 = fmaf(az, fr.e2[2], fmaf(ay, fr.e2[1], ax * fr.e2[0]));
    float an = fmaf(az, fr.n[2], fmaf(ay, fr.n[1], ax * fr.n[0]));
    float rp = fmaf(o.a1, o.a1, o.a2 * o.a2);
    float r2 = fmaxf(fmaf(an, an, rp), 1e-37f);
    float r = r2 * rsqrtf(r2);
    o.s = an >= 0.f ? r + an : __fdividef(rp, r - an);
    return o;
}

template <int K>
__global__ void __launch_bounds__(256) bterm3d_kernel(const float4 *__restrict__ bseq, int nb, Frame fr,
                                                      QuerySrc q, const int32_t *__restrict__ chi,
                                                      float *__restrict__ w_out, float *__restrict__ b_out,
                                                      unsigned long long *cnt, int *status) {
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * K + threadIdx.x;
    float px[K], py[K], pz[K];
    float pa1[K], pa2[K], ps[K], sum[K], cmp[K];
#pragma unroll
    for (int j = 0; j < K; j++) {
        int64_t idx = base + (int64_t)j * blockDim.x;
        float3 p = idx < q.n ? query_point3(q, idx) : make_float3(0.f, 0.f, 0.f);
        px[j] = p.x; py[j] = p.y; pz[j] = p.z;
        sum[j] = 0.f; cmp[j] = 0.f;
    }
    if (nb > 0) {
        float4 v0 = __ldg(&bseq[0]);
#pragma unroll
        for (int j = 0; j < K; j++) {
            VertexProj o = project(v0, px[j], py[j], pz[j], fr);
            pa1[j] = o.a1; pa2[j] = o.a2; ps[j] = o.s;
        }
        float4 vprev = v0;
#pragma unroll 2
        for (int k = 1; k < nb; k++) {
            float4 v = __ldg(&bseq[k]);
#pragma unroll
            for (int j = 0; j < K; j++) {
                VertexProj o = project(v, px[j], py[j], pz[j], fr);
                float num = fmaf(pa1[j], o.a2, -(pa2[j] * o.a1));
                float den = fmaf(ps[j], o.s, fmaf(pa1[j], o.a1, pa2[j] * o.a2));
                float th = atan2f(num, den);
                if (fabsf(th) > GWN_CUT_THRESHOLD && v.w != 0.f)
                    th = cut_fix(th, vprev, v, make_float3(px[j], py[j], pz[j]), fr, cnt, status);
                // compensated (Kahan) accumulation of w * th
                float y = fmaf(th, v.w, -cmp[j]);
                float t = sum[j] + y;
                cmp[j] = (t - sum[j]) - y;
                sum[j] = t;
                pa1[j] = o.a1; pa2[j] = o.a2; ps[j] = o.s;
            }
            vprev = v;
        }
    }
#pragma unroll
    for (int j = 0; j < K; j++) {
        int64_t idx = base + (int64_t)j * blockDim.x;
        if (idx < q.n) {
            float B = (sum[j] - cmp[j]) * GWN_INV_2PI;
            if (b_out) b_out[idx] = B;
            if (w_out) w_out[idx] = B + (chi ? (float)chi[idx] : 0.f);
        }
    }
}

// ---- packed variant: two queries per 64-bit register pair (f32x2) ----------
// Blackwell executes add/sub/mul/fma.rn.f32x2 on two float32 lanes per
// instruction.  Every per-query operation that is a plain add/mul/fma runs
// packed on a pair of queries; min/max, MUFU (rsqrt, reciprocal), compares and
// selects run per element.  atan2 is a degree-8 minimax polynomial of
// atan(t) on [0, 1] (t = min/max of |num|, |den|) with octant fix-ups; the
// coefficients were fitted by Lawson-weighted least squares to the relative
// error of t*P(t^2) ~ atan(t) (max 1.5e-8 in exact arithmetic).
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float lo2(f2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return a;
}
__device__ __forceinline__ float hi2(f2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return b;
}
// MUFU reciprocal (rcp.approx: about 1 ulp); arguments here are normal floats
__device__ __forceinline__ float frcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) { f2 d; asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b)); return d; }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { f2 d; asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b)); return d; }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { f2 d; asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b)); return d; }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

#define GWN_AT_C8 0.00284989f
#define GWN_AT_C7 -0.01606863f
#define GWN_AT_C6 0.04269152f
#define GWN_AT_C5 -0.07504295f
#define GWN_AT_C4 0.10640934f
#define GWN_AT_C3 -0.14203644f
#define GWN_AT_C2 0.19992619f
#define GWN_AT_C1 -0.33333073f
#define GWN_AT_C0 0.99999998f

// per-element octant fix-up of r = atan(min/max) into atan2(y, x)
__device__ __forceinline__ float octant(float r, float y, float x) {
    bool swp = fabsf(y) > fabsf(x), neg = x < 0.f;
    float base = swp ? 1.5707963267948966f : (neg ? 3.14159265358979f : 0.f);
    float sg = (swp != neg) ? -1.f : 1.f;
    return copysignf(fmaf(sg, r, base), y);
}

__device__ __forceinline__ f2 atan2_2(f2 y, f2 x) {
    float y0 = lo2(y), y1 = hi2(y), x0 = lo2(x), x1 = hi2(x);
    float mn0 = fminf(fabsf(y0), fabsf(x0)), mx0 = fmaxf(fmaxf(fabsf(y0), fabsf(x0)), 1e-37f);
    float mn1 = fminf(fabsf(y1), fabsf(x1)), mx1 = fmaxf(fmaxf(fabsf(y1), fabsf(x1)), 1e-37f);
    f2 t = mul2(pk(mn0, mn1), pk(frcp(mx0), frcp(mx1)));
    f2 t2 = mul2(t, t);
    f2 p = fma2(pk(GWN_AT_C8, GWN_AT_C8), t2, pk(GWN_AT_C7, GWN_AT_C7));
    p = fma2(p, t2, pk(GWN_AT_C6, GWN_AT_C6));
    p = fma2(p, t2, pk(GWN_AT_C5, GWN_AT_C5));
    p = fma2(p, t2, pk(GWN_AT_C4, GWN_AT_C4));
    p = fma2(p, t2, pk(GWN_AT_C3, GWN_AT_C3));
    p = fma2(p, t2, pk(GWN_AT_C2, GWN_AT_C2));
    p = fma2(p, t2, pk(GWN_AT_C1, GWN_AT_C1));
    p = fma2(p, t2, pk(GWN_AT_C0, GWN_AT_C0));
    f2 r = mul2(p, t);
    return pk(octant(lo2(r), y0, x0), octant(hi2(r), y1, x1));
}

template <int KP>   // KP query pairs per thread
__global__ void __launch_bounds__(256) bterm3d_x2_kernel(const float4 *__restrict__ bseq, int nb, Frame fr,
                                                         QuerySrc q, const int32_t *__restrict__ chi,
                                                         float *__restrict__ w_out, float *__restrict__ b_out,
                                                         unsigned long long *cnt, int *status) {
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * (2 * KP) + threadIdx.x;
    f2 px[KP], py[KP], pz[KP], pa1[KP], pa2[KP], ps[KP], sum[KP], cmp[KP];
    const f2 e1x = pk(fr.e1[0], fr.e1[0]), e1y = pk(fr.e1[1], fr.e1[1]), e1z = pk(fr.e1[2], fr.e1[2]);
    const f2 e2x = pk(fr.e2[0], fr.e2[0]), e2y = pk(fr.e2[1], fr.e2[1]), e2z = pk(fr.e2[2], fr.e2[2]);
    const f2 nx = pk(fr.n[0], fr.n[0]), ny = pk(fr.n[1], fr.n[1]), nz = pk(fr.n[2], fr.n[2]);
#pragma unroll
    for (int j = 0; j < KP; j++) {
        int64_t i0 = base + (int64_t)(2 * j) * blockDim.x, i1 = i0 + blockDim.x;
        float3 p0 = i0 < q.n ? query_point3(q, i0) : make_float3(0.f, 0.f, 0.f);
        float3 p1 = i1 < q.n ? query_point3(q, i1) : make_float3(0.f, 0.f, 0.f);
        px[j] = pk(p0.x, p1.x); py[j] = pk(p0.y, p1.y); pz[j] = pk(p0.z, p1.z);
        sum[j] = pk(0.f, 0.f); cmp[j] = pk(0.f, 0.f);
    }
    auto project = [&](float4 v, int j, f2 &a1, f2 &a2, f2 &s) {
        f2 ax = sub2(pk(v.x, v.x), px[j]), ay = sub2(pk(v.y, v.y), py[j]), az = sub2(pk(v.z, v.z), pz[j]);
        a1 = fma2(az, e1z, fma2(ay, e1y, mul2(ax, e1x)));
        a2 = fma2(az, e2z, fma2(ay, e2y, mul2(ax, e2x)));
        f2 an = fma2(az, nz, fma2(ay, ny, mul2(ax, nx)));
        f2 rp = fma2(a1, a1, mul2(a2, a2));
        f2 r2 = fma2(an, an, rp);
        float r20 = fmaxf(lo2(r2), 1e-37f), r21 = fmaxf(hi2(r2), 1e-37f);
        f2 r = mul2(pk(r20, r21), pk(rsqrtf(r20), rsqrtf(r21)));
        f2 sp = add2(r, an), dm = sub2(r, an);
        f2 sn = mul2(rp, pk(frcp(lo2(dm)), frcp(hi2(dm))));
        s = pk(lo2(an) >= 0.f ? lo2(sp) : lo2(sn), hi2(an) >= 0.f ? hi2(sp) : hi2(sn));
    };
    if (nb > 0) {
        float4 v0 = __ldg(&bseq[0]);
#pragma unroll
        for (int j = 0; j < KP; j++) project(v0, j, pa1[j], pa2[j], ps[j]);
        float4 vprev = v0;
        for (int k = 1; k < nb; k++) {
            float4 v = __ldg(&bseq[k]);
            const bool edge = v.w != 0.f;     // uniform across the block
#pragma unroll
            for (int j = 0; j < KP; j++) {
                f2 a1, a2, s;
                project(v, j, a1, a2, s);
                if (edge) {
                    f2 num = sub2(mul2(pa1[j], a2), mul2(pa2[j], a1));
                    f2 den = fma2(ps[j], s, fma2(pa1[j], a1, mul2(pa2[j], a2)));
                    f2 th = atan2_2(num, den);
                    float t0 = lo2(th), t1 = hi2(th);
                    if (fabsf(t0) > GWN_CUT_THRESHOLD)
                        t0 = cut_fix(t0, vprev, v, make_float3(lo2(px[j]), lo2(py[j]), lo2(pz[j])), fr, cnt, status);
                    if (fabsf(t1) > GWN_CUT_THRESHOLD)
                        t1 = cut_fix(t1, vprev, v, make_float3(hi2(px[j]), hi2(py[j]), hi2(pz[j])), fr, cnt, status);
                    th = pk(t0, t1);
                    f2 y = sub2(th, cmp[j]);
                    f2 t = add2(sum[j], y);
                    cmp[j] = sub2(sub2(t, sum[j]), y);
                    sum[j] = t;
                }
                pa1[j] = a1; pa2[j] = a2; ps[j] = s;
            }
            vprev = v;
        }
    }
#pragma unroll
    for (int j = 0; j < KP; j++) {
        f2 tot = sub2(sum[j], cmp[j]);
        float Bv[2] = {lo2(tot) * GWN_INV_2PI, hi2(tot) * GWN_INV_2PI};
        for (int h = 0; h < 2; h++) {
            int64_t idx = base + (int64_t)(2 * j + h) * blockDim.x;
            if (idx < q.n) {
                if (b_out) b_out[idx] = Bv[h];
                if (w_out) w_out[idx] = Bv[h] + (chi ? (float)chi[idx] : 0.f);
            }
        }
    }
}

cudaError_t launch_bterm3d(const float4 *bseq, int64_t n_bseq, const Frame &fr, const QuerySrc &q,
                           const int32_t *chi, float *w_out, float *b_out, unsigned long long *cnt,
                           int *status, int sm_count, cudaStream_t st) {
    (void)sm_count;
    if (q.n == 0) return cudaSuccess;
    const int threads = 256;
    static int impl = -1;
    if (impl < 0) {
        const char *e = getenv("GWN_BTERM_IMPL");
        impl = e ? atoi(e) : 0;
    }
    if (impl == 1) {
        constexpr int KP = 2;
        int64_t per_block = (int64_t)threads * 2 * KP;
        int64_t blocks = (q.n + per_block - 1) / per_block;
        if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
        bterm3d_x2_kernel<KP><<<(unsigned)blocks, threads, 0, st>>>(bseq, (int)n_bseq, fr, q, chi, w_out, b_out,
                                                                   cnt, status);
        return cudaGetLastError();
    }
    constexpr int K = 4;
    int64_t per_block = (int64_t)threads * K;
    int64_t blocks = (q.n + per_block - 1) / per_block;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    bterm3d_kernel<K><<<(unsigned)blocks, threads, 0, st>>>(bseq, (int)n_bseq, fr, q, chi, w_out, b_out,
                                                            cnt, status);
    return cudaGetLastError();
}

}  // namespace gwn
