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
// (a1, a2, s_a) is computed once per query and shared by its two edges, so
// the rounding of a vertex's direction cancels to first order between them.
//
// Exact-sign cases (rare, decided by the predicates the crossing count uses):
// * the ray p + t d crosses edge AB: num changes sign with den < 0 and Omega
//   jumps by 4pi while chi_d jumps by -1.  Pairs with |Omega/2| within 0.01 of
//   pi take their branch from -sign det[A-p, B-p, d_eps] (a wrong branch moves
//   by 2pi, the continuous extension of the right one);
// * a boundary vertex within 1e-3 rad of the forward ray: its azimuth around
//   the ray is ill-conditioned in float32, so both incident edges are
//   recomputed in float64 (they are flagged by |num + i den| < 2e-3 |a||b|,
//   which every edge of such a vertex satisfies); a vertex exactly on the ray
//   (decided exactly) is
//   seen by the perturbed ray d_eps in the direction -dp (dp = the first of
//   e_x, e_y, e_z not parallel to d, projected orthogonally to d), and its
//   edges take the limit of Omega under that perturbation.
//
// Arithmetic: two queries per 64-bit register pair; plain add/mul/fma run as
// packed f32x2 instructions (Blackwell), min/max, MUFU (rsqrt, reciprocal),
// compares and selects per element.  atan2(num, den) uses the half-angle
// identity (see half_angle_atan2) so that a single odd polynomial on [-1, 1]
// serves every quadrant: a degree-8 minimax polynomial P with atan(v) ~
// v P(v^2), fitted by Lawson-weighted least squares to the relative error
// (1.5e-8 in exact arithmetic).  Accumulation over edges is compensated
// (Kahan).
//
// Layout: bseq holds the boundary loops as float4 records (x, y, z, w) in loop
// order; each loop is v0 (w = 0), v1 .. v_{n-1} (w = 1), v0 again (w = 1).
// w = 1 marks an edge from the previous record.  All lanes of a warp read the
// same record (broadcast); every thread carries 2*KP queries.
#include <stdlib.h>

#include "gwn_internal.h"
#include "predicates.cuh"
#include "query.cuh"

namespace gwn {

#define GWN_CUT_THRESHOLD 3.1315926f   // pi - 0.01
#define GWN_INV_2PI 0.15915494309189535f

// ---- exact helpers for the slow path ---------------------------------------
// exact sign of ((X-P) x D)_k (products of two float32 values are exact in float64)
static __device__ __noinline__ int exact_cross_xd(float3 X, float3 P, float3 D, int k) {
    int i = (k + 1) % 3, j = (k + 2) % 3;
    Expansion<4> E;
    E.init();
    float xi = comp(X, i), xj = comp(X, j), pi = comp(P, i), pj = comp(P, j), di = comp(D, i), dj = comp(D, j);
    E.add((double)xi * dj); E.add(-(double)pi * dj); E.add(-(double)xj * di); E.add((double)pj * di);
    return E.sign();
}

// X lies exactly on the forward ray from P: (X-P) x D = 0 and (X-P).D > 0
static __device__ __noinline__ bool on_forward_ray(float3 X, float3 P, float3 D) {
    double x[3] = {(double)X.x - P.x, (double)X.y - P.y, (double)X.z - P.z};
    double dd[3] = {D.x, D.y, D.z};
    if (!(x[0] * dd[0] + x[1] * dd[1] + x[2] * dd[2] > 0.0)) return false;
    for (int k = 0; k < 3; k++) {
        int i = (k + 1) % 3, j = (k + 2) % 3;
        double c = x[i] * dd[j] - x[j] * dd[i];
        double bound = GWN_F64_BOUND * (fabs(x[i] * dd[j]) + fabs(x[j] * dd[i]));
        if (fabs(c) > bound) return false;
    }
    for (int k = 0; k < 3; k++)
        if (exact_cross_xd(X, P, D, k) != 0) return false;
    return true;
}

// Branch fix: theta = atan2(num, den) lies on the wrong side of the cut
// (den < 0, num ~ 0) when the rounded num has the wrong sign.  The exact sign
// s of num selects the branch; theta keeps its computed smooth part and moves
// by 2pi, which is the continuous extension of the correct branch (a sign
// flip would not be, and would break the first-order cancellation of vertex
// rounding between adjacent edges).
__device__ __forceinline__ double branch_fix(double th, int s_num) {
    if (s_num < 0 && th > 0.0) return th - 6.283185307179586;
    if (s_num > 0 && th < 0.0) return th + 6.283185307179586;
    return th;
}

// Omega/2 of edge A->B in float64 for flagged pairs (|z| small relative to
// |a||b|: an endpoint near the forward ray, or p near the edge).  Each
// endpoint within 1e-3 rad of the forward ray is recomputed in float64, or,
// when it lies exactly on the ray, replaced by the perturbation limit
// (x_perp = u = -dp in the frame, s_x = 0).  Other endpoints keep their
// float32 projection (fa*, fb*), the values their other edge uses, so the
// first-order cancellation of their rounding between their two edges holds.
// The decision depends only on the vertex and the query, so both edges of a
// vertex make the same one.
static __device__ __noinline__ float slow_theta(float4 va, float4 vb, float fa1, float fa2, float fsa, float fb1,
                                                float fb2, float fsb, float3 p, Frame fr, Frame64 f,
                                                unsigned long long *cnt, int *status) {
    float3 A = make_float3(va.x, va.y, va.z), B = make_float3(vb.x, vb.y, vb.z);
    float3 D = make_float3(fr.d[0], fr.d[1], fr.d[2]);
    double u1 = -(f.dp[0] * f.e1[0] + f.dp[1] * f.e1[1] + f.dp[2] * f.e1[2]);
    double u2 = -(f.dp[0] * f.e2[0] + f.dp[1] * f.e2[1] + f.dp[2] * f.e2[2]);
    double x1[2], x2[2], xs[2];
    bool onray[2] = {false, false};
    const float3 X3[2] = {A, B};
    const float f1[2] = {fa1, fb1}, f2v[2] = {fa2, fb2}, fs[2] = {fsa, fsb};
    for (int e = 0; e < 2; e++) {
        float3 X = X3[e];
        double x[3] = {(double)X.x - p.x, (double)X.y - p.y, (double)X.z - p.z};
        double a1 = x[0] * f.e1[0] + x[1] * f.e1[1] + x[2] * f.e1[2];
        double a2 = x[0] * f.e2[0] + x[1] * f.e2[1] + x[2] * f.e2[2];
        double an = x[0] * f.n[0] + x[1] * f.n[1] + x[2] * f.n[2];
        double rp = a1 * a1 + a2 * a2;
        bool near = an < 0.0 && rp < 1e-6 * (rp + an * an);
        if (!near) {
            x1[e] = f1[e]; x2[e] = f2v[e]; xs[e] = fs[e];
            continue;
        }
        if (on_forward_ray(X, p, D)) {
            onray[e] = true;
            x1[e] = u1; x2[e] = u2; xs[e] = 0.0;
            continue;
        }
        double r = sqrt(rp + an * an);
        x1[e] = a1; x2[e] = a2; xs[e] = rp / (r - an);
    }
    double num, den;
    if (onray[0] && onray[1]) {
        num = 0.0; den = 1.0;                         // edge along the ray: limit 0
    } else {
        num = x1[0] * x2[1] - x2[0] * x1[1];
        den = xs[0] * xs[1] + x1[0] * x1[1] + x2[0] * x2[1];
    }
    double th = atan2(num, den);
    double perm = fabs(x1[0] * x2[1]) + fabs(x2[0] * x1[1]) + 1e-300;
    if (den < 0.0 && fabs(num) <= 1e-2 * fabs(den) + 1e-5 * perm)   // close to the cut: exact branch
        th = branch_fix(th, -edge_sign_slow(A, B, p, D, cnt, status));  // sign(num) = -sign det[a, b, d]
    if (cnt) atomicAdd(&cnt[CNT_CUT_SIGN], 1ull);
    return (float)th;
}

// Exact branch for a pair whose |Omega/2| is within 0.01 of pi (ray close to
// crossing AB): theta moves by 2pi when the rounded num has the wrong sign.
static __device__ __noinline__ float cut_fix(float th, float4 va, float4 vb, float3 p, Frame fr,
                                             unsigned long long *cnt, int *status) {
    float3 A = make_float3(va.x, va.y, va.z), B = make_float3(vb.x, vb.y, vb.z);
    float3 D = make_float3(fr.d[0], fr.d[1], fr.d[2]);
    int s = -edge_sign_slow(A, B, p, D, cnt, status);   // sign(num) = -sign det[a, b, d]
    if (cnt) atomicAdd(&cnt[CNT_CUT_SIGN], 1ull);
    if (s < 0 && th > 0.f) return th - 6.2831853071795865f;
    if (s > 0 && th < 0.f) return th + 6.2831853071795865f;
    return th;
}

// ---- packed float32 pairs ---------------------------------------------------
// float2 with the compiler's packed builtins (__fadd2_rn, __fmul2_rn,
// __ffma2_rn: add/mul/fma.rn.f32x2 on sm_100 and later), so the compiler sees
// both lanes and can keep them in place.
typedef float2 f2;

__device__ __forceinline__ f2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float lo2(f2 v) { return v.x; }
__device__ __forceinline__ float hi2(f2 v) { return v.y; }
// MUFU reciprocal (rcp.approx, about 1 ulp); arguments here are normal floats
__device__ __forceinline__ float frcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }

#define GWN_AT_C8 0.00284989f
#define GWN_AT_C7 -0.01606863f
#define GWN_AT_C6 0.04269152f
#define GWN_AT_C5 -0.07504295f
#define GWN_AT_C4 0.10640934f
#define GWN_AT_C3 -0.14203644f
#define GWN_AT_C2 0.19992619f
#define GWN_AT_C1 -0.33333073f
#define GWN_AT_C0 0.99999998f

// Packed constants, materialised once per thread.
struct PackedConsts {
    f2 e1x, e1y, e1z, e2x, e2y, e2z, nx, ny, nz;
    f2 c[9];
    f2 pi;
    f2 near2;
};

__device__ __forceinline__ f2 abs2(f2 v) { return make_float2(fabsf(v.x), fabsf(v.y)); }

// Omega/2 = atan2(num, den) for two queries through the half-angle identity:
// with |z| = sqrt(num^2 + den^2) and v = num / (|z| + |den|) in [-1, 1],
//   atan2(num, den) = 2 atan(v)             if den >= 0
//                   = copysign(pi, num) - 2 atan(v)  if den < 0,
// atan(v) = v P(v^2) (odd minimax polynomial, valid on [-1, 1]).  `cut` gets
// one bit per element where den < 0 and |v| < 0.005, i.e. |Omega/2| within
// 0.01 of pi (the ray passes close to the edge: exact sign needed).
__device__ __forceinline__ f2 half_angle_atan2(f2 num, f2 den, const PackedConsts &K, int &cut, f2 &z2out) {
    f2 z2 = fma2(num, num, mul2(den, den));
    z2out = z2;
    float z20 = fmaxf(lo2(z2), 1e-37f), z21 = fmaxf(hi2(z2), 1e-37f);
    f2 za = mul2(pk(z20, z21), pk(rsqrtf(z20), rsqrtf(z21)));
    f2 D = add2(za, abs2(den));
    f2 v = mul2(num, pk(frcp(lo2(D)), frcp(hi2(D))));
    f2 v2 = mul2(v, v);
    f2 p = fma2(K.c[8], v2, K.c[7]);
    p = fma2(p, v2, K.c[6]);
    p = fma2(p, v2, K.c[5]);
    p = fma2(p, v2, K.c[4]);
    p = fma2(p, v2, K.c[3]);
    p = fma2(p, v2, K.c[2]);
    p = fma2(p, v2, K.c[1]);
    p = fma2(p, v2, K.c[0]);
    f2 a = mul2(p, v);
    f2 a2 = add2(a, a);
    f2 cpi = make_float2(copysignf(lo2(K.pi), num.x), copysignf(hi2(K.pi), num.y));   // copysign(pi, num)
    f2 neg = sub2(cpi, a2);
    float d0 = lo2(den), d1 = hi2(den);
    cut = ((d0 < 0.f) & (fabsf(lo2(v)) < 0.005f)) | (((d1 < 0.f) & (fabsf(hi2(v)) < 0.005f)) << 1);
    return pk(d0 >= 0.f ? lo2(a2) : lo2(neg), d1 >= 0.f ? hi2(a2) : hi2(neg));
}

template <int KP, int MINB>   // KP query pairs per thread, MINB blocks per SM
__global__ void __launch_bounds__(256, MINB) bterm3d_kernel(const float4 *__restrict__ bseq, int nb, Frame fr,
                                                            Frame64 f64, QuerySrc q, const int32_t *__restrict__ chi,
                                                            float *__restrict__ w_out, float *__restrict__ b_out,
                                                            unsigned long long *cnt, int *status) {
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * (2 * KP) + threadIdx.x;
    PackedConsts K;
    K.e1x = pk(fr.e1[0], fr.e1[0]); K.e1y = pk(fr.e1[1], fr.e1[1]); K.e1z = pk(fr.e1[2], fr.e1[2]);
    K.e2x = pk(fr.e2[0], fr.e2[0]); K.e2y = pk(fr.e2[1], fr.e2[1]); K.e2z = pk(fr.e2[2], fr.e2[2]);
    K.nx = pk(fr.n[0], fr.n[0]); K.ny = pk(fr.n[1], fr.n[1]); K.nz = pk(fr.n[2], fr.n[2]);
    K.c[0] = pk(GWN_AT_C0, GWN_AT_C0); K.c[1] = pk(GWN_AT_C1, GWN_AT_C1); K.c[2] = pk(GWN_AT_C2, GWN_AT_C2);
    K.c[3] = pk(GWN_AT_C3, GWN_AT_C3); K.c[4] = pk(GWN_AT_C4, GWN_AT_C4); K.c[5] = pk(GWN_AT_C5, GWN_AT_C5);
    K.c[6] = pk(GWN_AT_C6, GWN_AT_C6); K.c[7] = pk(GWN_AT_C7, GWN_AT_C7); K.c[8] = pk(GWN_AT_C8, GWN_AT_C8);
    K.pi = pk(3.14159265358979f, 3.14159265358979f);
    K.near2 = pk(4e-6f, 4e-6f);
    f2 px[KP], py[KP], pz[KP], pa1[KP], pa2[KP], ps[KP], pr2[KP], sum[KP], cmp[KP];
#pragma unroll
    for (int j = 0; j < KP; j++) {
        int64_t i0 = base + (int64_t)(2 * j) * blockDim.x, i1 = i0 + blockDim.x;
        float3 p0 = i0 < q.n ? query_point3(q, i0) : make_float3(0.f, 0.f, 0.f);
        float3 p1 = i1 < q.n ? query_point3(q, i1) : make_float3(0.f, 0.f, 0.f);
        px[j] = pk(p0.x, p1.x); py[j] = pk(p0.y, p1.y); pz[j] = pk(p0.z, p1.z);
        sum[j] = pk(0.f, 0.f); cmp[j] = pk(0.f, 0.f);
    }
    // (a1, a2, s, |a|^2) of record v for query pair j
    auto project = [&](const f2 &vx, const f2 &vy, const f2 &vz, int j, f2 &a1, f2 &a2, f2 &s, f2 &r2out) {
        f2 ax = sub2(vx, px[j]), ay = sub2(vy, py[j]), az = sub2(vz, pz[j]);
        a1 = fma2(az, K.e1z, fma2(ay, K.e1y, mul2(ax, K.e1x)));
        a2 = fma2(az, K.e2z, fma2(ay, K.e2y, mul2(ax, K.e2x)));
        f2 an = fma2(az, K.nz, fma2(ay, K.ny, mul2(ax, K.nx)));
        f2 rp = fma2(a1, a1, mul2(a2, a2));
        f2 r2 = fma2(an, an, rp);
        float r20 = fmaxf(lo2(r2), 1e-37f), r21 = fmaxf(hi2(r2), 1e-37f);
        r2out = pk(r20, r21);
        f2 r = mul2(r2out, pk(rsqrtf(r20), rsqrtf(r21)));
        f2 sp = add2(r, an), dm = sub2(r, an);
        f2 sn = mul2(rp, pk(frcp(lo2(dm)), frcp(hi2(dm))));
        s = pk(lo2(an) >= 0.f ? lo2(sp) : lo2(sn), hi2(an) >= 0.f ? hi2(sp) : hi2(sn));
    };
    if (nb > 0) {
        float4 v0 = __ldg(&bseq[0]);
        {
            f2 vx = pk(v0.x, v0.x), vy = pk(v0.y, v0.y), vz = pk(v0.z, v0.z);
#pragma unroll
            for (int j = 0; j < KP; j++) project(vx, vy, vz, j, pa1[j], pa2[j], ps[j], pr2[j]);
        }
        float4 vprev = v0;
        for (int k = 1; k < nb; k++) {
            float4 v = __ldg(&bseq[k]);
            const bool edge = v.w != 0.f;     // uniform across the block
            f2 vx = pk(v.x, v.x), vy = pk(v.y, v.y), vz = pk(v.z, v.z);
#pragma unroll
            for (int j = 0; j < KP; j++) {
                f2 a1, a2, s, r2;
                project(vx, vy, vz, j, a1, a2, s, r2);
                if (edge) {
                    f2 num = sub2(mul2(pa1[j], a2), mul2(pa2[j], a1));
                    f2 den = fma2(ps[j], s, fma2(pa1[j], a1, mul2(pa2[j], a2)));
                    int cut;
                    f2 z2;
                    f2 th = half_angle_atan2(num, den, K, cut, z2);
                    // |z|^2 < (2e-3)^2 |a|^2 |b|^2: an endpoint within ~1e-3 rad of
                    // the forward ray (or p near the edge): float64 slow path
                    f2 lim = mul2(mul2(pr2[j], r2), K.near2);
                    int slow = (lo2(z2) < lo2(lim)) | ((hi2(z2) < hi2(lim)) << 1);
                    if (slow | cut) {                     // rare: exact branches / float64
                        float t0 = lo2(th), t1 = hi2(th);
                        if (slow & 1)
                            t0 = slow_theta(vprev, v, lo2(pa1[j]), lo2(pa2[j]), lo2(ps[j]), lo2(a1), lo2(a2), lo2(s),
                                            make_float3(lo2(px[j]), lo2(py[j]), lo2(pz[j])), fr, f64, cnt, status);
                        else if (cut & 1)
                            t0 = cut_fix(t0, vprev, v, make_float3(lo2(px[j]), lo2(py[j]), lo2(pz[j])), fr, cnt, status);
                        if (slow & 2)
                            t1 = slow_theta(vprev, v, hi2(pa1[j]), hi2(pa2[j]), hi2(ps[j]), hi2(a1), hi2(a2), hi2(s),
                                            make_float3(hi2(px[j]), hi2(py[j]), hi2(pz[j])), fr, f64, cnt, status);
                        else if (cut & 2)
                            t1 = cut_fix(t1, vprev, v, make_float3(hi2(px[j]), hi2(py[j]), hi2(pz[j])), fr, cnt, status);
                        th = pk(t0, t1);
                    }
                    f2 y = sub2(th, cmp[j]);          // compensated (Kahan) accumulation
                    f2 t = add2(sum[j], y);
                    cmp[j] = sub2(sub2(t, sum[j]), y);
                    sum[j] = t;
                }
                pa1[j] = a1; pa2[j] = a2; ps[j] = s; pr2[j] = r2;
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

template <int KP, int MINB>
static cudaError_t launch_bt(const float4 *bseq, int64_t n_bseq, const Frame &fr, const Frame64 &f64,
                             const QuerySrc &q, const int32_t *chi, float *w_out, float *b_out,
                             unsigned long long *cnt, int *status, cudaStream_t st) {
    const int threads = 256;
    int64_t per_block = (int64_t)threads * 2 * KP;
    int64_t blocks = (q.n + per_block - 1) / per_block;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    bterm3d_kernel<KP, MINB><<<(unsigned)blocks, threads, 0, st>>>(bseq, (int)n_bseq, fr, f64, q, chi, w_out,
                                                                   b_out, cnt, status);
    return cudaGetLastError();
}

cudaError_t launch_bterm3d(const float4 *bseq, int64_t n_bseq, const Frame &fr, const Frame64 &f64,
                           const QuerySrc &q, const int32_t *chi, float *w_out, float *b_out,
                           unsigned long long *cnt, int *status, int sm_count, cudaStream_t st) {
    (void)sm_count;
    if (q.n == 0) return cudaSuccess;
    static int impl = -1;
    if (impl < 0) {
        const char *e = getenv("GWN_BTERM_CFG");
        impl = e ? atoi(e) : 0;
    }
    switch (impl) {
        case 1: return launch_bt<1, 3>(bseq, n_bseq, fr, f64, q, chi, w_out, b_out, cnt, status, st);
        case 2: return launch_bt<2, 2>(bseq, n_bseq, fr, f64, q, chi, w_out, b_out, cnt, status, st);
        case 3: return launch_bt<1, 4>(bseq, n_bseq, fr, f64, q, chi, w_out, b_out, cnt, status, st);
        default: return launch_bt<1, 2>(bseq, n_bseq, fr, f64, q, chi, w_out, b_out, cnt, status, st);
    }
}

}  // namespace gwn
