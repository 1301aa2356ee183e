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
//   pi take the sign of num from -sign det[A-p, B-p, d_eps];
// * a boundary vertex within 1e-3 rad of the forward ray: its azimuth around
//   the ray is ill-conditioned in float32, so both incident edges are
//   recomputed in float64; a vertex exactly on the ray (decided exactly) is
//   seen by the perturbed ray d_eps in the direction -dp (dp = the first of
//   e_x, e_y, e_z not parallel to d, projected orthogonally to d), and its
//   edges take the limit of Omega under that perturbation.
//
// Arithmetic: two queries per 64-bit register pair; plain add/mul/fma run as
// packed f32x2 instructions (Blackwell), min/max, MUFU (rsqrt, reciprocal),
// compares and selects per element.  atan2 is a degree-8 minimax polynomial
// of atan(t) on [0, 1] (t = min/max of |num|, |den|) with octant fix-ups; its
// coefficients were fitted by Lawson-weighted least squares to the relative
// error of t*P(t^2) ~ atan(t) (1.5e-8 in exact arithmetic, <= 3 ulp in
// float32 against float64 atan2).  Accumulation over edges is compensated
// (Kahan).
//
// Layout: bseq holds the boundary loops as float4 records (x, y, z, w) in loop
// order; each loop is v0 (w = 0), v1 .. v_{n-1} (w = 1), v0 again (w = 1).
// w = 1 marks an edge from the previous record.  All lanes of a warp read the
// same record (broadcast); every thread carries 2*KP queries.
#include "gwn_internal.h"
#include "predicates.cuh"
#include "query.cuh"

namespace gwn {

#define GWN_CUT_THRESHOLD 3.1315926f   // pi - 0.01
#define GWN_INV_2PI 0.15915494309189535f
#define GWN_NEAR_RAY2 1e-6f            // (1e-3 rad)^2: slow path for vertices this close to the ray

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

// Omega/2 of edge A->B in float64, with the exact-sign rules above.
static __device__ __noinline__ float slow_theta(float4 va, float4 vb, float3 p, Frame fr, Frame64 f,
                                                unsigned long long *cnt, int *status) {
    float3 A = make_float3(va.x, va.y, va.z), B = make_float3(vb.x, vb.y, vb.z);
    float3 D = make_float3(fr.d[0], fr.d[1], fr.d[2]);
    double a[3] = {(double)A.x - p.x, (double)A.y - p.y, (double)A.z - p.z};
    double b[3] = {(double)B.x - p.x, (double)B.y - p.y, (double)B.z - p.z};
    bool ra = on_forward_ray(A, p, D), rb = on_forward_ray(B, p, D);
    double num, den, perm;
    if (ra && rb) {
        num = 0.0; den = 1.0; perm = 1.0;           // edge along the ray: limit 0
    } else if (ra) {                                  // A seen in direction -dp
        double bx0 = b[1] * f.dh[2] - b[2] * f.dh[1], bx1 = b[2] * f.dh[0] - b[0] * f.dh[2],
               bx2 = b[0] * f.dh[1] - b[1] * f.dh[0];
        num = f.dp[0] * bx0 + f.dp[1] * bx1 + f.dp[2] * bx2;
        den = -(b[0] * f.dp[0] + b[1] * f.dp[1] + b[2] * f.dp[2]);
        perm = fabs(f.dp[0] * bx0) + fabs(f.dp[1] * bx1) + fabs(f.dp[2] * bx2) + 1e-300;
    } else if (rb) {                                  // B seen in direction -dp
        double px0 = f.dp[1] * f.dh[2] - f.dp[2] * f.dh[1], px1 = f.dp[2] * f.dh[0] - f.dp[0] * f.dh[2],
               px2 = f.dp[0] * f.dh[1] - f.dp[1] * f.dh[0];
        num = a[0] * px0 + a[1] * px1 + a[2] * px2;
        den = -(a[0] * f.dp[0] + a[1] * f.dp[1] + a[2] * f.dp[2]);
        perm = fabs(a[0] * px0) + fabs(a[1] * px1) + fabs(a[2] * px2) + 1e-300;
    } else {
        double a1 = a[0] * f.e1[0] + a[1] * f.e1[1] + a[2] * f.e1[2];
        double a2 = a[0] * f.e2[0] + a[1] * f.e2[1] + a[2] * f.e2[2];
        double an = a[0] * f.n[0] + a[1] * f.n[1] + a[2] * f.n[2];
        double b1 = b[0] * f.e1[0] + b[1] * f.e1[1] + b[2] * f.e1[2];
        double b2 = b[0] * f.e2[0] + b[1] * f.e2[1] + b[2] * f.e2[2];
        double bn = b[0] * f.n[0] + b[1] * f.n[1] + b[2] * f.n[2];
        double ra2 = a1 * a1 + a2 * a2, rb2 = b1 * b1 + b2 * b2;
        double la = sqrt(ra2 + an * an), lb = sqrt(rb2 + bn * bn);
        double sa = an >= 0.0 ? la + an : ra2 / (la - an);
        double sb = bn >= 0.0 ? lb + bn : rb2 / (lb - bn);
        num = a1 * b2 - a2 * b1;
        den = sa * sb + a1 * b1 + a2 * b2;
        perm = fabs(a1 * b2) + fabs(a2 * b1) + 1e-300;
    }
    if (den < 0.0 && fabs(num) <= 64.0 * 1.1102230246251565e-16 * perm) {
        int s = edge_sign_slow(A, B, p, D, cnt, status);   // sign(num) = -s
        if (s > 0) num = -fabs(num);
        else if (s < 0) num = fabs(num);
    }
    if (cnt) atomicAdd(&cnt[CNT_CUT_SIGN], 1ull);
    return (float)atan2(num, den);
}

// Take the sign of num from the exact predicate (ray close to crossing AB).
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

// ---- packed float32 pairs ---------------------------------------------------
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
// MUFU reciprocal (rcp.approx, about 1 ulp); arguments here are normal floats
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
__global__ void __launch_bounds__(256) bterm3d_kernel(const float4 *__restrict__ bseq, int nb, Frame fr, Frame64 f64,
                                                      QuerySrc q, const int32_t *__restrict__ chi,
                                                      float *__restrict__ w_out, float *__restrict__ b_out,
                                                      unsigned long long *cnt, int *status) {
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * (2 * KP) + threadIdx.x;
    f2 px[KP], py[KP], pz[KP], pa1[KP], pa2[KP], ps[KP], sum[KP], cmp[KP];
    int pnear[KP];
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
    // (a1, a2, s) of record v for query pair j; `near` gets one bit per
    // element whose vertex lies within 1e-3 rad of the forward ray
    auto project = [&](float4 v, int j, f2 &a1, f2 &a2, f2 &s, int &near) {
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
        float an0 = lo2(an), an1 = hi2(an);
        s = pk(an0 >= 0.f ? lo2(sp) : lo2(sn), an1 >= 0.f ? hi2(sp) : hi2(sn));
        near = ((an0 < 0.f) & (lo2(rp) < GWN_NEAR_RAY2 * r20)) | (((an1 < 0.f) & (hi2(rp) < GWN_NEAR_RAY2 * r21)) << 1);
    };
    if (nb > 0) {
        float4 v0 = __ldg(&bseq[0]);
#pragma unroll
        for (int j = 0; j < KP; j++) project(v0, j, pa1[j], pa2[j], ps[j], pnear[j]);
        float4 vprev = v0;
        for (int k = 1; k < nb; k++) {
            float4 v = __ldg(&bseq[k]);
            const bool edge = v.w != 0.f;     // uniform across the block
#pragma unroll
            for (int j = 0; j < KP; j++) {
                f2 a1, a2, s;
                int near;
                project(v, j, a1, a2, s, near);
                if (edge) {
                    f2 num = sub2(mul2(pa1[j], a2), mul2(pa2[j], a1));
                    f2 den = fma2(ps[j], s, fma2(pa1[j], a1, mul2(pa2[j], a2)));
                    f2 th = atan2_2(num, den);
                    float t0 = lo2(th), t1 = hi2(th);
                    int slow = pnear[j] | near;
                    if (slow & 1)
                        t0 = slow_theta(vprev, v, make_float3(lo2(px[j]), lo2(py[j]), lo2(pz[j])), fr, f64, cnt, status);
                    else if (fabsf(t0) > GWN_CUT_THRESHOLD)
                        t0 = cut_fix(t0, vprev, v, make_float3(lo2(px[j]), lo2(py[j]), lo2(pz[j])), fr, cnt, status);
                    if (slow & 2)
                        t1 = slow_theta(vprev, v, make_float3(hi2(px[j]), hi2(py[j]), hi2(pz[j])), fr, f64, cnt, status);
                    else if (fabsf(t1) > GWN_CUT_THRESHOLD)
                        t1 = cut_fix(t1, vprev, v, make_float3(hi2(px[j]), hi2(py[j]), hi2(pz[j])), fr, cnt, status);
                    th = pk(t0, t1);
                    f2 y = sub2(th, cmp[j]);          // compensated (Kahan) accumulation
                    f2 t = add2(sum[j], y);
                    cmp[j] = sub2(sub2(t, sum[j]), y);
                    sum[j] = t;
                }
                pa1[j] = a1; pa2[j] = a2; ps[j] = s; pnear[j] = near;
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

cudaError_t launch_bterm3d(const float4 *bseq, int64_t n_bseq, const Frame &fr, const Frame64 &f64,
                           const QuerySrc &q, const int32_t *chi, float *w_out, float *b_out,
                           unsigned long long *cnt, int *status, int sm_count, cudaStream_t st) {
    (void)sm_count;
    if (q.n == 0) return cudaSuccess;
    constexpr int KP = 2;
    const int threads = 256;
    int64_t per_block = (int64_t)threads * 2 * KP;
    int64_t blocks = (q.n + per_block - 1) / per_block;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    bterm3d_kernel<KP><<<(unsigned)blocks, threads, 0, st>>>(bseq, (int)n_bseq, fr, f64, q, chi, w_out, b_out, cnt,
                                                             status);
    return cudaGetLastError();
}

}  // namespace gwn
