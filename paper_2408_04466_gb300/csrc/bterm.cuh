// bterm.cuh -- device parts of the boundary term shared by the per-geometry
// kernels (bterm.cu) and the batched mesh launch (meshbatch.cu).  See
// bterm.cu for the method and its precision.
#pragma once
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
__device__ __forceinline__ float branch_fix(float th, int s_num) {
    if (s_num < 0 && th > 0.f) return th - 6.2831853071795865f;
    if (s_num > 0 && th < 0.f) return th + 6.2831853071795865f;
    return th;
}

// Omega/2 of edge A->B in float64 for flagged pairs (|z| small relative to
// |a||b|: an endpoint near the forward ray, or p near the edge).  Each
// endpoint within 2e-4 rad of the forward ray is recomputed in float64, or,
// when it lies exactly on the ray, replaced by the perturbation limit
// (x_perp = u = -dp in the frame, s_x = 0).  Other endpoints keep their
// float32 projection (fa*, fb*), the values their other edge uses, so the
// first-order cancellation of their rounding between their two edges holds.
// The decision depends only on the vertex and the query, so both edges of a
// vertex make the same one.  A spindle edge (p close to the edge relative to
// its length: a and b nearly opposite) takes both endpoints in float64: its
// angle rests on the small sum of their directions, which float32 rounding
// would perturb by ~u / sqrt(2 (1 + cos phi)); the float32/float64 mismatch
// this leaves at a shared endpoint moves that endpoint's direction by ~u,
// which changes w by ~u only.
static __device__ __noinline__ float slow_theta(float4 va, float4 vb, float fa1, float fa2, float fsa, float fb1,
                                                float fb2, float fsb, float3 p, Frame fr, Frame64 f, bool spindle,
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
        bool near = an < 0.0 && rp < 4e-8 * (rp + an * an);          // sin^2 < T^2
        if (!near && !spindle) {
            x1[e] = f1[e]; x2[e] = f2v[e]; xs[e] = fs[e];
            continue;
        }
        if (!near) {                                                  // spindle edge: float64 endpoint
            double r = sqrt(rp + an * an);
            x1[e] = a1; x2[e] = a2; xs[e] = an >= 0.0 ? r + an : rp / (r - an);
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
    // num and den are accurate to float64 rounding; the angle itself is only
    // needed to float32 accuracy, so it is taken in float32 (float64 is a
    // narrow pipe on this part) after scaling both by a power of two.
    double mx = fmax(fabs(num), fabs(den));
    int ex = mx > 0.0 ? ilogb(mx) : 0;
    float th = atan2f((float)scalbn(num, -ex), (float)scalbn(den, -ex));
    double perm = fabs(x1[0] * x2[1]) + fabs(x2[0] * x1[1]) + 1e-300;
    if (den < 0.0 && fabs(num) <= 1e-2 * fabs(den) + 1e-5 * perm)   // close to the cut: exact branch
        th = branch_fix(th, -edge_sign_slow(A, B, p, D, cnt, status));  // sign(num) = -sign det[a, b, d]
    if (cnt) atomicAdd(&cnt[CNT_CUT_SIGN], 1ull);
    return th;
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

// Packed constants (kernel parameters: both elements of each pair equal).
struct PackedConsts {
    f2 c[9];
    f2 pi;
    f2 nearv;    // -T^2 / 2: a vertex within T of the forward ray
    f2 spin;     // -tau: an edge seen from p at an angle within ~sqrt(tau) of pi
    f2 cut2n;    // -1e-4
};

// the constants of the main pass (host; bterm.cu)
PackedConsts bterm_consts();

__device__ __forceinline__ f2 abs2(f2 v) { return make_float2(fabsf(v.x), fabsf(v.y)); }
// MUFU reciprocal square root (rsqrt.approx, about 2 ulp); arguments here are
// normal floats (clamped to >= 1e-37)
__device__ __forceinline__ float frsqrt(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// One boundary record seen from a query pair: frame coordinates (a1, a2),
// stereographic scale s = |a| + a_n (or |a_perp|^2 / (|a| - a_n) when
// a_n < 0) and q = s |a|.
struct VState {
    f2 a1, a2, s, q;
};

// Frame coordinates of a = A - p as double-float differences: the record
// holds A.e (e = e1, e2, n) as hi + lo floats (computed per direction in
// float64), the query -p.e as hi + lo (error-free float32 transforms), so
//   a_e = (A_hi - p_hi) + (A_lo - p_lo)
// is correct to about 2u |a_e| + u^2 (|A| + |p|): relative to the component
// itself, not to |a| as a float32 projection of A - p would be, which keeps
// a vertex's azimuth around the ray well conditioned down to tiny angles.
struct QPair {
    f2 n1h, n2h, nnh, n1l, n2l, nnl;      // -(p.e1), -(p.e2), -(p.n) as hi + lo, two queries
};

// The sign bits of f0 / f1 are set when the vertex lies within T of the
// forward ray of query element 0 / 1: there 1 + a_n/|a| ~ delta^2 / 2, so the
// test is s < (T^2 / 2) |a|.
__device__ __forceinline__ void project(float4 rh, float4 rl, const QPair &Q, VState &o, const PackedConsts &K,
                                        unsigned &f0, unsigned &f1) {
    f2 h1 = pk(rh.x, rh.x), h2 = pk(rh.y, rh.y), hn = pk(rh.z, rh.z);
    f2 l1 = pk(rl.x, rl.x), l2 = pk(rl.y, rl.y), ln = pk(rl.z, rl.z);
    o.a1 = add2(add2(h1, Q.n1h), add2(l1, Q.n1l));
    o.a2 = add2(add2(h2, Q.n2h), add2(l2, Q.n2l));
    f2 an = add2(add2(hn, Q.nnh), add2(ln, Q.nnl));
    f2 rp = fma2(o.a1, o.a1, mul2(o.a2, o.a2));
    f2 r2 = fma2(an, an, rp);
    float r20 = fmaxf(lo2(r2), 1e-37f), r21 = fmaxf(hi2(r2), 1e-37f);
    f2 r = mul2(pk(r20, r21), pk(frsqrt(r20), frsqrt(r21)));
    f2 sp = add2(r, an), dm = sub2(r, an);
    f2 sn = mul2(rp, pk(frcp(lo2(dm)), frcp(hi2(dm))));
    o.s = pk(lo2(an) >= 0.f ? lo2(sp) : lo2(sn), hi2(an) >= 0.f ? hi2(sp) : hi2(sn));
    o.q = mul2(o.s, r);
    f2 tv = fma2(r, K.nearv, o.s);
    f0 |= __float_as_uint(lo2(tv));
    f1 |= __float_as_uint(hi2(tv));
}

// -(p.e) as hi + lo from float32 arithmetic: exact products (FMA), TwoSum
// of the high parts, float sum of the (small) error terms, renormalised.
__device__ __forceinline__ void neg_dot_df(float3 p, const float e[3], float &hi, float &lo) {
    float hx = p.x * e[0], lx = fmaf(p.x, e[0], -hx);
    float hy = p.y * e[1], ly = fmaf(p.y, e[1], -hy);
    float hz = p.z * e[2], lz = fmaf(p.z, e[2], -hz);
    float s = hx + hy, bs = s - hx, es = (hx - (s - bs)) + (hy - bs);
    float t = s + hz, bt = t - s, et = (s - (t - bt)) + (hz - bt);
    float l = ((lx + ly) + lz) + (es + et);
    float h = t + l;
    lo = -(l - (h - t));
    hi = -h;
}

// Omega/2 = atan2(num, den) of edge P -> Q for a query pair, through the
// half-angle identity: with |z| = sqrt(num^2 + den^2) and
// v = num / (|z| + |den|) in [-1, 1],
//   atan2(num, den) = 2 atan(v)                      if den >= 0
//                   = copysign(pi, num) - 2 atan(v)  if den < 0,
// atan(v) = v P(v^2) (odd minimax polynomial, valid on [-1, 1]).
// f0 / f1 get a set sign bit when element 0 / 1 needs the slow path:
//   cut:  den < 0 and num^2 < 1e-4 |z|^2 (|Omega/2| within ~0.01 of pi: the
//         ray passes close to the edge, the branch needs the exact sign);
//   spindle: |z|^2 < tau q_a q_b.  Since |z|^2 = 2 (1 + a.b/(|a||b|)) q_a q_b
//         (q = s |a|), this holds when the edge is seen from p at an angle
//         phi with 2 (1 + cos phi) < tau: p close to the edge relative to
//         the edge's length.  There a and b are nearly opposite and the plane
//         they span (the great circle of the edge's image) rests on their
//         small sum, whose float32 rounding error grows like
//         1 / sqrt(2 (1 + cos phi)); with tau = 1e-2 the float32 error of
//         an unflagged edge stays below ~1e-7 in w.
// (Vertices near the forward ray are flagged in project.)
__device__ __forceinline__ f2 edge_theta(const VState &P, const VState &Q, const PackedConsts &K, unsigned &f0,
                                         unsigned &f1) {
    f2 num = sub2(mul2(P.a1, Q.a2), mul2(P.a2, Q.a1));
    f2 den = fma2(P.s, Q.s, fma2(P.a1, Q.a1, mul2(P.a2, Q.a2)));
    f2 nn = mul2(num, num);
    f2 z2 = fma2(den, den, nn);
    float z20 = fmaxf(lo2(z2), 1e-37f), z21 = fmaxf(hi2(z2), 1e-37f);
    f2 za = mul2(pk(z20, z21), pk(frsqrt(z20), frsqrt(z21)));
    f2 Dn = add2(za, abs2(den));
    f2 v = mul2(num, pk(frcp(lo2(Dn)), frcp(hi2(Dn))));
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
    f2 tc = fma2(z2, K.cut2n, nn);
    f2 ts = fma2(mul2(P.q, Q.q), K.spin, z2);
    f0 = (__float_as_uint(lo2(den)) & __float_as_uint(lo2(tc))) | __float_as_uint(lo2(ts));
    f1 = (__float_as_uint(hi2(den)) & __float_as_uint(hi2(tc))) | __float_as_uint(hi2(ts));
    float d0 = lo2(den), d1 = hi2(den);
    return pk(d0 >= 0.f ? lo2(a2) : lo2(neg), d1 >= 0.f ? hi2(a2) : hi2(neg));
}

// Record vq after the previous record for KP query pairs: project vq into Q
// and, when vq closes an edge (w != 0), add Omega/2 of P -> Q to the
// compensated sums and its slow-path bits to the per-query flags.  Called
// with the roles of P and Q alternating, so no state is copied.
template <int KP>
__device__ __forceinline__ void bterm_step(const VState (&P)[KP], VState (&Q)[KP], float4 rh, float4 rl,
                                           const QPair (&qp)[KP], f2 (&sum)[KP], f2 (&cmp)[KP],
                                           unsigned (&fl)[KP][2], const PackedConsts &K) {
#pragma unroll
    for (int j = 0; j < KP; j++) project(rh, rl, qp[j], Q[j], K, fl[j][0], fl[j][1]);
    float4 vq = rh;
    if (vq.w == 0.f) return;                  // first record of a loop (uniform)
#pragma unroll
    for (int j = 0; j < KP; j++) {
        unsigned f0, f1;
        f2 th = edge_theta(P[j], Q[j], K, f0, f1);
        fl[j][0] |= f0;
        fl[j][1] |= f1;
        f2 y = sub2(th, cmp[j]);              // compensated (Kahan) accumulation
        f2 t = add2(sum[j], y);
        cmp[j] = sub2(sub2(t, sum[j]), y);
        sum[j] = t;
    }
}

// Main pass: every query, float32 only.  A query with a flagged pair is not
// written; its index goes to the deferred list, which the careful pass
// recomputes in full.
// The main pass of one block (bterm_main_pass.inc) as a function, for the
// batched mesh launch.
template <int KP>
__device__ __forceinline__ void bterm_block(const float4 *__restrict__ bframe, int nb, const Frame &fr,
                                           const PackedConsts &Kp, const QuerySrc &q, int64_t base, int64_t gofs,
                                           const int32_t *__restrict__ chi, float *__restrict__ w_out,
                                           float *__restrict__ b_out, uint8_t *__restrict__ in_out,
                                           int32_t *__restrict__ defer, int32_t *defer_count) {
#include "bterm_main_pass.inc"
}

// ---- careful pass: deferred queries, scalar ------------------------------------
struct VState1 {
    float a1, a2, s, r2, q;
};

__device__ __forceinline__ VState1 project1(float4 v, float3 p, const Frame &fr) {
    float ax = v.x - p.x, ay = v.y - p.y, az = v.z - p.z;
    VState1 o;
    o.a1 = fmaf(az, fr.e1[2], fmaf(ay, fr.e1[1], ax * fr.e1[0]));
    o.a2 = fmaf(az, fr.e2[2], fmaf(ay, fr.e2[1], ax * fr.e2[0]));
    float an = fmaf(az, fr.n[2], fmaf(ay, fr.n[1], ax * fr.n[0]));
    float rp = fmaf(o.a1, o.a1, o.a2 * o.a2);
    o.r2 = fmaxf(fmaf(an, an, rp), 1e-37f);
    float r = o.r2 * frsqrt(o.r2);
    o.s = an >= 0.f ? r + an : rp * frcp(r - an);
    o.q = o.s * r;
    return o;
}

// the same float32 formulation as edge_theta (one element), with the
// flagged cases resolved: float64 near the forward ray and for spindle edges
// (2 (1 + cos phi) < 2e-2, twice the main pass's bar, for the plain float32
// projections here), exact branch at the cut
__device__ __forceinline__ float edge_theta_careful(const VState1 &A, const VState1 &B, float4 va, float4 vb,
                                                    float3 p, const Frame &fr, const Frame64 &f64,
                                                    unsigned long long *cnt, int *status) {
    float num = A.a1 * B.a2 - A.a2 * B.a1;
    float den = fmaf(A.s, B.s, fmaf(A.a1, B.a1, A.a2 * B.a2));
    float nn = num * num;
    float z2 = fmaf(den, den, nn);
    bool spindle = fmaf(A.q * B.q, -2e-2f, z2) < 0.f;
    if (spindle || fmaf(A.r2 * B.r2, -4.1e-8f, z2) < 0.f)    // T = 2e-4 for float32 projections
        return slow_theta(va, vb, A.a1, A.a2, A.s, B.a1, B.a2, B.s, p, fr, f64, spindle, cnt, status);
    float zc = fmaxf(z2, 1e-37f);
    float v = num * frcp(zc * frsqrt(zc) + fabsf(den));
    float v2 = v * v;
    float q = fmaf(GWN_AT_C8, v2, GWN_AT_C7);
    q = fmaf(q, v2, GWN_AT_C6);
    q = fmaf(q, v2, GWN_AT_C5);
    q = fmaf(q, v2, GWN_AT_C4);
    q = fmaf(q, v2, GWN_AT_C3);
    q = fmaf(q, v2, GWN_AT_C2);
    q = fmaf(q, v2, GWN_AT_C1);
    q = fmaf(q, v2, GWN_AT_C0);
    float a2 = 2.f * (q * v);
    float th = den >= 0.f ? a2 : copysignf(3.14159265358979f, num) - a2;
    if (den < 0.f && fmaf(z2, -1e-4f, nn) < 0.f) th = cut_fix(th, va, vb, p, fr, cnt, status);
    return th;
}

// B_d of one query by one block of 128 threads (the careful pass): thread l
// sums the edges ending at records [k0, k1), a contiguous run of about
// (nb - 1)/128 records, starting from the projection of record k0 - 1.  A
// vertex on a run boundary is projected by both threads with the same
// arithmetic, so its rounding still cancels between its two edges.  The
// threads' compensated sums are combined by a TwoSum tree in a fixed order
// (warp shuffles, then the four warps in turn).  The result is returned on
// thread 0; every thread of the block must call.
__device__ __forceinline__ float careful_block_B(const float4 *__restrict__ bseq, int nb, const Frame &fr,
                                                const Frame64 &f64, float3 p, unsigned long long *cnt, int *status) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __shared__ float s_part[2][128 / 32];
    const int per = nb > 1 ? (nb - 1 + 127) / 128 : 0;
    float sum = 0.f, cmp = 0.f;
    int k0 = 1 + threadIdx.x * per, k1 = k0 + per < nb ? k0 + per : nb;
    if (k0 < k1) {
        float4 vp = __ldg(&bseq[k0 - 1]);
        VState1 A = project1(vp, p, fr);
        for (int k = k0; k < k1; k++) {
            float4 v = __ldg(&bseq[k]);
            VState1 B = project1(v, p, fr);
            if (v.w != 0.f) {
                float th = edge_theta_careful(A, B, vp, v, p, fr, f64, cnt, status);
                float y = th - cmp;
                float t = sum + y;
                cmp = (t - sum) - y;
                sum = t;
            }
            A = B;
            vp = v;
        }
    }
    // combine (value, error) pairs across the warp, then across the
    // block's warps in fixed order, with TwoSum
    float s = sum, e = -cmp;
    for (int off = 16; off > 0; off >>= 1) {
        float s2 = __shfl_down_sync(0xffffffffu, s, off), e2 = __shfl_down_sync(0xffffffffu, e, off);
        float t = s + s2, bv = t - s, err = (s - (t - bv)) + (s2 - bv);
        s = t;
        e = e + e2 + err;
    }
    if (lane == 0) { s_part[0][wid] = s; s_part[1][wid] = e; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 128 / 32; w++) {
            float s2 = s_part[0][w], e2 = s_part[1][w];
            float t = s + s2, bv = t - s, err = (s - (t - bv)) + (s2 - bv);
            s = t;
            e = e + e2 + err;
        }
    }
    float Bv = __fmul_rn(__fadd_rn(s, e), GWN_INV_2PI);
    __syncthreads();
    return Bv;
}

}  // namespace gwn
