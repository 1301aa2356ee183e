// predicates.cuh -- exact orientation predicates on float32 inputs (device).
//
// The signed crossing count (Eq. chi) is an integer decided by the signs of
//   edge(A, B; p, d)  = det[A - p, B - p, d]          (side of the ray line)
//   orient(v0,v1,v2; p) = det[v0 - p, v1 - p, v2 - p]  (ray origin vs plane)
// Every sign is exact.  Three stages, cheapest first:
//   1. float32 evaluation with a static forward-error bound (hot path);
//   2. float64 evaluation with its bound;
//   3. exact evaluation: the determinant is expanded into a sum of products of
//      the float32 inputs (each product of three float32 values is an exact
//      two-term float64 expansion via FMA), summed into a nonoverlapping
//      floating-point expansion by repeated two-sum ("Grow-Expansion",
//      Shewchuk, Adaptive Precision Floating-Point Arithmetic and Fast Robust
//      Geometric Predicates, 1997); its largest component carries the sign.
// Zero determinants of the edge test are broken by the symbolic perturbation
// d_eps = d + eps e_x + eps^2 e_y + eps^3 e_z: the sign is the first nonzero
// of det[a,b,d], (a x b)_x, (a x b)_y, (a x b)_z.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gwn_internal.h"

namespace gwn {

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = a + b;
    double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Nonoverlapping expansion (increasing magnitude, zeros eliminated).
template <int MAXC>
struct Expansion {
    double c[MAXC];
    int n;
    int overflow;
    __device__ __forceinline__ void init() { n = 0; overflow = 0; }
    // Grow-Expansion with zero elimination: e := e + x exactly.
    __device__ __forceinline__ void add(double x) {
        if (x == 0.0) return;
        double q = x;
        int k = 0;
        for (int i = 0; i < n; i++) {
            double s, h;
            two_sum(q, c[i], s, h);
            if (h != 0.0) c[k++] = h;
            q = s;
        }
        if (q != 0.0) {
            if (k < MAXC) c[k++] = q;
            else overflow = 1;
        }
        n = k;
    }
    __device__ __forceinline__ int sign() const {
        if (n == 0) return 0;
        return c[n - 1] > 0.0 ? 1 : -1;
    }
};

// exact product x*y*z of float32 values as hi + lo
__device__ __forceinline__ void prod3(float x, float y, float z, double &hi, double &lo) {
    double p = (double)x * (double)y;   // exact: 48-bit product
    hi = p * (double)z;
    lo = fma(p, (double)z, -hi);        // exact remainder
}

__device__ __forceinline__ float comp(const float3 &v, int i) { return i == 0 ? v.x : (i == 1 ? v.y : v.z); }

// Exact sign of det[A-P, B-P, D]: 6 permutations x 4 expansion terms.
static __device__ __noinline__ int exact_det_abd(float3 A, float3 B, float3 P, float3 D, int *status) {
    const int perm[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};
    Expansion<48> E;
    E.init();
    for (int k = 0; k < 6; k++) {
        double s = k < 3 ? 1.0 : -1.0;
        int i = perm[k][0], j = perm[k][1], l = perm[k][2];
        float ai = comp(A, i), pi = comp(P, i), bj = comp(B, j), pj = comp(P, j), dl = comp(D, l);
        double hi, lo;
        prod3(ai, bj, dl, hi, lo); E.add(s * hi); E.add(s * lo);
        prod3(ai, pj, dl, hi, lo); E.add(-s * hi); E.add(-s * lo);
        prod3(pi, bj, dl, hi, lo); E.add(-s * hi); E.add(-s * lo);
        prod3(pi, pj, dl, hi, lo); E.add(s * hi); E.add(s * lo);
    }
    if (E.overflow && status) atomicOr(status, ST_EXPANSION_OVERFLOW);
    return E.sign();
}

// Exact sign of ((A-P) x (B-P))_k.
static __device__ __noinline__ int exact_cross_comp(float3 A, float3 B, float3 P, int k) {
    int i = (k + 1) % 3, j = (k + 2) % 3;
    Expansion<8> E;
    E.init();
    float ai = comp(A, i), aj = comp(A, j), bi = comp(B, i), bj = comp(B, j);
    float pi = comp(P, i), pj = comp(P, j);
    // (ai - pi)(bj - pj) - (aj - pj)(bi - pi); two-factor products are exact in float64
    E.add((double)ai * bj); E.add(-(double)ai * pj); E.add(-(double)pi * bj); E.add((double)pi * pj);
    E.add(-(double)aj * bi); E.add((double)aj * pi); E.add((double)pj * bi); E.add(-(double)pj * pi);
    return E.sign();
}

// Exact sign of det[V0-P, V1-P, V2-P]: 6 permutations x 8 terms.
static __device__ __noinline__ int exact_orient(float3 V0, float3 V1, float3 V2, float3 P, int *status) {
    const int perm[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};
    Expansion<96> E;
    E.init();
    for (int k = 0; k < 6; k++) {
        double s = k < 3 ? 1.0 : -1.0;
        int i = perm[k][0], j = perm[k][1], l = perm[k][2];
        float x[2] = {comp(V0, i), comp(P, i)};
        float y[2] = {comp(V1, j), comp(P, j)};
        float z[2] = {comp(V2, l), comp(P, l)};
        for (int c = 0; c < 8; c++) {
            int neg = (c & 1) + ((c >> 1) & 1) + ((c >> 2) & 1);
            double sg = (neg & 1) ? -s : s;
            double hi, lo;
            prod3(x[c & 1], y[(c >> 1) & 1], z[(c >> 2) & 1], hi, lo);
            E.add(sg * hi);
            E.add(sg * lo);
        }
    }
    if (E.overflow && status) atomicOr(status, ST_EXPANSION_OVERFLOW);
    return E.sign();
}

// ---- float64 filters (16 ulp of the permanent) ----------------------------
#define GWN_F64_BOUND (16.0 * 1.1102230246251565e-16)
#define GWN_F32_BOUND (16.0f * 5.9604644775390625e-08f)

static __device__ __noinline__ int det_abd_sign_f64(float3 A, float3 B, float3 P, float3 D,
                                             unsigned long long *cnt, int *status) {
    double a0 = (double)A.x - P.x, a1 = (double)A.y - P.y, a2 = (double)A.z - P.z;
    double b0 = (double)B.x - P.x, b1 = (double)B.y - P.y, b2 = (double)B.z - P.z;
    double c0 = a1 * b2 - a2 * b1, c1 = a2 * b0 - a0 * b2, c2 = a0 * b1 - a1 * b0;
    double det = (double)D.x * c0 + (double)D.y * c1 + (double)D.z * c2;
    double perm = fabs((double)D.x) * (fabs(a1 * b2) + fabs(a2 * b1))
                + fabs((double)D.y) * (fabs(a2 * b0) + fabs(a0 * b2))
                + fabs((double)D.z) * (fabs(a0 * b1) + fabs(a1 * b0));
    if (fabs(det) > GWN_F64_BOUND * perm && perm > 1e-280) {
        if (cnt) atomicAdd(&cnt[CNT_FP64], 1ull);
        return det > 0 ? 1 : -1;
    }
    if (cnt) atomicAdd(&cnt[CNT_EXACT], 1ull);
    return exact_det_abd(A, B, P, D, status);
}

static __device__ __noinline__ int orient_sign_f64(float3 V0, float3 V1, float3 V2, float3 P,
                                            unsigned long long *cnt, int *status) {
    double a0 = (double)V0.x - P.x, a1 = (double)V0.y - P.y, a2 = (double)V0.z - P.z;
    double b0 = (double)V1.x - P.x, b1 = (double)V1.y - P.y, b2 = (double)V1.z - P.z;
    double c0 = (double)V2.x - P.x, c1 = (double)V2.y - P.y, c2 = (double)V2.z - P.z;
    double det = a0 * (b1 * c2 - b2 * c1) + a1 * (b2 * c0 - b0 * c2) + a2 * (b0 * c1 - b1 * c0);
    double perm = fabs(a0) * (fabs(b1 * c2) + fabs(b2 * c1)) + fabs(a1) * (fabs(b2 * c0) + fabs(b0 * c2))
                + fabs(a2) * (fabs(b0 * c1) + fabs(b1 * c0));
    if (fabs(det) > GWN_F64_BOUND * perm && perm > 1e-280) {
        if (cnt) atomicAdd(&cnt[CNT_FP64], 1ull);
        return det > 0 ? 1 : -1;
    }
    if (cnt) atomicAdd(&cnt[CNT_EXACT], 1ull);
    return exact_orient(V0, V1, V2, P, status);
}

// Perturbed edge sign when the unperturbed determinant is exactly zero.
static __device__ __noinline__ int sos_tiebreak(float3 A, float3 B, float3 P) {
    for (int k = 0; k < 3; k++) {
        int s = exact_cross_comp(A, B, P, k);
        if (s) return s;
    }
    return 0;
}

// Full (slow-path) perturbed edge sign from the original coordinates.
static __device__ __noinline__ int edge_sign_slow(float3 A, float3 B, float3 P, float3 D,
                                           unsigned long long *cnt, int *status) {
    int s = det_abd_sign_f64(A, B, P, D, cnt, status);
    if (s) return s;
    return sos_tiebreak(A, B, P);
}

// Float32 filters alone: +-1 when the float32 determinant settles the sign,
// 0 when it does not (the caller defers to the full predicate).
//
// They take edge vectors rather than the vectors to both end points:
// det[A-p, B-p, d] = det[A-p, B-A, d] exactly, and for a small triangle far
// from p the second form has permanent ~|A-p||B-A| instead of ~|A-p||B-p|,
// so the filter fails ~|B-A|/|A-p| times less often.  a = fl(A-p) and
// E = fl(B-A) each carry a relative rounding of u per component; with the
// products and sums the error stays below 16u times the permanent.
__device__ __forceinline__ int det3_sign_f32(float3 a, float3 b, float3 c) {
    float c0 = b.y * c.z - b.z * c.y;
    float c1 = b.z * c.x - b.x * c.z;
    float c2 = b.x * c.y - b.y * c.x;
    float det = a.x * c0 + a.y * c1 + a.z * c2;
    float perm = fabsf(a.x) * fmaf(fabsf(b.y), fabsf(c.z), fabsf(b.z) * fabsf(c.y))
               + fabsf(a.y) * fmaf(fabsf(b.z), fabsf(c.x), fabsf(b.x) * fabsf(c.z))
               + fabsf(a.z) * fmaf(fabsf(b.x), fabsf(c.y), fabsf(b.y) * fabsf(c.x));
    if (fabsf(det) > GWN_F32_BOUND * perm && perm > 1e-30f) return det > 0.f ? 1 : -1;
    return 0;
}

// Edge sign with the float32 filter (det3_sign_f32, on a = A-P and
// the edge vector B-A) first; falls back to the float64 filter, the exact
// expansion and the symbolic perturbation.
__device__ __forceinline__ int edge_sign(float3 a, float3 b, float3 A, float3 B, float3 P, float3 D,
                                         unsigned long long *cnt, int *status) {
    (void)b;
    float3 E = make_float3(B.x - A.x, B.y - A.y, B.z - A.z);
    int s = det3_sign_f32(D, a, E);
    if (s) return s;
    return edge_sign_slow(A, B, P, D, cnt, status);
}

// Orientation det[V0-P, V1-P, V2-P] with the float32 filter on
// -det[a, V1-V0, V0-V2] first, then float64 and exact.
__device__ __forceinline__ int orient_sign(float3 a, float3 b, float3 c, float3 V0, float3 V1, float3 V2,
                                           float3 P, unsigned long long *cnt, int *status) {
    (void)b; (void)c;
    float3 e0 = make_float3(V1.x - V0.x, V1.y - V0.y, V1.z - V0.z);
    float3 e2 = make_float3(V0.x - V2.x, V0.y - V2.y, V0.z - V2.z);
    int s = det3_sign_f32(a, e0, e2);
    if (s) return -s;
    return orient_sign_f64(V0, V1, V2, P, cnt, status);
}

// sign det[a, E, d] = sign det[A-p, B-p, d] (a = A-p, E = B-A)
__device__ __forceinline__ int edge_sign_f32(float3 a, float3 E, float3 D) { return det3_sign_f32(D, a, E); }

// tri_crossing (below) from float32 filters only: the result when every sign
// it depends on is settled in float32 (two settled edge signs that differ
// already rule a crossing out); otherwise `unsure` is set and 0 returned, and
// the caller recomputes the query with the full predicates.
//   edge (v0, v1): det[v0-p, v1-v0, d];  (v1, v2): det[v1-p, v2-v1, d];
//   (v2, v0): det[v2-p, v0-v2, d];  orientation det[v0-p, v1-p, v2-p] =
//   det[v0-p, v1-v0, v2-v0] = -det[v0-p, v1-v0, v0-v2].
__device__ __forceinline__ int tri_crossing_fast(float3 v0, float3 v1, float3 v2, float3 p, float3 d, bool &unsure) {
    float3 a = make_float3(v0.x - p.x, v0.y - p.y, v0.z - p.z);
    float3 b = make_float3(v1.x - p.x, v1.y - p.y, v1.z - p.z);
    float3 c = make_float3(v2.x - p.x, v2.y - p.y, v2.z - p.z);
    float3 e0 = make_float3(v1.x - v0.x, v1.y - v0.y, v1.z - v0.z);
    float3 e1 = make_float3(v2.x - v1.x, v2.y - v1.y, v2.z - v1.z);
    float3 e2 = make_float3(v0.x - v2.x, v0.y - v2.y, v0.z - v2.z);
    int s0 = edge_sign_f32(a, e0, d), s1 = edge_sign_f32(b, e1, d), s2 = edge_sign_f32(c, e2, d);
    if (s0 * s1 < 0 || s1 * s2 < 0 || s0 * s2 < 0) return 0;
    if (s0 == 0 || s1 == 0 || s2 == 0) { unsure = true; return 0; }
    int o = -det3_sign_f32(a, e0, e2);
    if (o == 0) { unsure = true; return 0; }
    return o == s0 ? s0 : 0;
}

// Signed crossing of the ray p + t d_eps (t > 0) with triangle (v0, v1, v2):
// +-1 when the three perturbed edge signs agree (their sum is d . n) and the
// origin is on the same side of the plane (t > 0); 0 otherwise (including p
// in the triangle's plane).
__device__ __forceinline__ int tri_crossing(float3 v0, float3 v1, float3 v2, float3 p, float3 d,
                                            unsigned long long *cnt, int *status) {
    float3 a = make_float3(v0.x - p.x, v0.y - p.y, v0.z - p.z);
    float3 b = make_float3(v1.x - p.x, v1.y - p.y, v1.z - p.z);
    float3 c = make_float3(v2.x - p.x, v2.y - p.y, v2.z - p.z);
    int s0 = edge_sign(a, b, v0, v1, p, d, cnt, status);
    if (s0 == 0) return 0;
    int s1 = edge_sign(b, c, v1, v2, p, d, cnt, status);
    if (s1 != s0) return 0;
    int s2 = edge_sign(c, a, v2, v0, p, d, cnt, status);
    if (s2 != s0) return 0;
    int o = orient_sign(a, b, c, v0, v1, v2, p, cnt, status);
    return o == s0 ? s0 : 0;
}

}  // namespace gwn
