// patches.cu -- one-shot winding numbers of surfaces made of bicubic Bezier
// patches (parametric surfaces), without discretising the surface.
//
//   w(p) = chi_d(p) + (1/4pi) sum_{boundary edges A->B} Omega(A - p, B - p, -d)
//
// The boundary term is taken over a polyline sampling of the surface's
// boundary curves (the patch edge curves that no other patch cancels), as
// the paper does for parametric surfaces (Sec. Implementation Details: only
// the boundary is discretised, which changes w slightly near the boundary);
// it runs in the mesh boundary-term kernel.
//
// Crossing count without root finding.  In the frame of d a ray is a point of
// the projection plane (the query's (e1.p, e2.p)) plus the depths > dh.p.  A
// patch (or sub-patch) whose control points all lie in front of p (depth >
// dh.p) is crossed by the ray with the signed multiplicity of the projected
// map at that point, i.e. its Brouwer degree, which equals the winding number
// of the projected boundary of the (sub-)patch around the point (degree
// theory: the signed count of preimages of a regular value of a map from a
// disk is the winding number of the image of the disk's boundary).  A patch
// whose control points all lie behind p, or whose projected control net
// misses the point, contributes nothing (convex hull).  A patch straddling
// the plane through p normal to d is split at u = v = 1/2 and its quarters
// are treated the same way; a quarter can keep straddling only while p is
// within its size of the surface, so the depth is bounded by
// log2(patch size / distance to the surface), capped at PATCH_MAXL (a query
// closer than that is on the surface, where w is undefined; it is counted in
// a status counter).  This replaces the paper's multi-start Newton search for
// all ray/patch roots, which can miss one of two nearby roots of a ray that
// grazes the surface.
//
// Winding numbers: the signed crossings of the half-line {y = 0, x > 0} (in
// coordinates relative to the query point) with each of the four boundary
// curves, counterclockwise in (u, v): each cubic is split at the roots of
// dy/ds into y-monotone pieces, a piece with end values y0, y1 is crossed iff
// min(y0, y1) <= 0 < max(y0, y1) (half-open), and the crossing counts when
// its x (bisection on the piece) is > 0, +1 upward.  A curve is always
// evaluated in a canonical orientation (its end points ordered), so the edge
// shared by two patches, or by two quarters of one split, gives exactly
// opposite counts on its two sides.  The frame satisfies e1 x e2 = -dh, so the
// crossing count chi (+1 where d . (f_u x f_v) > 0) is minus the winding
// number in the (e1, e2) plane.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <memory>
#include <new>
#include <vector>

#include "gwn_internal.h"
#include "predicates.cuh"
#include "query.cuh"

namespace gwn {

#define PATCH_MAXL 20      // maximal subdivision depth of a straddling patch
#define PATCH_STACK 64     // depth-first: at most 3 pending quarters per level

// ---- device ------------------------------------------------------------------

// signed crossings of the half-line {y = 0, x > 0} with the cubic Bezier
// (x[k], y[k]) in the given orientation (canonicalised by the caller); their
// parameters and signs go to sl / gl when given (at most three)
__device__ int cubic_crossings(const float *x, const float *y, float *sl = nullptr, int *gl = nullptr,
                               int *nl = nullptr) {
    float ymin = fminf(fminf(y[0], y[1]), fminf(y[2], y[3])), ymax = fmaxf(fmaxf(y[0], y[1]), fmaxf(y[2], y[3]));
    if (ymin > 0.f || ymax <= 0.f) return 0;
    if (fmaxf(fmaxf(x[0], x[1]), fmaxf(x[2], x[3])) <= 0.f) return 0;
    // dy/ds = 3 [d0 (1-s)^2 + 2 d1 s (1-s) + d2 s^2] = 3 (A s^2 + B s + C)
    const float d0 = y[1] - y[0], d1 = y[2] - y[1], d2 = y[3] - y[2];
    const float A = d0 - 2.f * d1 + d2, B = 2.f * (d1 - d0), C = d0;
    float cut[4];
    int nc = 0;
    cut[nc++] = 0.f;
    float r0 = 2.f, r1 = 2.f;
    const float scale = fabsf(A) + fabsf(B) + fabsf(C);
    if (scale > 0.f) {
        if (fabsf(A) <= 1e-7f * scale) {
            if (B != 0.f) r0 = -C / B;
        } else {
            const float disc = B * B - 4.f * A * C;
            if (disc > 0.f) {
                const float sq = sqrtf(disc);
                const float qq = -0.5f * (B + (B >= 0.f ? sq : -sq));
                r0 = qq / A;
                if (qq != 0.f) r1 = C / qq;
            }
        }
    }
    if (r0 > r1) { float t = r0; r0 = r1; r1 = t; }
    if (r0 > 0.f && r0 < 1.f) cut[nc++] = r0;
    if (r1 > 0.f && r1 < 1.f && r1 > cut[nc - 1]) cut[nc++] = r1;
    cut[nc++] = 1.f;
    auto ev = [&](const float *c, float s) {
        const float v = 1.f - s;
        return v * v * v * c[0] + 3.f * s * v * v * c[1] + 3.f * s * s * v * c[2] + s * s * s * c[3];
    };
    int count = 0;
    float ya = y[0];
    for (int k = 0; k + 1 < nc; k++) {
        const float sb = cut[k + 1];
        const float yb = k + 2 == nc ? y[3] : ev(y, sb);
        const bool up = ya <= 0.f && 0.f < yb, down = yb <= 0.f && 0.f < ya;
        if (up || down) {
            // the root of y on the monotone piece: Newton from the linear
            // guess, kept inside the bracket y(lo) <= 0 < y(hi) (bisection
            // when a step leaves it); the side decision x(s) > 0 needs the
            // root only to the accuracy of the curve itself
            float lo = up ? cut[k] : sb, hi = up ? sb : cut[k];
            const float yl = up ? ya : yb, yh = up ? yb : ya;
            float sr = lo + (hi - lo) * __fdividef(-yl, yh - yl);
            for (int it = 0; it < 40; it++) {
                const float g = ev(y, sr);
                if (g <= 0.f) lo = sr; else hi = sr;
                const float v = 1.f - sr;
                const float dg = 3.f * (v * v * (y[1] - y[0]) + 2.f * sr * v * (y[2] - y[1]) + sr * sr * (y[3] - y[2]));
                float sn = sr - __fdividef(g, dg);
                const float mn = fminf(lo, hi), mx = fmaxf(lo, hi);
                if (!(sn > mn && sn < mx)) sn = 0.5f * (lo + hi);
                const float step = fabsf(sn - sr);
                sr = sn;
                if (step <= 1e-7f || mx - mn <= 1e-7f) break;
            }
            if (ev(x, sr) > 0.f) {
                count += up ? 1 : -1;
                if (sl && *nl < 3) { sl[*nl] = sr; gl[*nl] = up ? 1 : -1; (*nl)++; }
            }
        }
        ya = yb;
    }
    return count;
}

// the same in canonical orientation: a curve and its reverse give exactly
// opposite counts
__device__ __forceinline__ bool canon_reversed(float x0, float y0, float x1, float y1, float x2, float y2, float x3,
                                               float y3) {
    return x3 < x0 || (x3 == x0 && (y3 < y0 || (y3 == y0 && (x2 < x1 || (x2 == x1 && y2 < y1)))));
}
__device__ __forceinline__ int curve_crossings(float x0, float y0, float x1, float y1, float x2, float y2, float x3,
                                               float y3) {
    const bool rev = canon_reversed(x0, y0, x1, y1, x2, y2, x3, y3);
    float x[4], y[4];
    if (rev) {
        x[0] = x3; x[1] = x2; x[2] = x1; x[3] = x0;
        y[0] = y3; y[1] = y2; y[2] = y1; y[3] = y0;
    } else {
        x[0] = x0; x[1] = x1; x[2] = x2; x[3] = x3;
        y[0] = y0; y[1] = y1; y[2] = y2; y[3] = y3;
    }
    const int c = cubic_crossings(x, y);
    return rev ? -c : c;
}

// winding number around the origin of the projected boundary of the net
// (X, Y)[i * 4 + j], counterclockwise in (u, v)
__device__ int net_winding(const float *X, const float *Y) {
#define NI(i, j) ((i) * 4 + (j))
    int w = 0;
    w += curve_crossings(X[NI(0, 0)], Y[NI(0, 0)], X[NI(1, 0)], Y[NI(1, 0)], X[NI(2, 0)], Y[NI(2, 0)], X[NI(3, 0)],
                         Y[NI(3, 0)]);
    w += curve_crossings(X[NI(3, 0)], Y[NI(3, 0)], X[NI(3, 1)], Y[NI(3, 1)], X[NI(3, 2)], Y[NI(3, 2)], X[NI(3, 3)],
                         Y[NI(3, 3)]);
    w += curve_crossings(X[NI(3, 3)], Y[NI(3, 3)], X[NI(2, 3)], Y[NI(2, 3)], X[NI(1, 3)], Y[NI(1, 3)], X[NI(0, 3)],
                         Y[NI(0, 3)]);
    w += curve_crossings(X[NI(0, 3)], Y[NI(0, 3)], X[NI(0, 2)], Y[NI(0, 2)], X[NI(0, 1)], Y[NI(0, 1)], X[NI(0, 0)],
                         Y[NI(0, 0)]);
#undef NI
    return w;
}

// keep the half `hi` (0: [0, 1/2], 1: [1/2, 1]) of the cubic c[0], c[s], c[2s], c[3s]
__device__ __forceinline__ void halve(float *c, int s, int hi) {
    const float p0 = c[0], p1 = c[s], p2 = c[2 * s], p3 = c[3 * s];
    const float a = 0.5f * (p0 + p1), b = 0.5f * (p1 + p2), e = 0.5f * (p2 + p3);
    const float f = 0.5f * (a + b), g = 0.5f * (b + e), m = 0.5f * (f + g);
    if (hi) { c[0] = m; c[s] = g; c[2 * s] = e; }
    else { c[s] = a; c[2 * s] = f; c[3 * s] = m; }
}

// the net of the sub-patch (level, iu, iv) replayed from the root by the
// sequence of halvings that leads to it (identical for the shared edges of
// siblings)
__device__ void subnet(const float *R, int level, int iu, int iv, float *N) {
    for (int k = 0; k < 16; k++) N[k] = R[k];
    for (int l = level - 1; l >= 0; l--) {
        const int bu = (iu >> l) & 1, bv = (iv >> l) & 1;
        for (int j = 0; j < 4; j++) halve(N + j, 4, bu);       // rows: u is the first index
        for (int i = 0; i < 4; i++) halve(N + 4 * i, 1, bv);
    }
}

// winding count of a patch cut by the plane through the query (out of line:
// rare, and kept out of the hot loop's instruction footprint)
__device__ __noinline__ int patch_winding_straddling(const float *X, const float *Y, const float *Z, bool *near);

// signed crossing count (winding convention) of one patch with the ray of the
// query at the origin of (X, Y, Z); *near set when a straddling quarter
// reached PATCH_MAXL
__device__ __forceinline__ int patch_winding(const float *X, const float *Y, const float *Z, bool *near) {
    float zmin = Z[0], zmax = Z[0];
    for (int k = 1; k < 16; k++) { zmin = fminf(zmin, Z[k]); zmax = fmaxf(zmax, Z[k]); }
    if (zmax <= 0.f) return 0;
    if (zmin > 0.f) return net_winding(X, Y);
    return patch_winding_straddling(X, Y, Z, near);
}

__device__ __noinline__ int patch_winding_straddling(const float *X, const float *Y, const float *Z, bool *near) {
    // depth-first over quarters (level, iu, iv) packed as
    // level << 48 | iu << 24 | iv
    long long stack[PATCH_STACK];
    int sp = 0, total = 0;
    for (int c = 0; c < 4; c++) stack[sp++] = (1ll << 48) | ((long long)(c & 1) << 24) | (c >> 1);
    float NX[16], NY[16], NZ[16];
    int guard = 0;
    while (sp > 0 && guard++ < 4096) {
        const long long code = stack[--sp];
        const int level = (int)(code >> 48), iu = (int)((code >> 24) & 0xffffff), iv = (int)(code & 0xffffff);
        subnet(X, level, iu, iv, NX);
        subnet(Y, level, iu, iv, NY);
        float xn = NX[0], xx = NX[0], yn = NY[0], yx = NY[0];
        for (int k = 1; k < 16; k++) {
            xn = fminf(xn, NX[k]); xx = fmaxf(xx, NX[k]);
            yn = fminf(yn, NY[k]); yx = fmaxf(yx, NY[k]);
        }
        if (xn > 0.f || xx < 0.f || yn > 0.f || yx < 0.f) continue;   // the net misses the ray
        subnet(Z, level, iu, iv, NZ);
        float zn = NZ[0], zx = NZ[0];
        for (int k = 1; k < 16; k++) { zn = fminf(zn, NZ[k]); zx = fmaxf(zx, NZ[k]); }
        if (zx <= 0.f) continue;                                       // behind
        if (zn > 0.f) { total += net_winding(NX, NY); continue; }      // in front
        if (level >= PATCH_MAXL || sp + 4 > PATCH_STACK) { *near = true; continue; }
        for (int c = 0; c < 4; c++)
            stack[sp++] = ((long long)(level + 1) << 48) | ((long long)(2 * iu + (c & 1)) << 24) |
                          (long long)(2 * iv + (c >> 1));
    }
    if (sp > 0) *near = true;
    return total;
}

// Boundary correction of one patch edge that lies on the surface boundary.
// The boundary term runs over the sampled boundary (chords v_k -> v_{k+1} of
// the edge curve), so the crossing count must be that of the surface whose
// boundary is the polyline: the patch edge's curve crossings are replaced by
// the chords' crossings.  The two differ only for a ray inside the thin
// region between a chord and its arc; per chord k that difference counts when
// the region lies in front of the query, is dropped behind it, and marks the
// query as on the surface when the region straddles it (depth range of the
// chord's ends widened by a host bound on the arc's distance from the chord).
// Curve crossings come from the same canonical evaluation as the winding
// number, attributed to chords by their parameter; a chord crossing takes its
// side from the exact sign of det[v_k - p, v_{k+1} - p, d], the predicate the
// boundary term uses for its branch, so chi and B jump together.
// ex, ey: the edge's control points in the patch's edge order (relative to
// the query); pv: the curve's projected samples (canonical order); xv: the
// same samples in 3D; dev: per chord arc-chord bound; against: the patch edge
// runs against the canonical order.
__device__ __noinline__ int boundary_edge_correction(const float *ex, const float *ey, const float4 *__restrict__ pv,
                                        const float4 *__restrict__ xv, const float *__restrict__ dev, int K,
                                        bool against, float qb, float qc, float3 P, float3 D,
                                        unsigned long long *cnt, int *status, bool *near) {
    // the half-line y = 0, x > 0 misses the edge's control hull (which holds
    // the arc and its chords): nothing to replace
    if (fminf(fminf(ey[0], ey[1]), fminf(ey[2], ey[3])) > 0.f || fmaxf(fmaxf(ey[0], ey[1]), fmaxf(ey[2], ey[3])) < 0.f ||
        fmaxf(fmaxf(ex[0], ex[1]), fmaxf(ex[2], ex[3])) < 0.f)
        return 0;
    // curve crossings (as the winding number evaluates them), in the canonical sample order
    const bool rev = canon_reversed(ex[0], ey[0], ex[1], ey[1], ex[2], ey[2], ex[3], ey[3]);
    float x[4], y[4];
    for (int k = 0; k < 4; k++) { x[k] = rev ? ex[3 - k] : ex[k]; y[k] = rev ? ey[3 - k] : ey[k]; }
    float sl[3];
    int gl[3], nl = 0;
    cubic_crossings(x, y, sl, gl, &nl);
    const bool flip = rev != against;          // device-canonical order against the sample order
    int corr = 0;
    float yk = __ldg(&pv[0]).y - qb;
    for (int k = 0; k < K; k++) {
        const float4 v0 = __ldg(&pv[k]), v1 = __ldg(&pv[k + 1]);
        const float yk1 = v1.y - qb;
        int d = 0;
        if (yk <= 0.f && 0.f < yk1) {              // upward chord: crossing right of q iff det[a, b, d] < 0
            const float4 A = __ldg(&xv[k]), B = __ldg(&xv[k + 1]);
            const float3 Af = make_float3(A.x, A.y, A.z), Bf = make_float3(B.x, B.y, B.z);
            const float3 a = make_float3(A.x - P.x, A.y - P.y, A.z - P.z), b = make_float3(B.x - P.x, B.y - P.y, B.z - P.z);
            if (edge_sign(a, b, Af, Bf, P, D, cnt, status) < 0) d += 1;
        } else if (yk1 <= 0.f && 0.f < yk) {       // downward chord: iff det[a, b, d] > 0
            const float4 A = __ldg(&xv[k]), B = __ldg(&xv[k + 1]);
            const float3 Af = make_float3(A.x, A.y, A.z), Bf = make_float3(B.x, B.y, B.z);
            const float3 a = make_float3(A.x - P.x, A.y - P.y, A.z - P.z), b = make_float3(B.x - P.x, B.y - P.y, B.z - P.z);
            if (edge_sign(a, b, Af, Bf, P, D, cnt, status) > 0) d -= 1;
        }
        for (int j = 0; j < nl; j++) {             // arc crossings attributed to this chord
            const float sh = flip ? 1.f - sl[j] : sl[j];
            int kk = (int)(sh * (float)K);
            kk = kk < 0 ? 0 : (kk >= K ? K - 1 : kk);
            if (kk == k) d -= flip ? -gl[j] : gl[j];
        }
        if (d) {
            const float z0 = v0.z - qc, z1 = v1.z - qc, dv = __ldg(&dev[k]);
            const float zlo = fminf(z0, z1) - dv, zhi = fmaxf(z0, z1) + dv;
            if (zlo > 0.f) corr += d;
            else if (!(zhi <= 0.f)) *near = true;
        }
        yk = yk1;
    }
    return against ? -corr : corr;
}

// The signed winding count of patch t seen from a query at the origin of
// (X, Y, Z) (its control net relative to the query's frame coordinates),
// with the boundary-edge corrections of its edges on the surface boundary.
__device__ __forceinline__ int patch_pair_winding(int t, const float *X, const float *Y, const float *Z,
                                                  const int32_t *__restrict__ bedge,
                                                  const float4 *__restrict__ pl_proj,
                                                  const float4 *__restrict__ pl_xyz, const float *__restrict__ pl_dev,
                                                  int K, const Frame &fr, float qb, float qc, float3 qp,
                                                  unsigned long long *cnt, int *status, bool *near) {
    int wn = patch_winding(X, Y, Z, near);
    if (bedge) {
        // edges on the surface boundary: chords instead of the curve
        static const int EIDX[4][4] = {{0, 4, 8, 12}, {12, 13, 14, 15}, {15, 11, 7, 3}, {3, 2, 1, 0}};
        const int4 be = *(const int4 *)&bedge[4 * (int64_t)t];
        const int codes[4] = {be.x, be.y, be.z, be.w};
        for (int e = 0; e < 4; e++) {
            if (codes[e] < 0) continue;
            float ex[4], ey[4];
            for (int m2 = 0; m2 < 4; m2++) { ex[m2] = X[EIDX[e][m2]]; ey[m2] = Y[EIDX[e][m2]]; }
            const int cv = codes[e] >> 1;
            const int64_t o = (int64_t)cv * (K + 1);
            wn += boundary_edge_correction(ex, ey, pl_proj + o, pl_xyz + o, pl_dev + (int64_t)cv * K, K,
                                           (codes[e] & 1) != 0, qb, qc, qp, make_float3(fr.d[0], fr.d[1], fr.d[2]),
                                           cnt, status, near);
        }
    }
    return wn;
}

// One ray per thread, with the (ray, patch) work compacted per warp: each
// lane walks the patches listed in its bin cell and keeps those whose
// projected box holds its ray and that reach in front of it; the kept pairs
// go to a per-warp buffer, and whenever 32 are pending every lane takes one
// (the ray's coordinates fetched from its lane by a shuffle) and adds the
// patch's winding number to that ray's total in shared memory.  The winding
// computation is long and most rays meet no patch, so this keeps the lanes
// busy instead of one lane per warp.  A pair whose patch straddles the plane
// through the query (subdivision) or has edges on the surface boundary
// (chord corrections) is long and rare: it goes to a list (dpairs, up to
// dcap) for chi_patches_deferred_kernel, so that one such lane does not hold
// the other 31 of its warp; the kernel writes chi without those pairs.
__global__ void __launch_bounds__(128) chi_patches_kernel(const float4 *__restrict__ qnet,
                                                          const float4 *__restrict__ box,
                                                          const float *__restrict__ zmax,
                                                          const int32_t *__restrict__ bin_off,
                                                          const int32_t *__restrict__ bin_idx, int nbx, int nby,
                                                          float bx0, float by0, float binv,
                                                          const int32_t *__restrict__ bedge,
                                                          const float4 *__restrict__ pl_proj,
                                                          const float4 *__restrict__ pl_xyz,
                                                          const float *__restrict__ pl_dev, int K, Frame fr,
                                                          QuerySrc q, int32_t *__restrict__ chi,
                                                          unsigned long long *cnt, int *status, int2 *dpairs,
                                                          int32_t *dcount, int dcap) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < q.n;
    float a = 0.f, b = 0.f, c = 0.f;
    float3 p = make_float3(0.f, 0.f, 0.f);
    int k0 = 0, k1 = 0;
    if (valid) {
        p = query_point3(q, i);
        a = fmaf(p.z, fr.e1[2], fmaf(p.y, fr.e1[1], p.x * fr.e1[0]));
        b = fmaf(p.z, fr.e2[2], fmaf(p.y, fr.e2[1], p.x * fr.e2[0]));
        c = fmaf(p.z, fr.dh[2], fmaf(p.y, fr.dh[1], p.x * fr.dh[0]));
        const float fx = (a - bx0) * binv, fy = (b - by0) * binv;
        if (fx >= 0.f && fy >= 0.f && fx < (float)nbx && fy < (float)nby) {
            const int cell = (int)fy * nbx + (int)fx;
            k0 = bin_off[cell];
            k1 = bin_off[cell + 1];
        }
    }
    __shared__ int s_pair[128 / 32][64];
    __shared__ int s_acc[128 / 32][32];
    __shared__ unsigned s_near[128 / 32];
    int *pairs = s_pair[w];
    s_acc[w][lane] = 0;
    if (lane == 0) s_near[w] = 0u;
    __syncwarp();
    int npairs = 0, tests = 0;
    // process the first min(n, 32) pending pairs, one per lane; returns how many remain
    auto flush = [&](int n) -> int {
        const int m = n < 32 ? n : 32;
        const int pr = lane < m ? pairs[lane] : -1;
        const int ql = pr >= 0 ? (pr & 31) : lane;
        const float qa = __shfl_sync(FULL, a, ql), qb = __shfl_sync(FULL, b, ql), qc = __shfl_sync(FULL, c, ql);
        const float3 qp = make_float3(__shfl_sync(FULL, p.x, ql), __shfl_sync(FULL, p.y, ql),
                                      __shfl_sync(FULL, p.z, ql));
        const int qi = __shfl_sync(FULL, (int)i, ql);
        if (pr >= 0) {
            const int t = pr >> 5;
            float X[16], Y[16], Z[16];
            float zmin = 3.4e38f, zmax = -3.4e38f;
#pragma unroll
            for (int m2 = 0; m2 < 16; m2++) {
                const float4 v = __ldg(&qnet[16 * (int64_t)t + m2]);
                X[m2] = v.x - qa;
                Y[m2] = v.y - qb;
                Z[m2] = v.z - qc;
                zmin = fminf(zmin, Z[m2]);
                zmax = fmaxf(zmax, Z[m2]);
            }
            bool defer = false;
            if (dpairs && zmax > 0.f) {
                bool edge = false;
                if (bedge) {
                    const int4 be = *(const int4 *)&bedge[4 * (int64_t)t];
                    edge = be.x >= 0 || be.y >= 0 || be.z >= 0 || be.w >= 0;
                }
                if (!(zmin > 0.f) || edge) {                  // straddling, or boundary edges
                    const int slot = atomicAdd(dcount, 1);
                    if (slot < dcap) {
                        dpairs[slot] = make_int2(qi, t);
                        defer = true;
                    }
                }
            }
            if (!defer) {
                bool near = false;
                const int wn = patch_pair_winding(t, X, Y, Z, bedge, pl_proj, pl_xyz, pl_dev, K, fr, qb, qc, qp, cnt,
                                                  status, &near);
                if (wn) atomicAdd(&s_acc[w][ql], wn);
                if (near) atomicOr(&s_near[w], 1u << ql);
            }
        }
        const int rem = n - m;
        __syncwarp();
        const int moved = lane < rem ? pairs[m + lane] : 0;
        __syncwarp();
        if (lane < rem) pairs[lane] = moved;
        __syncwarp();
        return rem;
    };
    // all lanes step through their own candidate lists together
    for (int k = k0;; k++) {
        const bool more = k < k1;
        if (!__any_sync(FULL, more)) break;
        bool keep = false;
        int t = 0;
        if (more) {
            t = bin_idx[k];
            const float4 bb = __ldg(&box[t]);
            keep = !(a < bb.x || a > bb.y || b < bb.z || b > bb.w) && __ldg(&zmax[t]) > c;
        }
        const unsigned mk = __ballot_sync(FULL, keep);
        if (mk) {
            if (keep) pairs[npairs + __popc(mk & ((1u << lane) - 1u))] = (t << 5) | lane;
            npairs += __popc(mk);
            tests += keep;
            __syncwarp();
            if (npairs >= 32) npairs = flush(npairs);
        }
    }
    while (npairs > 0) npairs = flush(npairs);
    __syncwarp();
    const bool near = (s_near[w] >> lane) & 1u;
    if (valid) chi[i] = -s_acc[w][lane];          // e1 x e2 = -dh
    if (cnt) {
        if (tests) atomicAdd(&cnt[CNT_TRI_TESTS], (unsigned long long)tests);
        if (valid && near) atomicAdd(&cnt[CNT_STACK_OVERFLOW], 1ull);
    }
}

// The pairs chi_patches_kernel listed, one per thread: their winding counts
// subtracted from chi (the kernel stores minus the sum: e1 x e2 = -dh).
__global__ void __launch_bounds__(128) chi_patches_deferred_kernel(
    const int2 *__restrict__ dpairs, const int32_t *__restrict__ dcount, int dcap, const float4 *__restrict__ qnet,
    const int32_t *__restrict__ bedge, const float4 *__restrict__ pl_proj, const float4 *__restrict__ pl_xyz,
    const float *__restrict__ pl_dev, int K, Frame fr, QuerySrc q, int32_t *__restrict__ chi,
    unsigned long long *cnt, int *status) {
    int n = *dcount;
    if (n > dcap) n = dcap;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int2 pr = dpairs[k];
        const int64_t i = pr.x;
        const int t = pr.y;
        const float3 p = query_point3(q, i);
        const float a = fmaf(p.z, fr.e1[2], fmaf(p.y, fr.e1[1], p.x * fr.e1[0]));
        const float b = fmaf(p.z, fr.e2[2], fmaf(p.y, fr.e2[1], p.x * fr.e2[0]));
        const float c = fmaf(p.z, fr.dh[2], fmaf(p.y, fr.dh[1], p.x * fr.dh[0]));
        float X[16], Y[16], Z[16];
        for (int m2 = 0; m2 < 16; m2++) {
            const float4 v = __ldg(&qnet[16 * (int64_t)t + m2]);
            X[m2] = v.x - a;
            Y[m2] = v.y - b;
            Z[m2] = v.z - c;
        }
        bool near = false;
        const int wn = patch_pair_winding(t, X, Y, Z, bedge, pl_proj, pl_xyz, pl_dev, K, fr, b, c, p, cnt, status,
                                          &near);
        if (wn) atomicAdd(&chi[i], -wn);
        if (near && cnt) atomicAdd(&cnt[CNT_STACK_OVERFLOW], 1ull);
    }
}

cudaError_t launch_chi_patches(const PatchSet &ps, const QuerySrc &q, int32_t *chi, unsigned long long *cnt,
                               int *status, cudaStream_t st, int2 *dpairs, int32_t *dcount, int dcap,
                               int sm_count) {
    if (q.n == 0) return cudaSuccess;
    const int64_t blocks = (q.n + 127) / 128;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    const bool deferred = dpairs && dcount && dcap > 0 && q.n <= 0x7fffffff;
    if (deferred) {
        cudaError_t e = cudaMemsetAsync(dcount, 0, sizeof(int32_t), st);
        if (e != cudaSuccess) return e;
    }
    chi_patches_kernel<<<(unsigned)blocks, 128, 0, st>>>(ps.qnet, ps.box, ps.zmax, ps.bin_off, ps.bin_idx, ps.nbx,
                                                         ps.nby, ps.bx0, ps.by0, ps.binv,
                                                         ps.n_bcurves ? ps.bedge : nullptr, ps.pl_proj, ps.pl_xyz,
                                                         ps.pl_dev, ps.segments, ps.frame, q, chi, cnt, status,
                                                         deferred ? dpairs : nullptr, dcount, dcap);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !deferred) return e;
    chi_patches_deferred_kernel<<<(unsigned)((sm_count > 0 ? sm_count : 152) * 8), 128, 0, st>>>(
        dpairs, dcount, dcap, ps.qnet, ps.n_bcurves ? ps.bedge : nullptr, ps.pl_proj, ps.pl_xyz, ps.pl_dev,
        ps.segments, ps.frame, q, chi, cnt, status);
    return cudaGetLastError();
}

// ---- host ----------------------------------------------------------------------

// the per-direction tables
static void patches_free_dir(PatchSet &ps) {
    if (ps.pl_proj) cudaFree(ps.pl_proj);
    ps.pl_proj = nullptr;
    if (ps.bframe) cudaFree(ps.bframe);
    if (ps.qnet) cudaFree(ps.qnet);
    if (ps.box) cudaFree(ps.box);
    if (ps.zmax) cudaFree(ps.zmax);
    if (ps.bin_off) cudaFree(ps.bin_off);
    if (ps.bin_idx) cudaFree(ps.bin_idx);
    ps.bframe = nullptr; ps.qnet = nullptr; ps.box = nullptr; ps.zmax = nullptr;
    ps.bin_off = nullptr; ps.bin_idx = nullptr;
    ps.valid = false;
}

void patches_free(PatchSet &ps) {
    patches_free_dir(ps);
    if (ps.bedge) cudaFree(ps.bedge);
    if (ps.pl_xyz) cudaFree(ps.pl_xyz);
    if (ps.pl_dev) cudaFree(ps.pl_dev);
    ps.bedge = nullptr; ps.pl_xyz = nullptr; ps.pl_dev = nullptr;
}

gwn_status patches_prepare(gwn_geom *g, const float d[3]) {
    PatchSet &ps = g->ps;
    if (!isfinite(d[0]) || !isfinite(d[1]) || !isfinite(d[2]) || (d[0] == 0.f && d[1] == 0.f && d[2] == 0.f)) {
        set_error("patches: direction must be finite and nonzero");
        return GWN_E_INVALID;
    }
    if (ps.valid && memcmp(ps.dkey, d, sizeof(float) * 3) == 0) return GWN_OK;
    patches_free_dir(ps);
    const Frame fr = make_frame(d);
    const int64_t n = ps.n;
    // projected control nets (float64 dot products rounded once) and boxes
    std::vector<float4> qn(16 * std::max<int64_t>(n, 1)), bx(std::max<int64_t>(n, 1));
    std::vector<float> zm(std::max<int64_t>(n, 1));
    double gx0 = INFINITY, gx1 = -INFINITY, gy0 = INFINITY, gy1 = -INFINITY;
    for (int64_t t = 0; t < n; t++) {
        float xn = INFINITY, xx = -INFINITY, yn = INFINITY, yx = -INFINITY, zx = -INFINITY;
        for (int m = 0; m < 16; m++) {
            const float *P = &ps.h_ctrl[48 * t + 3 * m];
            double v[3];
            const float *e[3] = {fr.e1, fr.e2, fr.dh};
            for (int c = 0; c < 3; c++) v[c] = (double)P[0] * e[c][0] + (double)P[1] * e[c][1] + (double)P[2] * e[c][2];
            const float4 f = make_float4((float)v[0], (float)v[1], (float)v[2], 0.f);
            qn[16 * t + m] = f;
            xn = fminf(xn, f.x); xx = fmaxf(xx, f.x); yn = fminf(yn, f.y); yx = fmaxf(yx, f.y); zx = fmaxf(zx, f.z);
        }
        bx[t] = make_float4(xn, xx, yn, yx);
        zm[t] = zx;
        gx0 = std::min(gx0, (double)xn); gx1 = std::max(gx1, (double)xx);
        gy0 = std::min(gy0, (double)yn); gy1 = std::max(gy1, (double)yx);
    }
    // bins: about four cells per patch, each patch listed in the cells its
    // box (widened by a cell fraction against rounding of the cell map) meets
    int nb = 1;
    if (n > 0) nb = (int)std::min<double>(1024.0, std::max(1.0, ceil(2.0 * sqrt((double)n))));
    double W = n > 0 ? std::max(gx1 - gx0, gy1 - gy0) : 1.0;
    if (!(W > 0.0)) W = 1.0;
    const double cell = W * (1.0 + 1e-6) / nb;
    ps.bx0 = n > 0 ? (float)(gx0 - 1e-3 * cell) : 0.f;
    ps.by0 = n > 0 ? (float)(gy0 - 1e-3 * cell) : 0.f;
    ps.binv = (float)(1.0 / cell);
    ps.nbx = nb + 1;
    ps.nby = nb + 1;
    std::vector<int32_t> cnt((size_t)ps.nbx * ps.nby + 1, 0);
    std::vector<int> c0(std::max<int64_t>(n, 1)), c1(std::max<int64_t>(n, 1)), r0(std::max<int64_t>(n, 1)),
        r1(std::max<int64_t>(n, 1));
    for (int64_t t = 0; t < n; t++) {
        auto clampi = [](double v, int hi) { return (int)std::max(0.0, std::min((double)hi, floor(v))); };
        c0[t] = clampi((bx[t].x - ps.bx0) * ps.binv - 1e-3, ps.nbx - 1);
        c1[t] = clampi((bx[t].y - ps.bx0) * ps.binv + 1e-3, ps.nbx - 1);
        r0[t] = clampi((bx[t].z - ps.by0) * ps.binv - 1e-3, ps.nby - 1);
        r1[t] = clampi((bx[t].w - ps.by0) * ps.binv + 1e-3, ps.nby - 1);
        for (int r = r0[t]; r <= r1[t]; r++)
            for (int c = c0[t]; c <= c1[t]; c++) cnt[(size_t)r * ps.nbx + c + 1]++;
    }
    for (size_t k = 0; k + 1 < cnt.size(); k++) cnt[k + 1] += cnt[k];
    std::vector<int32_t> idx(std::max<int32_t>(cnt.back(), 1));
    {
        std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
        for (int64_t t = 0; t < n; t++)
            for (int r = r0[t]; r <= r1[t]; r++)
                for (int c = c0[t]; c <= c1[t]; c++) idx[fill[(size_t)r * ps.nbx + c]++] = (int32_t)t;
    }
    cudaError_t e = cudaSuccess;
    auto up = [&](void **dst, const void *src, size_t bytes) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(dst, bytes);
        if (e == cudaSuccess) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up((void **)&ps.qnet, qn.data(), sizeof(float4) * qn.size());
    up((void **)&ps.box, bx.data(), sizeof(float4) * bx.size());
    up((void **)&ps.zmax, zm.data(), sizeof(float) * zm.size());
    up((void **)&ps.bin_off, cnt.data(), sizeof(int32_t) * cnt.size());
    up((void **)&ps.bin_idx, idx.data(), sizeof(int32_t) * idx.size());
    if (e == cudaSuccess && !ps.h_pl_xyz.empty()) {       // projected boundary samples
        std::vector<float4> pp(ps.h_pl_xyz.size());
        const float *e3[3] = {fr.e1, fr.e2, fr.dh};
        for (size_t k = 0; k < pp.size(); k++) {
            const float4 v = ps.h_pl_xyz[k];
            double r[3];
            for (int c = 0; c < 3; c++) r[c] = (double)v.x * e3[c][0] + (double)v.y * e3[c][1] + (double)v.z * e3[c][2];
            pp[k] = make_float4((float)r[0], (float)r[1], (float)r[2], 0.f);
        }
        up((void **)&ps.pl_proj, pp.data(), sizeof(float4) * pp.size());
    }
    if (e == cudaSuccess && g->n_bseq > 0) {
        e = cudaMalloc(&ps.bframe, sizeof(float4) * 2 * g->n_bseq);
        if (e == cudaSuccess) e = launch_bframe(g->bseq, g->n_bseq, fr, ps.bframe, g->ctx->stream);
    }
    if (e != cudaSuccess) {
        patches_free_dir(ps);
        return cuda_fail(e, "patch preparation");
    }
    ps.frame = fr;
    memcpy(ps.dkey, d, sizeof(float) * 3);
    ps.valid = true;
    return GWN_OK;
}

}  // namespace gwn

using namespace gwn;

#define CK(call, what)                                     \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Boundary of a patch set: each patch contributes its four edge curves along
// the counterclockwise boundary of the (u, v) square; a curve and its reverse
// cancel (net multiplicity over canonical keys, the twelve float32 bit
// patterns of the curve in its smaller orientation); a curve of net
// multiplicity m != 0 is sampled at `segments` intervals (float64 Bernstein
// values rounded to float32; its end points are its end control points
// exactly, so curves meeting at a corner share that vertex), and the unit
// edges are chained into loops.
extern "C" GWN_API gwn_status gwn_patches_create(gwn_ctx *ctx, const float *ctrl, int64_t n_patches, int segments,
                                                 int mem_kind, gwn_geom **out) {
    if (!out) { set_error("gwn_patches_create: out is NULL"); return GWN_E_INVALID; }
    *out = nullptr;
    if (!ctx || n_patches < 0 || (n_patches > 0 && !ctrl) || segments < 1 || segments > 65536 ||
        (mem_kind != GWN_MEM_HOST && mem_kind != GWN_MEM_DEVICE)) {
        set_error("gwn_patches_create: bad arguments");
        return GWN_E_INVALID;
    }
    if (n_patches > (1 << 26)) { set_error("gwn_patches_create: too many patches"); return GWN_E_INVALID; }
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    std::unique_ptr<gwn_geom> g(new (std::nothrow) gwn_geom());
    if (!g) { set_error("gwn_patches_create: out of host memory"); return GWN_E_OOM; }
    g->ctx = ctx;
    g->kind = GWN_GEOM_PATCHES;
    g->dtype = GWN_F32;
    PatchSet &ps = g->ps;
    ps.n = n_patches;
    ps.segments = segments;
    try {
        ps.h_ctrl.resize(48 * (size_t)n_patches);
    } catch (const std::bad_alloc &) {
        set_error("gwn_patches_create: out of host memory");
        return GWN_E_OOM;
    }
    if (n_patches) {
        if (mem_kind == GWN_MEM_HOST) memcpy(ps.h_ctrl.data(), ctrl, sizeof(float) * ps.h_ctrl.size());
        else CK(cudaMemcpy(ps.h_ctrl.data(), ctrl, sizeof(float) * ps.h_ctrl.size(), cudaMemcpyDeviceToHost), "copy ctrl");
    }
    for (float v : ps.h_ctrl)
        if (!isfinite(v)) { set_error("gwn_patches_create: non-finite control point"); return GWN_E_INVALID; }
    // net multiplicity of the edge curves
    typedef std::array<uint32_t, 12> Key;
    std::map<Key, int> net;
    static const int EDGE[4][4][2] = {{{0, 0}, {1, 0}, {2, 0}, {3, 0}},
                                      {{3, 0}, {3, 1}, {3, 2}, {3, 3}},
                                      {{3, 3}, {2, 3}, {1, 3}, {0, 3}},
                                      {{0, 3}, {0, 2}, {0, 1}, {0, 0}}};
    for (int64_t t = 0; t < n_patches; t++)
        for (int e = 0; e < 4; e++) {
            Key fwd, rev;
            for (int k = 0; k < 4; k++) {
                const float *P = &ps.h_ctrl[48 * t + 3 * (4 * EDGE[e][k][0] + EDGE[e][k][1])];
                const float *R = &ps.h_ctrl[48 * t + 3 * (4 * EDGE[e][3 - k][0] + EDGE[e][3 - k][1])];
                for (int c = 0; c < 3; c++) {
                    memcpy(&fwd[3 * k + c], &P[c], 4);
                    memcpy(&rev[3 * k + c], &R[c], 4);
                }
            }
            if (fwd <= rev) net[fwd] += 1;
            else net[rev] -= 1;
        }
    // sample the boundary curves, vertices shared through their bit patterns
    std::map<std::array<uint32_t, 3>, int32_t> vid;
    std::vector<float> hv;
    auto vertex = [&](const float x[3]) {
        std::array<uint32_t, 3> k;
        memcpy(k.data(), x, 12);
        auto it = vid.find(k);
        if (it != vid.end()) return it->second;
        int32_t id = (int32_t)(hv.size() / 3);
        vid[k] = id;
        hv.insert(hv.end(), x, x + 3);
        return id;
    };
    std::vector<std::pair<int32_t, int32_t>> bedges;
    std::map<Key, int32_t> curve_id;             // boundary curves: id in the sample tables
    for (auto &kv : net) {
        const int m = kv.second;
        if (m == 0) continue;
        float c[4][3];
        memcpy(c, kv.first.data(), sizeof(c));
        bool flat = true;
        for (int k = 1; k < 4; k++)
            for (int q = 0; q < 3; q++) flat = flat && c[k][q] == c[0][q];
        if (flat) continue;                       // a collapsed edge bounds nothing
        std::vector<int32_t> ids(segments + 1);
        std::vector<float4> xs(segments + 1);
        for (int s = 0; s <= segments; s++) {
            float x[3];
            if (s == 0 || s == segments) {
                memcpy(x, c[s == 0 ? 0 : 3], sizeof(x));
            } else {
                const double u = (double)s / segments, v = 1.0 - u;
                const double b[4] = {v * v * v, 3 * u * v * v, 3 * u * u * v, u * u * u};
                for (int q = 0; q < 3; q++)
                    x[q] = (float)(b[0] * c[0][q] + b[1] * c[1][q] + b[2] * c[2][q] + b[3] * c[3][q]);
            }
            ids[s] = vertex(x);
            xs[s] = make_float4(x[0], x[1], x[2], 0.f);
        }
        // per chord, a bound on the distance between the arc over [s_k, s_k+1]
        // and the chord: the arc lies in the hull of its own control points
        // (the cubic restricted to the interval), each within the bound of the
        // chord segment; widened for the float32 rounding of the samples
        curve_id[kv.first] = (int32_t)ps.n_bcurves++;
        for (int s = 0; s < segments; s++) {
            const double u0 = (double)s / segments, u1 = (double)(s + 1) / segments;
            double r[4][3];
            for (int q = 0; q < 3; q++) {
                // de Casteljau: split at u0 (right part), then at (u1 - u0) / (1 - u0) (left part)
                double p0 = c[0][q], p1 = c[1][q], p2 = c[2][q], p3 = c[3][q];
                double a = p0 + u0 * (p1 - p0), b = p1 + u0 * (p2 - p1), cc = p2 + u0 * (p3 - p2);
                double d2 = a + u0 * (b - a), e2 = b + u0 * (cc - b), m0 = d2 + u0 * (e2 - d2);
                p0 = m0; p1 = e2; p2 = cc;   // right part [u0, 1]: m0, e2, cc, p3
                const double t = (u1 - u0) / (1.0 - u0);
                a = p0 + t * (p1 - p0); b = p1 + t * (p2 - p1); cc = p2 + t * (p3 - p2);
                d2 = a + t * (b - a); e2 = b + t * (cc - b);
                r[0][q] = p0; r[1][q] = a; r[2][q] = d2; r[3][q] = d2 + t * (e2 - d2);
            }
            const float4 A = xs[s], B = xs[s + 1];
            const double ab[3] = {(double)B.x - A.x, (double)B.y - A.y, (double)B.z - A.z};
            const double L2 = ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2];
            double dmax = 0.0, scale = 0.0;
            for (int k = 0; k < 4; k++) {
                const double w[3] = {r[k][0] - A.x, r[k][1] - A.y, r[k][2] - A.z};
                double tt = L2 > 0.0 ? (w[0] * ab[0] + w[1] * ab[1] + w[2] * ab[2]) / L2 : 0.0;
                tt = tt < 0.0 ? 0.0 : (tt > 1.0 ? 1.0 : tt);
                const double dd[3] = {w[0] - tt * ab[0], w[1] - tt * ab[1], w[2] - tt * ab[2]};
                dmax = std::max(dmax, sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]));
                scale = std::max(scale, fabs(r[k][0]) + fabs(r[k][1]) + fabs(r[k][2]));
            }
            ps.h_pl_dev.push_back((float)(dmax * (1.0 + 1e-3) + 4e-7 * scale));
        }
        ps.h_pl_xyz.insert(ps.h_pl_xyz.end(), xs.begin(), xs.end());
        for (int r = 0; r < (m > 0 ? m : -m); r++)
            for (int s = 0; s < segments; s++) {
                if (ids[s] == ids[s + 1]) continue;
                if (m > 0) bedges.emplace_back(ids[s], ids[s + 1]);
                else bedges.emplace_back(ids[s + 1], ids[s]);
            }
    }
    ps.h_bedge.assign(4 * (size_t)n_patches, -1);
    for (int64_t t = 0; t < n_patches && ps.n_bcurves > 0; t++)
        for (int e = 0; e < 4; e++) {
            Key fwd, rev;
            for (int k = 0; k < 4; k++) {
                const float *P = &ps.h_ctrl[48 * t + 3 * (4 * EDGE[e][k][0] + EDGE[e][k][1])];
                const float *R = &ps.h_ctrl[48 * t + 3 * (4 * EDGE[e][3 - k][0] + EDGE[e][3 - k][1])];
                for (int c = 0; c < 3; c++) {
                    memcpy(&fwd[3 * k + c], &P[c], 4);
                    memcpy(&rev[3 * k + c], &R[c], 4);
                }
            }
            const bool against = !(fwd <= rev);
            auto it = curve_id.find(against ? rev : fwd);
            if (it != curve_id.end()) ps.h_bedge[4 * t + e] = (it->second << 1) | (against ? 1 : 0);
        }
    BoundaryLoops bl;
    gwn_status s = chain_unit_edges(bedges, (int64_t)(hv.size() / 3), bl);
    if (s != GWN_OK) return s;
    g->loop_off = bl.off;
    g->loop_vid = bl.vid;
    std::vector<float4> rec;
    const int64_t L = (int64_t)bl.off.size() - 1;
    for (int64_t j = 0; j < L; j++) {
        const int64_t lo = bl.off[j], hi = bl.off[j + 1];
        for (int64_t i = lo; i <= hi; i++) {
            const int32_t v = bl.vid[i < hi ? i : lo];
            rec.push_back(make_float4(hv[3 * (size_t)v], hv[3 * (size_t)v + 1], hv[3 * (size_t)v + 2], i == lo ? 0.f : 1.f));
        }
    }
    g->n_bseq = (int64_t)rec.size();
    g->nv = (int64_t)(hv.size() / 3);
    cudaError_t e = cudaSuccess;
    auto up = [&](void **dst, const void *src, size_t bytes) {
        if (e != cudaSuccess || bytes == 0) return;
        e = cudaMalloc(dst, bytes);
        if (e == cudaSuccess) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up((void **)&g->bseq, rec.data(), sizeof(float4) * rec.size());
    if (ps.n_bcurves > 0) {
        up((void **)&ps.bedge, ps.h_bedge.data(), sizeof(int32_t) * ps.h_bedge.size());
        up((void **)&ps.pl_xyz, ps.h_pl_xyz.data(), sizeof(float4) * ps.h_pl_xyz.size());
        up((void **)&ps.pl_dev, ps.h_pl_dev.data(), sizeof(float) * ps.h_pl_dev.size());
    }
    if (e != cudaSuccess) {
        if (g->bseq) cudaFree(g->bseq);
        g->bseq = nullptr;
        patches_free(ps);
        return cuda_fail(e, "gwn_patches_create");
    }
    ctx_add_geometry(ctx);
    *out = g.release();
    return GWN_OK;
}
