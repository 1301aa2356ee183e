// patches.cu -- one-shot winding numbers of surfaces made of bicubic Bezier
// patches (parametric surfaces), without discretising the surface.
//
//   w(p) = chi_d(p) + (1/4pi) sum_{boundary edges A->B} Omega(A - p, B - p, -d)
//
// The boundary term is taken over a polyline sampling of the surface's
// boundary curves (the patch edge curves that no other patch cancels), as
// the paper does for parametric surfaces ("we discretize the boundary ...
// this boundary discretization may lead only to minor differences ... close
// to the boundary"); it runs in the mesh boundary-term kernel.
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
#include "query.cuh"

namespace gwn {

#define PATCH_MAXL 20      // maximal subdivision depth of a straddling patch
#define PATCH_STACK 64     // depth-first: at most 3 pending quarters per level

// ---- device ------------------------------------------------------------------

// signed crossings of the half-line {y = 0, x > 0} with the cubic Bezier
// (x[k], y[k]) in the given orientation (canonicalised by the caller)
__device__ int cubic_crossings(const float *x, const float *y) {
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
            // the root of y on [cut[k], sb]: bisection keeping y(lo) <= 0 < y(hi)
            float lo = up ? cut[k] : sb, hi = up ? sb : cut[k];
            for (int it = 0; it < 40; it++) {
                const float mid = 0.5f * (lo + hi);
                if (mid == lo || mid == hi) break;
                if (ev(y, mid) <= 0.f) lo = mid; else hi = mid;
            }
            if (ev(x, 0.5f * (lo + hi)) > 0.f) count += up ? 1 : -1;
        }
        ya = yb;
    }
    return count;
}

// the same in canonical orientation: a curve and its reverse give exactly
// opposite counts
__device__ __forceinline__ int curve_crossings(float x0, float y0, float x1, float y1, float x2, float y2, float x3,
                                               float y3) {
    const bool rev = x3 < x0 || (x3 == x0 && (y3 < y0 || (y3 == y0 && (x2 < x1 || (x2 == x1 && y2 < y1)))));
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

// signed crossing count (winding convention) of one patch with the ray of the
// query at the origin of (X, Y, Z); *near set when a straddling quarter
// reached PATCH_MAXL
__device__ int patch_winding(const float *X, const float *Y, const float *Z, bool *near) {
    float zmin = Z[0], zmax = Z[0];
    for (int k = 1; k < 16; k++) { zmin = fminf(zmin, Z[k]); zmax = fmaxf(zmax, Z[k]); }
    if (zmax <= 0.f) return 0;
    if (zmin > 0.f) return net_winding(X, Y);
    // straddling: depth-first over quarters (level, iu, iv) packed as
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

__global__ void __launch_bounds__(128) chi_patches_kernel(const float4 *__restrict__ qnet,
                                                          const float4 *__restrict__ box,
                                                          const float *__restrict__ zmax,
                                                          const int32_t *__restrict__ bin_off,
                                                          const int32_t *__restrict__ bin_idx, int nbx, int nby,
                                                          float bx0, float by0, float binv, Frame fr, QuerySrc q,
                                                          int32_t *__restrict__ chi, unsigned long long *cnt,
                                                          int *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= q.n) return;
    const float3 p = query_point3(q, i);
    const float a = fmaf(p.z, fr.e1[2], fmaf(p.y, fr.e1[1], p.x * fr.e1[0]));
    const float b = fmaf(p.z, fr.e2[2], fmaf(p.y, fr.e2[1], p.x * fr.e2[0]));
    const float c = fmaf(p.z, fr.dh[2], fmaf(p.y, fr.dh[1], p.x * fr.dh[0]));
    int wsum = 0, tests = 0;
    bool near = false;
    const float fx = (a - bx0) * binv, fy = (b - by0) * binv;
    if (fx >= 0.f && fy >= 0.f && fx < (float)nbx && fy < (float)nby) {
        const int cell = (int)fy * nbx + (int)fx;
        for (int k = bin_off[cell]; k < bin_off[cell + 1]; k++) {
            const int t = bin_idx[k];
            const float4 bb = __ldg(&box[t]);
            if (a < bb.x || a > bb.y || b < bb.z || b > bb.w || !(__ldg(&zmax[t]) > c)) continue;
            float X[16], Y[16], Z[16];
#pragma unroll
            for (int m = 0; m < 16; m++) {
                const float4 v = __ldg(&qnet[16 * (int64_t)t + m]);
                X[m] = v.x - a;
                Y[m] = v.y - b;
                Z[m] = v.z - c;
            }
            wsum += patch_winding(X, Y, Z, &near);
            tests++;
        }
    }
    chi[i] = -wsum;                      // e1 x e2 = -dh
    if (cnt) {
        if (tests) atomicAdd(&cnt[CNT_TRI_TESTS], (unsigned long long)tests);
        if (near) atomicAdd(&cnt[CNT_STACK_OVERFLOW], 1ull);
    }
    (void)status;
}

cudaError_t launch_chi_patches(const PatchSet &ps, const QuerySrc &q, int32_t *chi, unsigned long long *cnt,
                               int *status, cudaStream_t st) {
    if (q.n == 0) return cudaSuccess;
    const int64_t blocks = (q.n + 127) / 128;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    chi_patches_kernel<<<(unsigned)blocks, 128, 0, st>>>(ps.qnet, ps.box, ps.zmax, ps.bin_off, ps.bin_idx, ps.nbx,
                                                         ps.nby, ps.bx0, ps.by0, ps.binv, ps.frame, q, chi, cnt,
                                                         status);
    return cudaGetLastError();
}

// ---- host ----------------------------------------------------------------------

void patches_free(PatchSet &ps) {
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

gwn_status patches_prepare(gwn_geom *g, const float d[3]) {
    PatchSet &ps = g->ps;
    if (!isfinite(d[0]) || !isfinite(d[1]) || !isfinite(d[2]) || (d[0] == 0.f && d[1] == 0.f && d[2] == 0.f)) {
        set_error("patches: direction must be finite and nonzero");
        return GWN_E_INVALID;
    }
    if (ps.valid && memcmp(ps.dkey, d, sizeof(float) * 3) == 0) return GWN_OK;
    patches_free(ps);
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
    if (e == cudaSuccess && g->n_bseq > 0) {
        e = cudaMalloc(&ps.bframe, sizeof(float4) * 2 * g->n_bseq);
        if (e == cudaSuccess) e = launch_bframe(g->bseq, g->n_bseq, fr, ps.bframe, g->ctx->stream);
    }
    if (e != cudaSuccess) {
        patches_free(ps);
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
        }
        for (int r = 0; r < (m > 0 ? m : -m); r++)
            for (int s = 0; s < segments; s++) {
                if (ids[s] == ids[s + 1]) continue;
                if (m > 0) bedges.emplace_back(ids[s], ids[s + 1]);
                else bedges.emplace_back(ids[s + 1], ids[s]);
            }
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
    if (g->n_bseq) {
        e = cudaMalloc(&g->bseq, sizeof(float4) * g->n_bseq);
        if (e == cudaSuccess) e = cudaMemcpy(g->bseq, rec.data(), sizeof(float4) * g->n_bseq, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        if (g->bseq) cudaFree(g->bseq);
        g->bseq = nullptr;
        return cuda_fail(e, "gwn_patches_create");
    }
    ctx_add_geometry(ctx);
    *out = g.release();
    return GWN_OK;
}
