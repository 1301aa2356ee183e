// bezier2d.cu -- one-shot winding numbers of open cubic Bezier chains on
// regular grids, with one ray (+x) per grid row.
//
// For an open chain C from s to e, closing it with the chord e -> s gives a
// closed curve whose winding number at p is the signed crossing count of any
// ray from p; hence, relative to the +x ray,
//     w_C(p) = chi_x(C; p) + chi_x(chord e->s; p)
//              + (1/2pi) atan2(cross(s-p, e-p), dot(s-p, e-p)),
// the last term being minus the angle the chord subtends.  (Algorithm 1 in 2D:
// the boundary is the two end points, the circle has two arcs, and the arc
// areas and pairwise difference collapse to this form.)
//
// All queries of one grid row share the ray direction and the ray line, so
// the crossings of that line with the chain are computed once per row and
// every query counts the crossings to its right (the "Optimization" of the
// one-shot algorithm: one ray serves all points on it).
//
// Crossings: each segment is split on the host into y-monotone pieces at the
// roots of dy/du.  A piece with end values y0, y1 is crossed by the row y_r
// iff min(y0,y1) <= y_r < max(y0,y1) (the ray is taken infinitesimally above
// the row, which makes shared end points count once); its direction is
// sign(y1 - y0) (the curve's normal is the tangent turned clockwise: Eq. chi
// counts +1 where the curve crosses the ray upward).  The crossing parameter
// is found by safeguarded Halley iteration on the monotone piece, in the
// chain's precision.
//
// Work: a persistent kernel pops work items (set, block of rows) from an
// atomic counter.  An item counts the crossings of its rows, finds each
// (piece, row) root with the work spread over the whole block, bins the
// roots by row and column in shared memory, and then one warp per row turns
// the binned crossings into each query's count of crossings to its right,
// adds the chord terms and writes w (details at eval2d_kernel).
#include <string.h>

#include <algorithm>

#include "gwn_internal.h"
#include "predicates.cuh"

namespace gwn {

template <typename T> struct Num;
// Root tolerances.  The root iteration stops once the curve point at u lies within
// ytol (|y(u0)| + |y(u1)|) of the row in y, or once its step (or the bracket)
// is below tol in u.  A computed root whose curve point is within e of the
// row can change the crossing count of a query on the row only if the query
// lies between the computed and the true crossing, and every such query is
// within e of the curve (the arc of the monotone piece between the two runs
// over those x values with y within e of the row).  That is far inside the
// band (1e-4 of the grid diagonal) where w is not compared.  The y test ends
// the iteration early near a piece end, where dy/du vanishes (pieces are
// split at the extrema of y) and the step in u shrinks slowly.
template <> struct Num<float> {
    static constexpr float inv2pi = 0.15915494309189535f;
    static constexpr int max_iter = 60;
    static constexpr float tol = 1e-6f;
    static constexpr float ytol = 1e-6f;
    // iteration quotients: an approximate quotient (2 ulp) only perturbs the
    // iterates; the stopping test on the step decides the accuracy
    static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
    // a product and a sum the compiler may not fuse (every path rounds alike)
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <> struct Num<double> {
    static constexpr double inv2pi = 0.15915494309189533577;
    static constexpr int max_iter = 200;
    static constexpr double tol = 1e-16;
    static constexpr double ytol = 1e-15;
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
};

// Piece records (PC_FIELDS values in the chain's precision, written at
// creation in float64 and rounded): the monotone piece [u0, u1] of a segment
// reparametrised to t in [0, 1] (u = u0 + t (u1 - u0)) in power form,
//   x(t) = ((r0 t + r1) t + r2) t + r3,   y(t) = ((r4 t + r5) t + r6) t + r7,
// r7 = y(u0), r8 = 3 r4, r9 = 2 r5 (so y'(t) = (r8 t + r9) t + r6),
// r10 = y(u1), r11 unused.  Local coefficients scale with the piece, so the
// evaluation error is a few ulps of |y| rather than of the segment's size.
constexpr int PC_FIELDS = 12;

// x of the crossing of the piece with record r and the row y = yr
// (min(r7, r10) <= yr < max(r7, r10)): safeguarded Halley iteration, the
// bracket oriented so that g(lo) <= 0 < g(hi), g = y(t) - yr.  The bracket
// starts as the half of [0, 1] that holds the root (g at t = 1/2 against 0),
// and the first iterate is the secant on that half.
template <typename T>
__device__ __forceinline__ T piece_root_rec(const T *r, T yr, int *iters_out, T *t_out = nullptr) {
    const T ya = r[7], yb = r[10];
    const bool inc = yb > ya;
    T lo = inc ? T(0) : T(1), hi = inc ? T(1) : T(0);
    const T c0 = ya - yr;
    const T gm = Num<T>::fma_(Num<T>::fma_(Num<T>::fma_(r[4], T(0.5), r[5]), T(0.5), r[6]), T(0.5), c0);
    T glo = inc ? c0 : yb - yr, ghi = inc ? yb - yr : c0;
    if (gm <= T(0)) { lo = T(0.5); glo = gm; } else { hi = T(0.5); ghi = gm; }
    T t = lo + Num<T>::div(-glo, ghi - glo) * (hi - lo);
    const T ytol = Num<T>::ytol * ((ya < T(0) ? -ya : ya) + (yb < T(0) ? -yb : yb));
    const T r8x2 = T(2) * r[8];
    int it = 0;
    for (; it < Num<T>::max_iter; it++) {
        const T g = Num<T>::fma_(Num<T>::fma_(Num<T>::fma_(r[4], t, r[5]), t, r[6]), t, c0);
        if ((g < T(0) ? -g : g) <= ytol) break;     // the curve point is within ytol of the row
        if (g < T(0)) lo = t; else hi = t;
        const T dg = Num<T>::fma_(Num<T>::fma_(r[8], t, r[9]), t, r[6]);
        const T d2g = Num<T>::fma_(r8x2, t, r[9]);
        // Halley's step t - 2 g g' / (2 g'^2 - g g'') (cubic convergence)
        const T gdg = g * dg;
        T tn = t - Num<T>::div(gdg + gdg, Num<T>::fma_(dg + dg, dg, -g * d2g));
        const T mn = lo < hi ? lo : hi, mx = lo < hi ? hi : lo;
        if (!(tn > mn && tn < mx)) tn = T(0.5) * (lo + hi);
        const T step = tn - t;
        t = tn;
        if ((step < T(0) ? -step : step) <= Num<T>::tol || (mx - mn) <= Num<T>::tol) break;
    }
    *iters_out = it;
    if (t_out) *t_out = t;
    return Num<T>::fma_(Num<T>::fma_(Num<T>::fma_(r[0], t, r[1]), t, r[2]), t, r[3]);
}

// ---- certification of crossings ---------------------------------------------
// A crossing computed from a piece record can sit on the wrong side of a
// query for three reasons: the iteration stops at a tolerance, the record's
// coefficients are rounded, and the row test uses end values rounded at
// interior extrema of y.  The kernels bound the first two per crossing
// (root_band) and hand every (piece, row) whose bound contains a query
// column -- and every row within rounding of an interior extremum value -- to
// the certification pass, which decides those queries in float64 from the
// control points.
template <typename T> struct Unit;
template <> struct Unit<float> { static constexpr float u = 5.9604645e-8f; };              // 2^-24
template <> struct Unit<double> { static constexpr double u = 1.1102230246251565e-16; };   // 2^-53

// Half-width of an interval about the computed crossing x_r that contains the
// crossing of the exact curve, or +inf where the bound below does not apply.
// With g(t) = y(t) - yr evaluated at the iteration's final t: |g_exact(t)| <= |g| +
// eg, eg covering the evaluation and the rounded coefficients; |y''| <= m2 on
// [0, 1], so if m2 bt <= |y'(t)| / 2 (y' shrunk by its own error), y' keeps
// at least half its size on [t - bt, t + bt] and the root lies within
// bt = 2 (|g| + eg) / |y'(t)| of t; x moves by at most (|x'(t)| + m2x bt) bt
// there, plus the error ex of x itself.
// Error terms: Horner's rule on t in [0, 1] errs by at most ~3u of the sum of
// the absolute terms, the coefficients carry half an ulp each from rounding
// (the constant term y(u0) or x(u0) included: exact at control points, one
// rounding at an extremum), so eg = 8u (|r4| + |r5| + |r6| + |r7 - yr|) +
// u |r7| and ex = 8u (|r0| + |r1| + |r2|) + u |r3| cover them with margin.
template <typename T>
__device__ __forceinline__ T root_band(const T *r, T yr, T t) {
    const T u = Unit<T>::u;
    const T c0 = r[7] - yr;
    const T g = Num<T>::fma_(Num<T>::fma_(Num<T>::fma_(r[4], t, r[5]), t, r[6]), t, c0);
    const T dg = Num<T>::fma_(Num<T>::fma_(r[8], t, r[9]), t, r[6]);
    const T eg = T(8) * u * (fabs(r[4]) + fabs(r[5]) + fabs(r[6]) + fabs(c0)) + u * fabs(r[7]);
    const T adg = fabs(dg) - T(8) * u * (fabs(r[8]) + fabs(r[9]) + fabs(r[6]));
    const T m2 = T(6) * fabs(r[4]) + T(2) * fabs(r[5]);
    // (a quotient of at most 2 ulp error in float32, enlarged by 2^-21 so
    // that bt is not below the exact value)
    const T bt = T(2) * (fabs(g) + eg) * Num<T>::div(T(1) + T(4.76837158203125e-7) * (sizeof(T) == 4), adg);
    if (!(adg > T(0)) || !(m2 * bt <= T(0.5) * adg)) return T(INFINITY);
    const T dx = Num<T>::fma_(Num<T>::fma_(T(3) * r[0], t, T(2) * r[1]), t, r[2]);
    const T m2x = T(6) * fabs(r[0]) + T(2) * fabs(r[1]);
    return (fabs(dx) + m2x * bt) * bt + T(8) * u * (fabs(r[0]) + fabs(r[1]) + fabs(r[2])) + u * fabs(r[3]);
}

// An interval that contains the exact crossing and the float one (x, the
// root the float path counts with).  Where root_band at the iteration's own stopping
// point is too wide to settle a query, two more Newton steps from t usually
// shrink it to the rounding level: the interval is then the hull of x and
// the refined root's band.  Returns false (no bound) where the bound does not
// apply.
template <typename T>
__device__ __forceinline__ bool cert_interval(const T *r, T yr, T t, T x, T &lo, T &hi) {
    T t2 = t;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const T g = Num<T>::fma_(Num<T>::fma_(Num<T>::fma_(r[4], t2, r[5]), t2, r[6]), t2, r[7] - yr);
        const T dg = Num<T>::fma_(Num<T>::fma_(r[8], t2, r[9]), t2, r[6]);
        T tn = t2 - g / dg;
        tn = tn < T(0) ? T(0) : (tn > T(1) ? T(1) : tn);
        t2 = tn == tn ? tn : t2;
    }
    const T b2 = root_band<T>(r, yr, t2);
    if (!(b2 < T(INFINITY))) return false;
    const T x2 = Num<T>::fma_(Num<T>::fma_(Num<T>::fma_(r[0], t2, r[1]), t2, r[2]), t2, r[3]);
    lo = x2 - b2 < x ? x2 - b2 : x;
    hi = x2 + b2 > x ? x2 + b2 : x;
    return true;
}

// the row yr lies within the rounding of one of the piece's interior-extremum
// end values (ya = y(u0), yb = y(u1) as stored, eps their bounds).  The
// bounds are read only when yr is within 8u (|ya| + |yb|) + eps_abs of an
// end, which every bound is below.
template <typename T>
__device__ __forceinline__ T near_window(T ya, T yb, T eps_abs) {
    return T(8) * Unit<T>::u * (fabs(ya) + fabs(yb)) + eps_abs;
}
template <typename T>
__device__ __forceinline__ bool near_extremum(T yr, T ya, T yb, const T *eps_p, T eps_abs) {
    const T win = near_window<T>(ya, yb, eps_abs);
    if (!(fabs(yr - ya) <= win || fabs(yr - yb) <= win)) return false;
    const T e0 = eps_p[0], e1 = eps_p[1];
    return (e0 > T(0) && fabs(yr - ya) <= e0) || (e1 > T(0) && fabs(yr - yb) <= e1);
}

// first column j in [0, nx] with ax[j] > x
template <typename T>
__device__ __forceinline__ int upper_bound_cols_lin(const T *ax, int nx, T x) {
    int lo = 0, hi = nx;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (ax[mid] > x) hi = mid; else lo = mid + 1;
    }
    return lo;
}
// first column j in [0, nx] with ax[j] >= x
template <typename T>
__device__ __forceinline__ int lower_bound_cols_lin(const T *ax, int nx, T x) {
    int lo = 0, hi = nx;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (ax[mid] >= x) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// append one certification entry: queries (set, row, columns [c0, c1)) against
// piece p (and its partner q >= 0 at an interior extremum)
__device__ __forceinline__ void cert_push(int4 *cert, int32_t *cert_count, int *status, unsigned long long *cnt,
                                          int set, int row, int p, int q, int c0, int c1) {
    if (c1 <= c0) return;
    const int slot = atomicAdd(cert_count, 1);
    if (slot >= GWN_CERT_CAP) {
        if (status) atomicOr(status, ST_CERT_OVERFLOW);
        return;
    }
    cert[2 * slot] = make_int4(set, row, p, q);
    cert[2 * slot + 1] = make_int4(c0, c1, 0, 0);
    if (cnt) atomicAdd(&cnt[CNT_CERT], 1ull);
}

// Certification (see root_band): the scan of an item's pieces lists the rows
// within rounding of a piece's interior-extremum end value, once per pair of
// pieces sharing it, with the columns of both pieces' x-ranges; the root pass
// lists each crossing whose error bound contains a query column.
struct CertArgs2D {
    double eps_abs;            // see near_window
    const void *piece_eps;     // [n_pieces][2], chain dtype
    const int2 *piece_part;    // [n_pieces]
    const void *piece_x;       // [n_pieces][2] conservative x-ranges, chain dtype
    int4 *cert;
    int32_t *count;
};

// float64 decision for one piece on the row yr: whether the exact curve
// crosses the row there (half-open in y) and, if so, the x of the crossing and
// its direction.  From the segment's control points: the row test on the end
// values y(u0), y(u1) (exact at control points), then bisection of the
// monotone y(u) - yr on [u0, u1] to the resolution of float64 and x there.
// A query (xq, yr) counts the crossing iff x > xq.
struct ExactCross {
    double x;
    int dir;          // 0: the row does not cross the piece
};
template <typename T>
__device__ __noinline__ ExactCross piece_exact(const T *__restrict__ ctrl, int64_t seg, double2 uu, double yr) {
    double c[8];
    for (int k = 0; k < 8; k++) c[k] = (double)ctrl[2 * seg + k];
    auto bez = [&](int d, double u) {
        const double v = 1.0 - u;
        const double p01 = v * c[d] + u * c[2 + d], p12 = v * c[2 + d] + u * c[4 + d], p23 = v * c[4 + d] + u * c[6 + d];
        const double q0 = v * p01 + u * p12, q1 = v * p12 + u * p23;
        return v * q0 + u * q1;
    };
    ExactCross r{0.0, 0};
    const double y0 = uu.x <= 0.0 ? c[1] : bez(1, uu.x), y1 = uu.y >= 1.0 ? c[7] : bez(1, uu.y);
    const double lo = y0 < y1 ? y0 : y1, hi = y0 < y1 ? y1 : y0;
    if (!(lo <= yr && yr < hi)) return r;
    const bool inc = y1 > y0;
    double a = uu.x, b = uu.y;                        // y(a) <= yr < y(b) in the increasing sense
    for (int it = 0; it < 128; it++) {
        const double m = 0.5 * (a + b);
        if (!(m > a && m < b)) break;
        const double ym = bez(1, m);
        if ((ym > yr) == inc) b = m; else a = m;
    }
    r.x = bez(0, 0.5 * (a + b));
    r.dir = inc ? 1 : -1;
    return r;
}

// a piece record from global memory (16-byte aligned, read as 16-byte words)
template <typename T>
__device__ __forceinline__ void load_rec(const T *__restrict__ piece_rec, int64_t p, T *v) {
    constexpr int W = PC_FIELDS * (int)sizeof(T) / 16;
    const uint4 *rp = (const uint4 *)(piece_rec + (int64_t)PC_FIELDS * p);
#pragma unroll
    for (int m = 0; m < W; m++) ((uint4 *)v)[m] = rp[m];
}

constexpr int MAX_ROWS = 256;        // rows per work item

// a piece record into L1 ahead of its use (no registers held)
template <typename T>
__device__ __forceinline__ void prefetch_rec(const T *__restrict__ piece_rec, int64_t p) {
    const char *a = (const char *)(piece_rec + (int64_t)PC_FIELDS * p);
    asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(a + PC_FIELDS * sizeof(T) - 1));
}

// Chord term arithmetic.  For the chord from s to e seen from p = (xq, yr),
// with sy = s.y - yr, ey = e.y - yr (per row) and sx = s.x - xq, ex = e.x - xq:
//   cr = cross(e - p, s - p) = ex sy - ey sx,   dt = dot(s - p, e - p),
// and the term is atan2(-cr, dt) / 2 pi.  Every path (scalar, and the packed
// float32 path of the row queries) evaluates these with the same fused
// operations in the same order, so they round alike and agree bit for bit.
template <typename T>
__device__ __forceinline__ void chord_cd(T spx, T sy, T epx, T ney, T syey, T xq, T &cr, T &dt) {
    const T sx = Num<T>::add(spx, -xq), ex = Num<T>::add(epx, -xq);
    cr = Num<T>::fma_(ex, sy, Num<T>::mul(sx, ney));
    dt = Num<T>::fma_(sx, ex, syey);
}

// piece_exact by one warp: each step evaluates y at 32 interior points of
// the bracket (one per lane) and keeps the sub-interval where y - yr changes
// sign, shrinking the bracket 33-fold, so about eleven steps reach the
// resolution of float64 (the scalar bisection needs about 53).  Every lane
// returns the same result.
template <typename T>
__device__ __noinline__ ExactCross piece_exact_warp(const T *__restrict__ ctrl, int64_t seg, double2 uu, double yr) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const double x0 = (double)ctrl[2 * seg], y0c = (double)ctrl[2 * seg + 1];
    const double x1 = (double)ctrl[2 * seg + 2], y1c = (double)ctrl[2 * seg + 3];
    const double x2 = (double)ctrl[2 * seg + 4], y2c = (double)ctrl[2 * seg + 5];
    const double x3 = (double)ctrl[2 * seg + 6], y3c = (double)ctrl[2 * seg + 7];
    auto casteljau = [](double p0, double p1, double p2, double p3, double u) {
        const double v = 1.0 - u;
        const double p01 = v * p0 + u * p1, p12 = v * p1 + u * p2, p23 = v * p2 + u * p3;
        return v * (v * p01 + u * p12) + u * (v * p12 + u * p23);
    };
    ExactCross r{0.0, 0};
    const double ya = uu.x <= 0.0 ? y0c : casteljau(y0c, y1c, y2c, y3c, uu.x);
    const double yb = uu.y >= 1.0 ? y3c : casteljau(y0c, y1c, y2c, y3c, uu.y);
    const double lo = ya < yb ? ya : yb, hi = ya < yb ? yb : ya;
    if (!(lo <= yr && yr < hi)) return r;
    const bool inc = yb > ya;
    double a = uu.x, b = uu.y;                        // y(a) <= yr < y(b) in the increasing sense
    for (int it = 0; it < 24; it++) {                 // warp-uniform: a, b are the same on every lane
        const double m = a + (b - a) * ((double)(lane + 1) / 33.0);
        const bool interior = m > a && m < b;        // the points are non-decreasing in the lane
        const unsigned ib = __ballot_sync(FULL, interior);
        if (!ib) break;                               // float64 resolution reached
        const bool right = (casteljau(y0c, y1c, y2c, y3c, m) > yr) == inc;   // the crossing is at or left of m
        const unsigned rb = __ballot_sync(FULL, interior && right);
        if (rb) {
            const int k = __ffs(rb) - 1;
            const double nb = __shfl_sync(FULL, m, k);
            const double na = __shfl_sync(FULL, m, k > 0 ? k - 1 : 0);
            if (k > 0 && ((ib >> (k - 1)) & 1u)) a = na;
            b = nb;
        } else {
            a = __shfl_sync(FULL, m, 31 - __clz(ib));  // the last interior point
        }
    }
    r.x = casteljau(x0, x1, x2, x3, 0.5 * (a + b));
    r.dir = inc ? 1 : -1;
    return r;
}

// Side of the chord for the crossing count.  The chord e -> s crosses the
// ray to the right of p iff cr = cross(e - p, s - p) has the sign of the
// chord's direction in y; the angle term takes its branch from the same cr,
// so w is the same on either side (the count's step and the angle's 2 pi
// step cancel) and only the count itself depends on the sign.  cr as
// computed (two rounded differences, a product and a fused product-add) is
// off by at most 8u (|ex sy| + |sx ey|); within that its sign is uncertain,
// and the certification pass takes it exactly: cr expands into six products
// of the input coordinates (the p.x p.y terms cancel), each split into an
// exact hi + lo pair by FMA, summed as a nonoverlapping expansion.
template <typename T>
__device__ __noinline__ int chord_sign_exact(T spx, T spy, T epx, T epy, T xq, T yr) {
    const double a[6] = {(double)epx, -(double)epx, -(double)xq, -(double)spx, (double)spx, (double)xq};
    const double b[6] = {(double)spy, (double)yr, (double)spy, (double)epy, (double)yr, (double)epy};
    Expansion<16> E;
    E.init();
    for (int k = 0; k < 6; k++) {
        const double hi = a[k] * b[k];
        E.add(fma(a[k], b[k], -hi));
        E.add(hi);
    }
    return E.sign();
}

// The float path counts the chord's crossing with the ray (right of the
// query) iff the sign bit of cr is that of a crossing in the chord's
// direction in y (up: clear, down: set).  The angle term takes its sign from
// the same bit, so w is continuous across the chord, cr = +0 and -0 included.
template <typename T>
__device__ __forceinline__ bool chord_right(T cr, bool up) { return up != (bool)signbit(cr); }

template <typename T>
__device__ __forceinline__ bool chord_uncertain(T cr, T sx, T ex, T sy, T ey) {
    return !(fabs(cr) > T(8) * Unit<T>::u * (fabs(ex * sy) + fabs(sx * ey)));
}

// the float path's chord crossing at (xq, yr) for chain c, as chord_angles
// counts it, and the exact one: (float, exact) signed counts
template <typename T>
__device__ __forceinline__ int2 chord_counts(const T *__restrict__ ctrl, const int64_t *__restrict__ chain_off,
                                             int64_t c, T xq, T yr);

// Odd polynomial atan(v) ~ v P(v^2) on [-1, 1] for the chord term, P of
// degree 7 fitted by Lawson-weighted least squares to the relative error
// (1.0e-7 in exact arithmetic).  Evaluated in float32 its error (1.5e-7
// absolute) is that of the float32 rounding, as for a degree-8 fit: a query
// adds a single chord angle, so w is off by at most ~5e-8 from it.
#define GWN_ATC7 -0.0046932739f
#define GWN_ATC6 0.024252396f
#define GWN_ATC5 -0.059486382f
#define GWN_ATC4 0.099142924f
#define GWN_ATC3 -0.1401948f
#define GWN_ATC2 0.19969724f
#define GWN_ATC1 -0.3333199f
#define GWN_ATC0 0.99999988f
#define GWN_PI_2_F 1.5707963267948966f

// atan2(-cr, dt) in float32.  With z = |(cr, dt)| and v = dt / (|cr| + z) in
// [-1, 1] (no cancellation: the denominator is at least z),
//   atan2(-cr, dt) = sign(-cr) (pi/2 - 2 atan(v)),
// the half-angle identity for the angle between the direction (dt, |cr|)
// and the axis (0, 1); its branch cut (-cr changing sign where dt < 0) is
// where the chord's crossing count changes, so w stays continuous.  The sign
// is applied by flipping the sign bit (multiplying by sign(-cr)).  MUFU
// rsqrt and reciprocal (~2 ulp); z^2 = cr^2 + dt^2 + 1e-37 (the constant in
// the first FMA) so that a query on a chord end point (z = 0) gets a finite
// term (+-pi/2; w is undefined on the curve).
__device__ __forceinline__ float frsqrt_(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float frcp_(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sign_of_neg(float phi, float cr) {      // sign(-cr) * phi
    return __uint_as_float(__float_as_uint(phi) ^ (~__float_as_uint(cr) & 0x80000000u));
}
__device__ __forceinline__ float chord_angle(float cr, float dt) {
    const float z2 = __fmaf_rn(dt, dt, __fmaf_rn(cr, cr, 1e-37f));
    const float d = __fmaf_rn(z2, frsqrt_(z2), fabsf(cr));
    const float v = __fmul_rn(dt, frcp_(d)), v2 = __fmul_rn(v, v);
    float q = __fmaf_rn(GWN_ATC7, v2, GWN_ATC6);
    q = __fmaf_rn(q, v2, GWN_ATC5);
    q = __fmaf_rn(q, v2, GWN_ATC4);
    q = __fmaf_rn(q, v2, GWN_ATC3);
    q = __fmaf_rn(q, v2, GWN_ATC2);
    q = __fmaf_rn(q, v2, GWN_ATC1);
    q = __fmaf_rn(q, v2, GWN_ATC0);
    const float phi = __fmaf_rn(-2.f, __fmul_rn(q, v), GWN_PI_2_F);     // pi/2 - 2 atan(v)
    return sign_of_neg(phi, cr);
}

// two chord angles at once: the same operations as chord_angle, the
// add/mul/fma ones as packed f32x2 (fma.rn/mul.rn per element)
__device__ __forceinline__ float2 chord_angle2(float2 cr, float2 dt) {
    const float2 z2 = __ffma2_rn(dt, dt, __ffma2_rn(cr, cr, make_float2(1e-37f, 1e-37f)));
    const float2 acr = make_float2(fabsf(cr.x), fabsf(cr.y));
    const float2 d = __ffma2_rn(z2, make_float2(frsqrt_(z2.x), frsqrt_(z2.y)), acr);
    const float2 v = __fmul2_rn(dt, make_float2(frcp_(d.x), frcp_(d.y)));
    const float2 v2 = __fmul2_rn(v, v);
    float2 q = __ffma2_rn(make_float2(GWN_ATC7, GWN_ATC7), v2, make_float2(GWN_ATC6, GWN_ATC6));
    q = __ffma2_rn(q, v2, make_float2(GWN_ATC5, GWN_ATC5));
    q = __ffma2_rn(q, v2, make_float2(GWN_ATC4, GWN_ATC4));
    q = __ffma2_rn(q, v2, make_float2(GWN_ATC3, GWN_ATC3));
    q = __ffma2_rn(q, v2, make_float2(GWN_ATC2, GWN_ATC2));
    q = __ffma2_rn(q, v2, make_float2(GWN_ATC1, GWN_ATC1));
    q = __ffma2_rn(q, v2, make_float2(GWN_ATC0, GWN_ATC0));
    const float2 phi = __ffma2_rn(make_float2(-2.f, -2.f), __fmul2_rn(q, v), make_float2(GWN_PI_2_F, GWN_PI_2_F));
    return make_float2(sign_of_neg(phi.x, cr.x), sign_of_neg(phi.y, cr.y));
}

template <typename T> struct Chord;
template <> struct Chord<float> {
    static __device__ __forceinline__ float angle(float cr, float dt) { return chord_angle(cr, dt); }
};
template <> struct Chord<double> {
    static __device__ __forceinline__ double angle(double cr, double dt) { return atan2(-cr, dt); }
};

// first row i in [0, n) with ys[i] >= v (n if none), on the item's rows (a
// run of a grid axis: non-decreasing, spaced ~uniformly, y0 = ys[0], inv_h =
// (n - 1) / (ys[n-1] - ys[0])): a guess from the spacing, corrected against
// the stored values, so the result is exactly the lower bound
template <typename T>
__device__ __forceinline__ int lower_bound_rows_grid(const T *ys, int n, T y0, T inv_h, T v) {
    if (!(v > y0)) return 0;
    if (!(v <= ys[n - 1])) return n;
    // here ys[0] < v <= ys[n-1], so the bound lies in [1, n-1]
    T g = (v - y0) * inv_h;
    int j = g >= T(n - 1) ? n - 1 : (int)ceil(g);
    if (j < 1) j = 1;
    while (j > 1 && ys[j - 1] >= v) j--;
    while (ys[j] < v) j++;
    return j;
}

// first column j in [0, nx] with ax[j] >= x, on a grid axis (non-decreasing,
// spaced ~uniformly; here the item's copy in shared memory): a guess from the
// spacing, corrected against the stored values, so the result is exactly the
// lower bound
template <typename T>
__device__ __forceinline__ int lower_bound_cols(const T *ax, int nx, T a0, T inv_step, T x) {
    const T g = (x - a0) * inv_step;
    int j = !(g > T(0)) ? 0 : (g >= T(nx) ? nx : (int)ceil(g));
    while (j > 0 && ax[j - 1] >= x) j--;
    while (j < nx && ax[j] < x) j++;
    return j;
}

// chord terms of the set's chains at (xq, yr): each chord's crossing with the
// +x ray (half-open in y) is added to chi; returns the sum A of the angles
// atan2(-cr, dt) (w = chi + A / 2 pi)
// (on_unc(c) is called for each chain whose chord side is uncertain at the
// query; see chord_uncertain)
template <typename T, typename F>
__device__ __forceinline__ T chord_angles(const T *__restrict__ ctrl, const int64_t *__restrict__ chain_off,
                                         const Set2D &S, T xq, T yr, int &chi, F on_unc) {
    T A = T(0);
    for (int64_t c = S.c_lo; c < S.c_hi; c++) {
        const T *sp = ctrl + 2 * chain_off[c];
        const T *ep = ctrl + 2 * (chain_off[c + 1] - 1);
        const T sy = sp[1] - yr, ey = ep[1] - yr;
        T cr, dt;
        chord_cd<T>(sp[0], sy, ep[0], -ey, sy * ey, xq, cr, dt);
        T lo = ey < sy ? ey : sy, hi = ey < sy ? sy : ey;
        if (lo <= T(0) && T(0) < hi) {
            bool up = sy > ey;
            const bool right = chord_right<T>(cr, up);
            if (right) chi += up ? 1 : -1;
            if (chord_uncertain<T>(cr, Num<T>::add(sp[0], -xq), Num<T>::add(ep[0], -xq), sy, ey)) on_unc(c);
        }
        A = Num<T>::add(A, Chord<T>::angle(cr, dt));
    }
    return A;
}

template <typename T>
__device__ __forceinline__ int2 chord_counts(const T *__restrict__ ctrl, const int64_t *__restrict__ chain_off,
                                             int64_t c, T xq, T yr) {
    const T *sp = ctrl + 2 * chain_off[c];
    const T *ep = ctrl + 2 * (chain_off[c + 1] - 1);
    const T sy = sp[1] - yr, ey = ep[1] - yr;
    T cr, dt;
    chord_cd<T>(sp[0], sy, ep[0], -ey, sy * ey, xq, cr, dt);
    const T lo = ey < sy ? ey : sy, hi = ey < sy ? sy : ey;
    if (!(lo <= T(0) && T(0) < hi)) return make_int2(0, 0);
    const bool up = sy > ey;
    const int d = up ? 1 : -1;
    const int f = chord_right<T>(cr, up) ? d : 0;
    const int sg = chord_sign_exact<T>(sp[0], sp[1], ep[0], ep[1], xq, yr);
    const int e = (up ? (sg > 0) : (sg < 0)) ? d : 0;
    return make_int2(f, e);
}

// w = chi + A / 2 pi, formed as one fused multiply-add on every path;
// b = A / 2 pi
template <typename T>
__device__ __forceinline__ T w_of(int chi, T A) { return Num<T>::fma_(A, Num<T>::inv2pi, (T)chi); }

template <typename T>
__device__ __forceinline__ void store_w(const Set2D &S, int64_t row, int64_t i, int chi, T A, T *w_out,
                                        int32_t *chi_out, T *b_out) {
    int64_t o = S.out_off + row * S.nx + i;
    if (w_out) w_out[o] = w_of<T>(chi, A);
    if (chi_out) chi_out[o] = chi;
    if (b_out) b_out[o] = Num<T>::mul(A, Num<T>::inv2pi);
}

// Row stride of a work item's difference cells: the grid width rounded up to
// 256 columns (int cells).
__host__ __device__ constexpr int eval2d_dstride(int nx) { return (nx + 255) & ~255; }

// The queries of one grid row, by one warp.  D holds the row's difference
// cells: crossing k lies to the right of the queries i < j_k (j_k = first
// column with x >= x_k), and added its direction to D[j_k - 1], so
//   chi(i) = sum_{j >= i} D[j].
// Lane l takes 8 consecutive columns of every 256: local suffix sums in
// registers, one warp suffix scan of the lane totals per 256 columns, the
// chunks taken from the right so the carry is known; each lane resets the
// cells it read.  Then the chord term is added and w stored (two 16-byte
// stores per lane when aligned).
template <typename T>
__device__ __forceinline__ void row_queries(const Set2D &S, const T *__restrict__ ctrl,
                                            const int64_t *__restrict__ chain_off, const T *__restrict__ ax,
                                            int nx, int *D, T yr, int64_t row, int lane, T *w_out,
                                            int32_t *chi_out, T *b_out, const CertArgs2D &ca, int *status,
                                            unsigned long long *cnt, int set) {
    const unsigned FULL = 0xffffffffu;
    const int nxp = eval2d_dstride(nx);
    // chord of a single-chain set: end points and row constants hoisted
    const bool one = S.c_hi - S.c_lo == 1;
    T spx = T(0), sy = T(0), epx = T(0), ey = T(0);
    bool crosses = false, up = false;
    if (one) {
        const T *sp = ctrl + 2 * chain_off[S.c_lo];
        const T *ep = ctrl + 2 * (chain_off[S.c_lo + 1] - 1);
        spx = sp[0]; sy = sp[1] - yr; epx = ep[0]; ey = ep[1] - yr;
        const T lo = ey < sy ? ey : sy, hi = ey < sy ? sy : ey;
        crosses = lo <= T(0) && T(0) < hi;
        up = sy > ey;
    }
    const int64_t obase = S.out_off + row * S.nx;
    int carry = 0;
    for (int c0 = nxp - 256; c0 >= 0; c0 -= 256) {
        const int i0 = c0 + 8 * lane;
        int4 *d4 = (int4 *)(D + i0);
        const int4 da = d4[0], db = d4[1];
        d4[0] = make_int4(0, 0, 0, 0);
        d4[1] = make_int4(0, 0, 0, 0);
        int t[8];
        t[7] = db.w; t[6] = db.z + t[7]; t[5] = db.y + t[6]; t[4] = db.x + t[5];
        t[3] = da.w + t[4]; t[2] = da.z + t[3]; t[1] = da.y + t[2]; t[0] = da.x + t[1];
        int x = t[0];
        for (int off = 1; off < 32; off <<= 1) {
            int y = __shfl_down_sync(FULL, x, off);
            if (lane + off < 32) x += y;
        }
        const int before = carry + x - t[0];        // crossings right of this lane's 8 columns
        carry += __shfl_sync(FULL, x, 0);
        if (i0 >= nx) continue;
        T out[8];
#pragma unroll
        for (int m = 0; m < 8; m++) {
            const int i = i0 + m;
            if (i < nx) {
                int chi = before + t[m];
                T xq = ax[i], A;
                if (one) {
                    T cr, dt;
                    chord_cd<T>(spx, sy, epx, -ey, sy * ey, xq, cr, dt);
                    if (crosses && chord_right<T>(cr, up)) chi += up ? 1 : -1;
                    if (crosses && chi_out &&
                        chord_uncertain<T>(cr, Num<T>::add(spx, -xq), Num<T>::add(epx, -xq), sy, ey))
                        cert_push(ca.cert, ca.count, status, cnt, set, (int)row, (int)(-2 - S.c_lo), -1, i, i + 1);
                    A = Chord<T>::angle(cr, dt);
                } else {
                    A = chord_angles<T>(ctrl, chain_off, S, xq, yr, chi, [&](int64_t c) {
                        if (chi_out) cert_push(ca.cert, ca.count, status, cnt, set, (int)row, (int)(-2 - c), -1, i, i + 1);
                    });
                }
                out[m] = w_of<T>(chi, A);
                if (b_out) b_out[obase + i] = Num<T>::mul(A, Num<T>::inv2pi);
                if (chi_out) chi_out[obase + i] = chi;
            }
        }
        if (w_out) {
            T *wp = w_out + obase + i0;
            if (sizeof(T) == 4 && i0 + 8 <= nx && ((uintptr_t)wp & 15) == 0) {
                ((float4 *)wp)[0] = make_float4((float)out[0], (float)out[1], (float)out[2], (float)out[3]);
                ((float4 *)wp)[1] = make_float4((float)out[4], (float)out[5], (float)out[6], (float)out[7]);
            } else {
#pragma unroll
                for (int m = 0; m < 8; m++)
                    if (i0 + m < nx) wp[m] = out[m];
            }
        }
    }
}

// The row queries on the float32 fast path (a set of one chain, w only): the
// same counts and chord terms as row_queries, laid out for stores: of every
// 256 columns lane l takes the 4 at 4l and the 4 at 128 + 4l, so that each
// 16-byte store instruction of the warp writes 512 contiguous bytes.  The
// suffix sums of both groups of 4 run in one warp scan of the lane totals
// packed as lo + 2^16 hi (exact while every partial sum is below 2^15 in
// magnitude: the caller passes pack only when the item has fewer than 32767
// pieces, and a row crosses each piece at most once); otherwise two scans.
// The counts become floats without the conversion unit (exact: the caller
// takes this path only when the item has fewer than 2^22 - 1 pieces), and
// the chord terms are computed two columns at a time in packed f32x2
// arithmetic, rounding exactly as the generic path does.  (spx, spy), (epx,
// epy): the chain's end points.
__device__ __forceinline__ int warp_suffix_sum(int x, int lane) {
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_down_sync(0xffffffffu, x, off);
        if (lane + off < 32) x += y;
    }
    return x;
}
// ALIGNED: nx is a multiple of 256 and ax and the row's w are 16-byte
// aligned (no bounds or alignment tests per group), and pack holds.
template <bool ALIGNED>
__device__ __forceinline__ void row_queries_f32(const float *__restrict__ ax, int nx, int *D, float yr, float spx,
                                                float spy, float epx, float epy, float *__restrict__ wrow,
                                                int lane, bool pack_) {
    const bool pack = ALIGNED || pack_;
    const unsigned FULL = 0xffffffffu;
    const int nxp = eval2d_dstride(nx);
    const float sy = spy - yr, ey = epy - yr, ney = -ey, syey = sy * ey;
    const float clo = ey < sy ? ey : sy, chi_ = ey < sy ? sy : ey;
    const bool crosses = clo <= 0.f && 0.f < chi_;
    const bool up = sy > ey;
    // the chord's crossing (chord_right) in the integer domain: with s = 1
    // where cr's sign bit is set, up adds 1 - s and down adds -s
    const int cm = crosses ? 1 : 0, cup = crosses && up ? 1 : 0;
    const float2 spx2 = make_float2(spx, spx), epx2 = make_float2(epx, epx);
    const float2 sy2 = make_float2(sy, sy), ney2 = make_float2(ney, ney), syey2 = make_float2(syey, syey);
    const float2 inv2pi2 = make_float2(Num<float>::inv2pi, Num<float>::inv2pi);
    const float2 unbias2 = make_float2(-12582912.f, -12582912.f), mone2 = make_float2(-1.f, -1.f);
    int carry = 0;
    for (int c0 = nxp - 256; c0 >= 0; c0 -= 256) {
        const int ia = c0 + 4 * lane, ib = ia + 128;
        int4 *da4 = (int4 *)(D + ia), *db4 = (int4 *)(D + ib);
        const int4 da = *da4, db = *db4;
        *da4 = make_int4(0, 0, 0, 0);
        *db4 = make_int4(0, 0, 0, 0);
        int t[8];
        t[3] = da.w; t[2] = da.z + t[3]; t[1] = da.y + t[2]; t[0] = da.x + t[1];
        t[7] = db.w; t[6] = db.z + t[7]; t[5] = db.y + t[6]; t[4] = db.x + t[5];
        int ea, eb, ta, tb;               // sums over the lanes right of this one, and over all lanes
        if (pack) {
            const int own = t[0] + t[4] * 65536;
            const int x = warp_suffix_sum(own, lane);
            const int tot = __shfl_sync(FULL, x, 0), ex = x - own;
            ea = (int)(short)(ex & 0xffff);
            eb = (ex - ea) >> 16;
            ta = (int)(short)(tot & 0xffff);
            tb = (tot - ta) >> 16;
        } else {
            const int xa = warp_suffix_sum(t[0], lane), xb = warp_suffix_sum(t[4], lane);
            ea = xa - t[0];
            eb = xb - t[4];
            ta = __shfl_sync(FULL, xa, 0);
            tb = __shfl_sync(FULL, xb, 0);
        }
        // float of (count + bias 1.5 * 2^23) by integer addition
        const int ba = carry + tb + ea + cup + 0x4B400000, bb = carry + eb + cup + 0x4B400000;
        carry += ta + tb;
#pragma unroll
        for (int g = 0; g < 2; g++) {
            const int i0 = g ? ib : ia;
            if (!ALIGNED && i0 >= nx) continue;
            const bool full = ALIGNED || i0 + 4 <= nx;
            float xq[4];
            if (ALIGNED || (full && ((uintptr_t)(ax + i0) & 15) == 0)) {
                const float4 xa = *(const float4 *)(ax + i0);
                xq[0] = xa.x; xq[1] = xa.y; xq[2] = xa.z; xq[3] = xa.w;
            } else {
#pragma unroll
                for (int m = 0; m < 4; m++) xq[m] = ax[i0 + m < nx ? i0 + m : nx - 1];
            }
            float out[4];
#pragma unroll
            for (int m = 0; m < 4; m += 2) {
                const float2 X = make_float2(xq[m], xq[m + 1]);
                const float2 sx = __ffma2_rn(X, mone2, spx2), ex = __ffma2_rn(X, mone2, epx2);   // spx - x, epx - x
                const float2 cr = __ffma2_rn(ex, sy2, __fmul2_rn(sx, ney2));
                const float2 dt = __ffma2_rn(sx, ex, syey2);
                const float2 A = chord_angle2(cr, dt);
                const int bias = g ? bb : ba;
                const int s0 = (__float_as_int(cr.x) >> 31) & cm, s1 = (__float_as_int(cr.y) >> 31) & cm;
                const float2 k = __fadd2_rn(make_float2(__int_as_float(bias + t[4 * g + m] - s0),
                                                        __int_as_float(bias + t[4 * g + m + 1] - s1)), unbias2);
                const float2 o = __ffma2_rn(A, inv2pi2, k);     // w = chi + A / 2 pi
                out[m] = o.x;
                out[m + 1] = o.y;
            }
            float *wp = wrow + i0;
            if (ALIGNED || (full && ((uintptr_t)wp & 15) == 0)) {
                *(float4 *)wp = make_float4(out[0], out[1], out[2], out[3]);
            } else {
#pragma unroll
                for (int m = 0; m < 4; m++)
                    if (i0 + m < nx) wp[m] = out[m];
            }
        }
    }
}

// Work items are (set, block of rows[, run of pieces]).  A piece with end
// values y0, y1 is crossed by row r iff min <= y_r < max, and since the row
// values are non-decreasing those rows form one range [ra, rb), found from
// the row spacing and corrected against the item's row values.  A work list
// gives each item the run of pieces that can reach its rows (pieces are
// ordered by their lowest y per chain); a single set scans all its pieces.
//
// Roots: the run is taken in rounds of one piece per thread.  A block-wide
// prefix sum of the pieces' row counts numbers the round's (piece, row)
// pairs, and every thread takes every blockDim-th pair, its owner found by a
// binary search over the prefix sums (the owner's record, prefetched into L1
// when its row count was found, is read again by the threads that take its
// pairs) -- a piece spanning many rows is spread over the block, and the
// threads' shares stay alike.  Each root x_k is turned into its column j_k =
// first grid column with x >= x_k, and its direction is added to the item's
// difference cell (row, j_k - 1) in shared memory.
//
// Queries: one warp per row.  A suffix sum over the row's cells gives each
// query i its signed count of crossings to the right,
//   chi(i) = sum_{k : x_k > xq_i} dir_k = sum_{j >= i} D[row][j],
// in O(1) per query, whatever the number of crossings on the row.  The
// chord terms are added and w is stored (coalesced).

template <typename T>
__device__ __forceinline__ void cert_hull_cols(const T *px, int64_t p, int64_t q, const T *ax, int nx, int &c0,
                                               int &c1) {
    T lo = px[2 * p], hi = px[2 * p + 1];
    if (q >= 0) {
        lo = px[2 * q] < lo ? px[2 * q] : lo;
        hi = px[2 * q + 1] > hi ? px[2 * q + 1] : hi;
    }
    const T m = T(16) * Unit<T>::u * (fabs(lo) + fabs(hi));
    c0 = lower_bound_cols_lin(ax, nx, lo - m);
    c1 = upper_bound_cols_lin(ax, nx, hi + m);
}

// shared memory of eval2d_kernel: the difference cells (rows x stride ints),
// then the item's row values
__host__ __device__ constexpr size_t eval2d_d2_bytes(int rows, int max_nx) {
    return (sizeof(int) * (size_t)rows * (size_t)eval2d_dstride(max_nx) + 15) & ~(size_t)15;
}

// FAST: every set is one float32 chain, only w is written, and the chain set
// has fewer than 2^22 - 1 pieces (the float32 row path serves every item;
// the generic one is not compiled in).
template <typename T, bool FAST>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) eval2d_kernel(const T *__restrict__ ctrl, const int64_t *__restrict__ chain_off,
                              const T *__restrict__ piece_y, const T *__restrict__ piece_rec,
                              const Set2D *__restrict__ sets, const int4 *__restrict__ items, const Set2D single,
                              int64_t n_items,
                              unsigned long long *counter, int rows_per_item, T *__restrict__ w_out,
                              int32_t *__restrict__ chi_out, T *__restrict__ b_out, unsigned long long *cnt,
                              int *status, int max_nx, const CertArgs2D ca) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nthr = blockDim.x;
    int *D2 = (int *)smem_raw;                                              // rows_per_item x stride cells
    T *ys = (T *)(smem_raw + eval2d_d2_bytes(rows_per_item, max_nx));      // the item's row values
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = nthr >> 5;
    __shared__ long long item_sh;
    __shared__ int s_ofs[256], s_ra[256], s_wsum[8];       // a round's pair offsets and first rows
    unsigned long long nroots_thread = 0;
    // the cells start at zero; the row queries reset every cell they read
    for (int i = threadIdx.x, nc = rows_per_item * eval2d_dstride(max_nx); i < nc; i += nthr) D2[i] = 0;
    // the next item is claimed while the current one runs (thread 0 keeps the
    // claim in a register and publishes it at the end of the item)
    if (threadIdx.x == 0) item_sh = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    for (int64_t guard = 0; guard <= n_items; guard++) {
        // (thread 0 overwrites item_sh only after the barriers below, which
        // every thread reaches after this read)
        const long long item = item_sh;
        if (item >= n_items) break;
        long long next_item = 0;
        if (threadIdx.x == 0) next_item = (long long)atomicAdd(counter, 1ull);
        // one set passed by value (items are its row blocks), or a work list
        const int4 it = items ? items[item] : make_int4(0, (int)item, 0, 0);
        const Set2D S = sets ? sets[it.x] : single;
        const int set_id = sets ? it.x : -1;
        // the pieces that can reach the item's rows (a work list carries them)
        const int64_t pA = items ? (int64_t)it.z : S.p_lo, pB = items ? (int64_t)it.w : S.p_hi;
        const T *ay = (const T *)S.ay;
        const T *ax = (const T *)S.ax;
        const int nx = (int)S.nx;
        const int ds = eval2d_dstride(nx);
        const int64_t r0 = (int64_t)it.y * rows_per_item;
        const int64_t r1 = r0 + rows_per_item < S.ny ? r0 + rows_per_item : S.ny;
        const int nr = (int)(r1 - r0);
        for (int i = threadIdx.x; i < nr; i += nthr) ys[i] = ay[r0 + i];
        __syncthreads();
        const T y_first = ys[0], y_last = ys[nr - 1];
        const T inv_hy = nr > 1 && y_last > y_first ? T(nr - 1) / (y_last - y_first) : T(0);
        const T a0 = ax[0];
        const T inv_step = nx > 1 && ax[nx - 1] > ax[0] ? T(nx - 1) / (ax[nx - 1] - ax[0]) : T(0);
        for (int64_t pc = pA; pc < pB; pc += nthr) {             // block-uniform
            const int64_t p = pc + threadIdx.x;
            int ra = 0, n = 0;
            if (p < pB) {
                const T ya = piece_y[2 * p], yb = piece_y[2 * p + 1];
                const T lo = ya < yb ? ya : yb, hi = ya < yb ? yb : ya;
                const bool overlap = hi > y_first && lo <= y_last;
                int rb = 0;
                if (overlap) {
                    ra = lower_bound_rows_grid(ys, nr, y_first, inv_hy, lo);
                    rb = lower_bound_rows_grid(ys, nr, y_first, inv_hy, hi);
                    n = rb > ra ? rb - ra : 0;
                }
                if (n > 0) prefetch_rec<T>(piece_rec, p);     // read again below by the lanes taking its roots
                // certification: a row of the item within rounding of an
                // interior-extremum end value (the nearest rows to each end
                // decide whether any row is within near_window of it)
                const T win = near_window<T>(ya, yb, (T)ca.eps_abs);
                if (hi > y_first - win && lo <= y_last + win) {
                    int ca_ = ra, cb_ = rb;
                    if (!overlap) {
                        ca_ = lower_bound_rows_grid(ys, nr, y_first, inv_hy, lo);
                        cb_ = lower_bound_rows_grid(ys, nr, y_first, inv_hy, hi);
                    }
                    const bool close = (ca_ < nr && ys[ca_] - lo <= win) || (ca_ > 0 && lo - ys[ca_ - 1] <= win) ||
                                       (cb_ < nr && ys[cb_] - hi <= win) || (cb_ > 0 && hi - ys[cb_ - 1] <= win);
                    if (close) {
                        const T *ep = (const T *)ca.piece_eps + 2 * p;
                        const int2 pq = ca.piece_part[p];
#pragma unroll 1
                        for (int end = 0; end < 2; end++) {
                            const T ev = end ? ep[1] : ep[0], yv = end ? yb : ya;
                            const int q = end ? pq.y : pq.x;
                            // an exact end, or a partner in this item's run lists it
                            if (!(ev > T(0)) || (q >= 0 && q < p && q >= pA)) continue;
                            if (!(yv + T(2) * ev >= y_first && yv - T(2) * ev <= y_last)) continue;
                            int c0 = 0, c1 = 0;
                            bool have = false;
                            // the rows near_extremum selects (the same comparison), searched in a wider window
                            for (int i = lower_bound_rows_grid(ys, nr, y_first, inv_hy, yv - T(2) * ev);
                                 i < nr && ys[i] <= yv + T(2) * ev; i++) {
                                if (!(fabs(ys[i] - yv) <= ev)) continue;
                                if (!have) {
                                    cert_hull_cols<T>((const T *)ca.piece_x, p, q, ax, nx, c0, c1);
                                    have = true;
                                }
                                cert_push(ca.cert, ca.count, status, cnt, set_id, (int)(r0 + i), (int)p, q, c0, c1);
                            }
                        }
                    }
                }
            }
            // the round's (piece, row) pairs: thread i's are [s_ofs[i], s_ofs[i] + n)
            int x = n;
            for (int off = 1; off < 32; off <<= 1) {
                const int t = __shfl_up_sync(FULL, x, off);
                if (lane >= off) x += t;
            }
            if (lane == 31) s_wsum[warp] = x;
            __syncthreads();
            int tot = 0, before = 0;
            for (int w = 0; w < nwarps; w++) {
                const int sw = s_wsum[w];
                before += w < warp ? sw : 0;
                tot += sw;
            }
            s_ofs[threadIdx.x] = before + x - n;
            s_ra[threadIdx.x] = ra;
            __syncthreads();
            for (int k = threadIdx.x; k < tot; k += nthr) {
                int o = 0;                     // owner: last thread with s_ofs <= k (s_ofs[0] = 0; blocks <= 256)
#pragma unroll
                for (int step = 128; step >= 1; step >>= 1)
                    if (o + step < nthr && s_ofs[o + step] <= k) o += step;
                const int r = s_ra[o] + (k - s_ofs[o]);
                const int64_t pp = pc + o;
                T rec[PC_FIELDS];
                load_rec<T>(piece_rec, pp, rec);
                const T ya = rec[7], yb = rec[10];
                int iters;
                T tf;
                const T xr = piece_root_rec<T>(rec, ys[r], &iters, &tf);
                if (iters >= Num<T>::max_iter && status) atomicOr(status, ST_TIMEOUT);
                nroots_thread += (unsigned long long)iters << 32 | 1ull;
                const int col = lower_bound_cols(ax, nx, a0, inv_step, xr);     // its column
                if (col > 0) atomicAdd(&D2[r * ds + col - 1], yb > ya ? 1 : -1);
                const T band = root_band<T>(rec, ys[r], tf);
                const bool amb = !(band < T(INFINITY)) || (col > 0 && ax[col - 1] >= xr - band) ||
                                 (col < nx && ax[col] <= xr + band);
                if (amb && !near_extremum<T>(ys[r], ya, yb, (const T *)ca.piece_eps + 2 * pp, (T)ca.eps_abs)) {
                    int c0, c1;
                    T xlo, xhi;
                    if (cert_interval<T>(rec, ys[r], tf, xr, xlo, xhi)) {
                        c0 = lower_bound_cols_lin(ax, nx, xlo);
                        c1 = upper_bound_cols_lin(ax, nx, xhi);
                    } else {
                        cert_hull_cols<T>((const T *)ca.piece_x, pp, -1, ax, nx, c0, c1);
                    }
                    cert_push(ca.cert, ca.count, status, cnt, set_id, (int)(r0 + r), (int)pp, -1, c0, c1);
                }
            }
            // s_wsum, s_ofs, s_ra are rewritten by the next round, and the
            // row queries read the cells (when the run is empty no cell was
            // written and no barrier is needed)
            __syncthreads();
        }
        // queries: one warp per row
        if (FAST || (sizeof(T) == 4 && S.c_hi - S.c_lo == 1 && !chi_out && !b_out && w_out && pB - pA < (1 << 22) - 1)) {
            const float *sp = (const float *)ctrl + 2 * chain_off[S.c_lo];
            const float *ep = (const float *)ctrl + 2 * (chain_off[S.c_lo + 1] - 1);
            const float spx = sp[0], spy = sp[1], epx = ep[0], epy = ep[1];
            float *w0 = (float *)w_out + S.out_off + r0 * S.nx;
            const bool aligned = (nx & 255) == 0 && ((uintptr_t)ax & 15) == 0 && ((uintptr_t)w0 & 15) == 0 &&
                                 pB - pA < 32767;
            if (aligned) {
                for (int r = warp; r < nr; r += nwarps)
                    row_queries_f32<true>((const float *)ax, nx, D2 + r * ds, (float)ys[r], spx, spy, epx, epy,
                                          w0 + (int64_t)r * nx, lane, pB - pA < 32767);
            } else {
                for (int r = warp; r < nr; r += nwarps)
                    row_queries_f32<false>((const float *)ax, nx, D2 + r * ds, (float)ys[r], spx, spy, epx, epy,
                                           w0 + (int64_t)r * nx, lane, pB - pA < 32767);
            }
        } else if (!FAST) {
            for (int r = warp; r < nr; r += nwarps)
                row_queries<T>(S, ctrl, chain_off, ax, nx, D2 + r * ds, ys[r], r0 + r, lane, w_out, chi_out, b_out,
                               ca, status, cnt, set_id);
        }
        if (threadIdx.x == 0) item_sh = next_item;
        __syncthreads();
    }
    if (cnt && nroots_thread) {
        atomicAdd(&cnt[CNT_ROOTS], nroots_thread & 0xffffffffull);
        atomicAdd(&cnt[CNT_NEWTON], nroots_thread >> 32);
    }
}

// Certification pass: one warp per listed (set, row, piece [, partner],
// columns).  Per piece, once: the float path's own crossing (the same row
// test and the same root as eval2d_kernel; a query counts it iff xq < x) and
// the float64 one (piece_exact); then the lanes take the columns, and where
// the two counts differ the query's count, and w, are corrected by the
// difference.  Entries are rare (a crossing within its error bound of a
// query, or a row within rounding of an extremum value).
// An entry with piece index -2 - c lists the chord of chain c instead: its
// side is taken exactly (chord_counts) and only the count changes (w is the
// same on both sides of the chord).
template <typename T>
__global__ void __launch_bounds__(128) eval2d_cert_kernel(
    const T *__restrict__ ctrl, const int64_t *__restrict__ chain_off, const T *__restrict__ piece_y,
    const T *__restrict__ piece_rec, const int64_t *__restrict__ piece_seg, const double2 *__restrict__ piece_u,
    const Set2D *__restrict__ sets, const Set2D single, const int4 *__restrict__ cert,
    const int32_t *__restrict__ cert_count, T *w_out, int32_t *chi_out, unsigned long long *cnt) {
    int n = *cert_count;
    if (n > GWN_CERT_CAP) n = GWN_CERT_CAP;
    const int lane = threadIdx.x & 31;
    // consecutive entries go to different blocks (and so to different SMs:
    // an entry's float64 bisection is bound by the SM's float64 rate)
    const int warp = (threadIdx.x >> 5) * gridDim.x + blockIdx.x, nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < n; i += nwarps) {               // warp-uniform
        const int4 a = cert[2 * i], b = cert[2 * i + 1];
        const Set2D S = a.x >= 0 ? sets[a.x] : single;
        const T *ax = (const T *)S.ax;
        const T yr = ((const T *)S.ay)[a.y];
        if (a.z <= -2) {                                    // a chord side
            if (lane == 0 && chi_out) {
                for (int c = b.x; c < b.y; c++) {
                    const int2 fe = chord_counts<T>(ctrl, chain_off, (int64_t)(-2 - a.z), ax[c], yr);
                    if (fe.x != fe.y) {
                        atomicAdd(&chi_out[S.out_off + (int64_t)a.y * S.nx + c], fe.y - fe.x);
                        if (cnt) atomicAdd(&cnt[CNT_CERT_FIX], 1ull);
                    }
                }
            }
            continue;
        }
        T fx[2];
        int fdir[2];
        ExactCross ec[2];
        for (int k = 0; k < 2; k++) {
            const int pp = k ? a.w : a.z;
            fdir[k] = 0;
            fx[k] = T(0);
            ec[k].dir = 0;
            ec[k].x = 0.0;
            if (pp < 0) continue;
            const T ya = piece_y[2 * pp], yb = piece_y[2 * pp + 1];
            const T lo = ya < yb ? ya : yb, hi = ya < yb ? yb : ya;
            if (lo <= yr && yr < hi) {
                T rec[PC_FIELDS];
                load_rec<T>(piece_rec, pp, rec);
                int iters;
                fx[k] = piece_root_rec<T>(rec, yr, &iters);
                fdir[k] = yb > ya ? 1 : -1;
            }
            ec[k] = piece_exact_warp<T>(ctrl, piece_seg[pp], piece_u[pp], (double)yr);
        }
        int nfix = 0;
        for (int c = b.x + lane; c < b.y; c += 32) {
            const T xq = ax[c];
            int f = 0, e = 0;
            for (int k = 0; k < 2; k++) {
                if (fdir[k] && xq < fx[k]) f += fdir[k];
                if (ec[k].dir && ec[k].x > (double)xq) e += ec[k].dir;
            }
            if (e != f) {
                const int64_t o = S.out_off + (int64_t)a.y * S.nx + c;
                if (w_out) atomicAdd(&w_out[o], (T)(e - f));
                if (chi_out) atomicAdd(&chi_out[o], e - f);
                nfix++;
            }
        }
        if (cnt && nfix) atomicAdd(&cnt[CNT_CERT_FIX], (unsigned long long)nfix);
    }
}

size_t eval2d_smem(int dtype, int64_t max_nx, int rows) {
    return eval2d_d2_bytes(rows, (int)max_nx) + (dtype == GWN_F64 ? 8 : 4) * (size_t)rows;
}

cudaError_t launch_eval2d_items(const ChainSet &cs, const Set2D *d_sets, const int4 *d_items, const Set2D *single,
                                int64_t n_items, unsigned long long *d_counter, int rows_per_item, int threads,
                                int64_t max_nx, void *w_out, int32_t *chi_out, void *b_out, unsigned long long *cnt,
                                int *status, int sm_count, cudaStream_t st, int4 *cert, int32_t *cert_count) {
    if (n_items == 0) return cudaSuccess;
    if (!d_sets && !single) return cudaErrorInvalidValue;
    if (rows_per_item < 1 || rows_per_item > MAX_ROWS || threads < 32 || threads > 256 || threads % 32)
        return cudaErrorInvalidValue;
    Set2D s0;
    memset(&s0, 0, sizeof(s0));
    if (single) s0 = *single;
    if (!cert || !cert_count) return cudaErrorInvalidValue;
    if (max_nx < 1 || max_nx > 16384) return cudaErrorInvalidValue;
    size_t smem = eval2d_smem(cs.dtype, max_nx, rows_per_item);
    if (smem > EVAL2D_SMEM_MAX) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cert_count, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    CertArgs2D ca;
    ca.eps_abs = cs.eps_abs;
    ca.piece_eps = cs.piece_eps;
    ca.piece_part = cs.piece_part;
    ca.piece_x = cs.piece_xT;
    ca.cert = cert;
    ca.count = cert_count;
    // persistent grid: as many blocks as fit on the device at once; the
    // instantiation without the generic row path when the float32
    // single-chain path serves every item
    const bool fast = cs.dtype != GWN_F64 && !chi_out && !b_out && w_out && cs.n_pieces < (1 << 22) - 1 &&
                      (d_sets ? true : s0.c_hi - s0.c_lo == 1);
    const void *kfn = cs.dtype == GWN_F64 ? (const void *)eval2d_kernel<double, false>
                      : fast ? (const void *)eval2d_kernel<float, true> : (const void *)eval2d_kernel<float, false>;
    int per_sm = 0;
    e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t blocks = (int64_t)sm_count * per_sm;
    if (blocks > n_items) blocks = n_items;
    if (cs.dtype == GWN_F64) {
        eval2d_kernel<double, false><<<(unsigned)blocks, threads, smem, st>>>(
            (const double *)cs.ctrl, cs.chain_off,
            (const double *)cs.piece_yT, (const double *)cs.piece_rec, d_sets, d_items, s0, n_items, d_counter,
            rows_per_item, (double *)w_out,
            chi_out, (double *)b_out, cnt, status, (int)max_nx, ca);
    } else if (fast) {
        eval2d_kernel<float, true><<<(unsigned)blocks, threads, smem, st>>>(
            (const float *)cs.ctrl, cs.chain_off,
            (const float *)cs.piece_yT, (const float *)cs.piece_rec, d_sets, d_items, s0, n_items, d_counter,
            rows_per_item, (float *)w_out,
            chi_out, (float *)b_out, cnt, status, (int)max_nx, ca);
    } else {
        eval2d_kernel<float, false><<<(unsigned)blocks, threads, smem, st>>>(
            (const float *)cs.ctrl, cs.chain_off,
            (const float *)cs.piece_yT, (const float *)cs.piece_rec, d_sets, d_items, s0, n_items, d_counter,
            rows_per_item, (float *)w_out,
            chi_out, (float *)b_out, cnt, status, (int)max_nx, ca);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // certification pass: a small fixed grid over the (rare) listed entries
    if (cs.dtype == GWN_F64)
        eval2d_cert_kernel<double><<<(unsigned)((sm_count > 0 ? sm_count : 152) * 2), 128, 0, st>>>((const double *)cs.ctrl, cs.chain_off, (const double *)cs.piece_yT,
                                                      (const double *)cs.piece_rec, cs.piece_seg, cs.piece_u, d_sets,
                                                      s0, cert, cert_count, (double *)w_out, chi_out, cnt);
    else
        eval2d_cert_kernel<float><<<(unsigned)((sm_count > 0 ? sm_count : 152) * 2), 128, 0, st>>>((const float *)cs.ctrl, cs.chain_off, (const float *)cs.piece_yT,
                                                     (const float *)cs.piece_rec, cs.piece_seg, cs.piece_u, d_sets,
                                                     s0, cert, cert_count, (float *)w_out, chi_out, cnt);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Point queries (no ray reuse): one +x ray per query.  The query's y picks a
// bucket of the y-bucket index; for each listed piece the exact half-open
// y-test decides whether the ray's line crosses it, and the piece's
// conservative x-range decides most crossings outright (entirely right of the
// query: counted; entirely left: not); only a piece whose x-range straddles
// the query needs its root.  Then the chord terms of every chain.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ int bucket_of_dev(T y, T y0, T inv_h, int nb) {
    T v = (y - y0) * inv_h;
    if (!(v >= T(0))) return 0;
    if (v >= T(nb)) return nb - 1;
    int b = (int)v;
    return b < nb ? b : nb - 1;
}

// One listed piece seen from a point query: its contribution to the float
// count, and whether that contribution is uncertain (a row within rounding
// of an interior-extremum end value, or a root whose error bound contains the
// query).  The same tests serve the counting loop and the listing loop.
template <typename T>
__device__ __forceinline__ int point_piece(const T *__restrict__ piece_y, const T *__restrict__ piece_rec,
                                           const T *__restrict__ piece_x, const T *__restrict__ piece_eps,
                                           T eps_abs, int p, T px, T py, int *status, int &nroots, bool &unc) {
    unc = false;
    const T ya = piece_y[2 * p], yb = piece_y[2 * p + 1];
    const T lo = ya < yb ? ya : yb, hi = ya < yb ? yb : ya;
    const bool crossed = lo <= py && py < hi;
    const bool near = near_extremum<T>(py, ya, yb, piece_eps + 2 * p, eps_abs);
    unc = near;
    if (!crossed) return 0;
    const int dir = yb > ya ? 1 : -1;
    if (px < piece_x[2 * p]) return dir;                      // crossing certainly to the right
    if (px >= piece_x[2 * p + 1]) return 0;                   // certainly not to the right
    T rec[PC_FIELDS];
    load_rec<T>(piece_rec, p, rec);
    int iters;
    T tf;
    const T x = piece_root_rec<T>(rec, py, &iters, &tf);
    if (iters >= Num<T>::max_iter && status) atomicOr(status, ST_TIMEOUT);
    nroots++;
    if (!near && !(fabs(x - px) > root_band<T>(rec, py, tf))) {
        T xlo, xhi;
        unc = !cert_interval<T>(rec, py, tf, x, xlo, xhi) || (xlo <= px && px <= xhi);
    }
    return x > px ? dir : 0;
}

// Certification: the uncertain (query, piece) pairs are listed for
// eval2d_points_cert_kernel, which decides them in float64 from the control
// points and corrects the count; the float contribution made here stays in
// the count until then.  The counting loop only notes that a query has such
// a pair; the (rare) listing loop runs the same tests again and lists them,
// so the hot loop has no memory side effects.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 8 : 3) eval2d_points_kernel(
    const T *__restrict__ ctrl, const int64_t *__restrict__ chain_off, int64_t n_chains,
    const T *__restrict__ piece_y, const T *__restrict__ piece_rec,
    const T *__restrict__ piece_x, const int32_t *__restrict__ bucket_off, const int32_t *__restrict__ bucket_idx,
    int nb, T y0, T inv_h, const T *__restrict__ pts, int64_t n, T *__restrict__ w_out, int32_t *__restrict__ chi_out,
    T *__restrict__ b_out, unsigned long long *cnt, int *status, const T *__restrict__ piece_eps, T eps_abs,
    int4 *cert, int32_t *cert_count, const int32_t *__restrict__ order) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    // the queries in bucket order when an order is given (the warps then walk
    // the same bucket lists), else as given
    const int64_t i = order ? (int64_t)order[k] : k;
    const T px = pts[2 * i], py = pts[2 * i + 1];
    const int b = bucket_of_dev<T>(py, y0, inv_h, nb);
    int chi = 0, nroots = 0;
    bool any_unc = false;
    for (int j = bucket_off[b]; j < bucket_off[b + 1]; j++) {
        bool unc;
        chi += point_piece<T>(piece_y, piece_rec, piece_x, piece_eps, eps_abs, bucket_idx[j], px, py, status, nroots,
                              unc);
        any_unc = any_unc || unc;
    }
    if (any_unc) {
        int nr2 = 0;
        for (int j = bucket_off[b]; j < bucket_off[b + 1]; j++) {
            bool unc;
            point_piece<T>(piece_y, piece_rec, piece_x, piece_eps, eps_abs, bucket_idx[j], px, py, nullptr, nr2, unc);
            if (unc) cert_push(cert, cert_count, status, cnt, -2, (int)i, bucket_idx[j], -1, 0, 1);
        }
    }
    if (cnt && nroots) atomicAdd(&cnt[CNT_ROOTS], (unsigned long long)nroots);
    Set2D S;
    S.c_lo = 0;
    S.c_hi = n_chains;
    const T A = chord_angles<T>(ctrl, chain_off, S, px, py, chi, [&](int64_t c) {
        if (chi_out) cert_push(cert, cert_count, status, cnt, -3, (int)i, (int)c, -1, 0, 1);
    });
    if (w_out) w_out[i] = w_of<T>(chi, A);
    if (chi_out) chi_out[i] = chi;
    if (b_out) b_out[i] = Num<T>::mul(A, Num<T>::inv2pi);
}

// Listed (query, piece) pairs of the point path: the float path's own
// decision (the same tests as eval2d_points_kernel, including its x-range
// shortcuts) against the float64 one; the count, and w, corrected by the
// difference.
template <typename T>
__global__ void __launch_bounds__(128) eval2d_points_cert_kernel(
    const T *__restrict__ ctrl, const int64_t *__restrict__ chain_off, const T *__restrict__ piece_y,
    const T *__restrict__ piece_rec, const T *__restrict__ piece_x, const int64_t *__restrict__ piece_seg,
    const double2 *__restrict__ piece_u, const T *__restrict__ pts, const int4 *__restrict__ cert,
    const int32_t *__restrict__ cert_count, T *w_out, int32_t *chi_out, unsigned long long *cnt) {
    int n = *cert_count;
    if (n > GWN_CERT_CAP) n = GWN_CERT_CAP;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int4 a = cert[2 * k];
        const int64_t i = a.y;
        const int p = a.z;
        const T px = pts[2 * i], py = pts[2 * i + 1];
        if (a.x == -3) {                                    // the chord of chain p: the count only
            const int2 fe = chord_counts<T>(ctrl, chain_off, (int64_t)p, px, py);
            if (fe.x != fe.y && chi_out) {
                atomicAdd(&chi_out[i], fe.y - fe.x);
                if (cnt) atomicAdd(&cnt[CNT_CERT_FIX], 1ull);
            }
            continue;
        }
        const T ya = piece_y[2 * p], yb = piece_y[2 * p + 1];
        const T lo = ya < yb ? ya : yb, hi = ya < yb ? yb : ya;
        int f = 0;
        if (lo <= py && py < hi) {
            const int dir = yb > ya ? 1 : -1;
            if (px < piece_x[2 * p]) {
                f = dir;
            } else if (px < piece_x[2 * p + 1]) {
                T rec[PC_FIELDS];
                load_rec<T>(piece_rec, p, rec);
                int iters;
                const T x = piece_root_rec<T>(rec, py, &iters);
                f = x > px ? dir : 0;
            }
        }
        const ExactCross ec = piece_exact<T>(ctrl, piece_seg[p], piece_u[p], (double)py);
        const int e = ec.dir && ec.x > (double)px ? ec.dir : 0;
        if (e != f) {
            if (w_out) atomicAdd(&w_out[i], (T)(e - f));
            if (chi_out) atomicAdd(&chi_out[i], e - f);
            if (cnt) atomicAdd(&cnt[CNT_CERT_FIX], 1ull);
        }
    }
}

// Bucket order of the point queries (a counting sort, one launch per step):
// count the queries per bucket, an exclusive scan of the counts (one block),
// then each query takes the next slot of its bucket.  The order within a
// bucket is arbitrary; every query's result is the same in any order.
template <typename T>
__global__ void points_bucket_count_kernel(const T *__restrict__ pts, int64_t n, T y0, T inv_h, int nb,
                                           int32_t *__restrict__ count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&count[bucket_of_dev<T>(pts[2 * i + 1], y0, inv_h, nb)], 1);
}
__global__ void __launch_bounds__(1024) points_bucket_scan_kernel(int32_t *__restrict__ count, int nb) {
    // count[0 .. nb) -> exclusive prefix sums, in chunks of 1024 with a carry
    __shared__ int32_t s_w[32];
    __shared__ int32_t s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? count[i] : 0;
        int x = v;
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += t;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        int before = s_carry, tot = s_carry;
        for (int w = 0; w < 32; w++) {
            const int sw = s_w[w];
            before += w < warp ? sw : 0;
            tot += sw;
        }
        if (i < nb) count[i] = before + x - v;
        __syncthreads();                              // every thread has read s_w and s_carry
        if (threadIdx.x == 0) s_carry = tot;
        __syncthreads();
    }
}
template <typename T>
__global__ void points_bucket_scatter_kernel(const T *__restrict__ pts, int64_t n, T y0, T inv_h, int nb,
                                             int32_t *__restrict__ next, int32_t *__restrict__ order) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        order[atomicAdd(&next[bucket_of_dev<T>(pts[2 * i + 1], y0, inv_h, nb)], 1)] = (int32_t)i;
}

size_t eval2d_points_order_bytes(const ChainSet &cs, int64_t n) {
    if (n < EVAL2D_POINTS_ORDER_MIN || cs.n_buckets < 2 || cs.n_buckets > EVAL2D_POINTS_ORDER_MAX_BUCKETS) return 0;
    return sizeof(int32_t) * ((size_t)n + (size_t)cs.n_buckets);
}

cudaError_t launch_eval2d_points(const ChainSet &cs, const QuerySrc &q, void *w_out, int32_t *chi_out, void *b_out,
                                 unsigned long long *cnt, int *status, cudaStream_t st, int4 *cert,
                                 int32_t *cert_count, int32_t *order_buf, int sm_count) {
    if (q.n == 0) return cudaSuccess;
    if (!cert || !cert_count) return cudaErrorInvalidValue;
    int64_t blocks = (q.n + 255) / 256;
    if (blocks > 0x7fffffff || q.n > 0x7fffffff) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(cert_count, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    // bucket order (order_buf: n + n_buckets ints from eval2d_points_order_bytes, or null)
    const int32_t *order = nullptr;
    if (order_buf && eval2d_points_order_bytes(cs, q.n) > 0) {
        int32_t *count = order_buf + q.n;
        const int nb = (int)cs.n_buckets;
        const unsigned g = (unsigned)std::min<int64_t>(blocks, (int64_t)(sm_count > 0 ? sm_count : 152) * 8);
        e = cudaMemsetAsync(count, 0, sizeof(int32_t) * nb, st);
        if (e != cudaSuccess) return e;
        if (cs.dtype == GWN_F64)
            points_bucket_count_kernel<double><<<g, 256, 0, st>>>(q.pts64, q.n, cs.bucket_y0, cs.bucket_inv_h, nb, count);
        else
            points_bucket_count_kernel<float><<<g, 256, 0, st>>>(q.pts, q.n, (float)cs.bucket_y0, (float)cs.bucket_inv_h,
                                                                 nb, count);
        points_bucket_scan_kernel<<<1, 1024, 0, st>>>(count, nb);
        if (cs.dtype == GWN_F64)
            points_bucket_scatter_kernel<double><<<g, 256, 0, st>>>(q.pts64, q.n, cs.bucket_y0, cs.bucket_inv_h, nb,
                                                                    count, order_buf);
        else
            points_bucket_scatter_kernel<float><<<g, 256, 0, st>>>(q.pts, q.n, (float)cs.bucket_y0,
                                                                   (float)cs.bucket_inv_h, nb, count, order_buf);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        order = order_buf;
    }
    if (cs.dtype == GWN_F64) {
        eval2d_points_kernel<double><<<(unsigned)blocks, 256, 0, st>>>(
            (const double *)cs.ctrl, cs.chain_off, cs.n_chains, (const double *)cs.piece_yT,
            (const double *)cs.piece_rec, (const double *)cs.piece_xT, cs.bucket_off, cs.bucket_idx, cs.n_buckets,
            cs.bucket_y0, cs.bucket_inv_h, q.pts64, q.n, (double *)w_out, chi_out, (double *)b_out, cnt, status,
            (const double *)cs.piece_eps, cs.eps_abs, cert, cert_count, order);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            eval2d_points_cert_kernel<double><<<64, 128, 0, st>>>(
                (const double *)cs.ctrl, cs.chain_off, (const double *)cs.piece_yT, (const double *)cs.piece_rec,
                (const double *)cs.piece_xT, cs.piece_seg, cs.piece_u, q.pts64, cert, cert_count, (double *)w_out,
                chi_out, cnt);
    } else {
        eval2d_points_kernel<float><<<(unsigned)blocks, 256, 0, st>>>(
            (const float *)cs.ctrl, cs.chain_off, cs.n_chains, (const float *)cs.piece_yT,
            (const float *)cs.piece_rec, (const float *)cs.piece_xT, cs.bucket_off, cs.bucket_idx, cs.n_buckets,
            (float)cs.bucket_y0, (float)cs.bucket_inv_h, q.pts, q.n, (float *)w_out, chi_out, (float *)b_out, cnt,
            status, (const float *)cs.piece_eps, (float)cs.eps_abs, cert, cert_count, order);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            eval2d_points_cert_kernel<float><<<64, 128, 0, st>>>(
                (const float *)cs.ctrl, cs.chain_off, (const float *)cs.piece_yT, (const float *)cs.piece_rec,
                (const float *)cs.piece_xT, cs.piece_seg, cs.piece_u, q.pts, cert, cert_count, (float *)w_out,
                chi_out, cnt);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// cubic Bernstein polynomial and its derivative (comparator quadrature)
template <typename T>
__device__ __forceinline__ T bern(T p0, T p1, T p2, T p3, T u) {
    T v = T(1) - u;
    return v * v * v * p0 + T(3) * u * v * v * p1 + T(3) * u * u * v * p2 + u * u * u * p3;
}
template <typename T>
__device__ __forceinline__ T dbern(T p0, T p1, T p2, T p3, T u) {
    T v = T(1) - u;
    return T(3) * (v * v * (p1 - p0) + T(2) * u * v * (p2 - p1) + u * u * (p3 - p2));
}

// ---------------------------------------------------------------------------
// brute-force comparator: per (query, segment) the subtended angle by
// Gauss-Legendre quadrature on 2^L equal subintervals, L doubled until two
// consecutive levels agree to the working tolerance (capped).
// ---------------------------------------------------------------------------
__constant__ double GL8_X[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290, -0.1834346424956498,
                                0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
__constant__ double GL8_W[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873, 0.3626837833783620,
                                0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};

template <typename T>
__device__ T seg_angle_gl(const T *c, T px, T py, int nsub) {
    T acc = T(0);
    T h = T(1) / (T)nsub;
    for (int s = 0; s < nsub; s++) {
        T a = s * h;
        for (int k = 0; k < 8; k++) {
            T u = a + T(0.5) * h * (T(1) + (T)GL8_X[k]);
            T x = bern(c[0], c[2], c[4], c[6], u) - px, y = bern(c[1], c[3], c[5], c[7], u) - py;
            T dx = dbern(c[0], c[2], c[4], c[6], u), dy = dbern(c[1], c[3], c[5], c[7], u);
            acc += (T)GL8_W[k] * (x * dy - y * dx) / (x * x + y * y);
        }
    }
    return acc * T(0.5) * h;
}

template <typename T>
__global__ void bruteforce2d_kernel(const T *__restrict__ ctrl, const int64_t *__restrict__ chain_off, int64_t n_chains,
                                    const T *__restrict__ ax, const T *__restrict__ ay, int64_t nx, int64_t n,
                                    T *__restrict__ w_out, T tol) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T px = ax[i % nx], py = ay[i / nx];
    T total = T(0);
    for (int64_t ch = 0; ch < n_chains; ch++) {
        for (int64_t s = chain_off[ch]; s + 3 < chain_off[ch + 1]; s += 3) {
            T c[8];
            for (int k = 0; k < 8; k++) c[k] = ctrl[2 * s + k];
            int nsub = 1;
            T prev = seg_angle_gl<T>(c, px, py, nsub);
            for (int lvl = 0; lvl < 10; lvl++) {
                nsub *= 2;
                T cur = seg_angle_gl<T>(c, px, py, nsub);
                T dlt = cur - prev;
                prev = cur;
                if ((dlt < T(0) ? -dlt : dlt) <= tol) break;
            }
            total += prev;
        }
    }
    w_out[i] = total * Num<T>::inv2pi;
}

cudaError_t launch_bruteforce2d(const ChainSet &cs, const QuerySrc &q, void *w_out, int sm_count, cudaStream_t st) {
    (void)sm_count;
    if (q.n == 0) return cudaSuccess;
    int64_t blocks = (q.n + 127) / 128;
    if (cs.dtype == GWN_F64)
        bruteforce2d_kernel<double><<<(unsigned)blocks, 128, 0, st>>>((const double *)cs.ctrl, cs.chain_off,
                                                                       cs.n_chains, q.ax64[0], q.ax64[1], q.dims[0],
                                                                       q.n, (double *)w_out, 1e-13);
    else
        bruteforce2d_kernel<float><<<(unsigned)blocks, 128, 0, st>>>((const float *)cs.ctrl, cs.chain_off, cs.n_chains,
                                                                      q.ax[0], q.ax[1], q.dims[0], q.n,
                                                                      (float *)w_out, 1e-6f);
    return cudaGetLastError();
}

}  // namespace gwn
