/*
 * gwn_oracle.c -- FP64 CPU reference for generalized winding numbers.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file;
 * it is used by the tests, by the smoke check and by the CPU baseline leg of
 * the bench.  It shares no code with the CUDA library.
 *
 * Every floating-point input is a float32 value promoted exactly to double.
 * Exact predicate signs are computed with integer arithmetic on the float32
 * bit patterns (a fixed-width big integer), after a plain float64 filter.
 *
 * Contents (paper sections cited per function):
 *   - 3D definition: sum of per-triangle solid angles (Background, 3D GWN).
 *   - signed crossing count of one ray (Eq. chi) by brute force over all
 *     triangles with exact orientation predicates and a symbolic perturbation
 *     of the ray direction.
 *   - boundary edge multiplicities and the boundary term relative to one ray
 *     direction (one-shot algorithm, Lemma 1/Lemma 2 and the closure used in
 *     the proof of Appendix A).
 *   - gradient of the 3D definition (analytic derivative of the per-triangle
 *     solid angle, chain rule).
 *   - 2D definition: per-segment adaptive Gauss-Kronrod quadrature of the
 *     subtended angle (Background, 2D GWN).
 *   - 2D one-shot by Algorithm 1 (project the boundary points on the circle,
 *     two regions, one ray in the largest region, pairwise difference, sum).
 *   - 2D closed form relative to the +x ray (chord closure).
 *   - 3D one-shot by Algorithm 1 literally (arrangement of the projected
 *     boundary on the unit sphere, region areas, one ray in the largest
 *     region, counts propagated across the arcs by Lemma 2, area-weighted
 *     sum of Eq. wn_discrete_sum), for tiny inputs.
 */
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_API __attribute__((visibility("default")))

/* ======================================================================== */
/* Exact sign of a sum of products of float32 values                        */
/* ======================================================================== */
/* A float32 x equals mant * 2^ex with |mant| < 2^24.  A product of up to
 * three such numbers is an integer of at most 72 bits times a power of two;
 * a sum of such products is accumulated exactly in a two's-complement big
 * integer of BIG_LIMBS 64-bit words.  The exponent span of float32 triple
 * products is below 800 bits, so 16 limbs (1024 bits) always suffice. */
#define BIG_LIMBS 18

typedef struct { uint64_t w[BIG_LIMBS]; } big_t;

static void split_f32(float x, int64_t *mant, int *ex) {
    if (x == 0.0f) { *mant = 0; *ex = 0; return; }
    int k;
    double f = frexp((double)x, &k);           /* x = f * 2^k, 0.5 <= |f| < 1 */
    *mant = (int64_t)ldexp(f, 24);              /* exact: float has 24 bits */
    *ex = k - 24;
}

typedef struct { __int128 mant; int ex; } term_t;

/* add (mag << shift) with sign to the accumulator */
static void big_add_shifted(big_t *acc, unsigned __int128 mag, int neg, int shift) {
    uint64_t limbs[BIG_LIMBS];
    memset(limbs, 0, sizeof limbs);
    int q = shift / 64, r = shift % 64;
    uint64_t lo = (uint64_t)mag, hi = (uint64_t)(mag >> 64);
    /* place the 128-bit magnitude at bit offset shift (spans up to 3 limbs) */
    uint64_t parts[3];
    if (r == 0) { parts[0] = lo; parts[1] = hi; parts[2] = 0; }
    else {
        parts[0] = lo << r;
        parts[1] = (hi << r) | (lo >> (64 - r));
        parts[2] = hi >> (64 - r);
    }
    for (int i = 0; i < 3; i++)
        if (q + i < BIG_LIMBS) limbs[q + i] = parts[i];
    if (neg) {           /* two's complement negate of the full width */
        unsigned __int128 carry = 1;
        for (int i = 0; i < BIG_LIMBS; i++) {
            unsigned __int128 v = (unsigned __int128)(~limbs[i]) + carry;
            limbs[i] = (uint64_t)v;
            carry = v >> 64;
        }
    }
    unsigned __int128 carry = 0;
    for (int i = 0; i < BIG_LIMBS; i++) {
        unsigned __int128 v = (unsigned __int128)acc->w[i] + limbs[i] + carry;
        acc->w[i] = (uint64_t)v;
        carry = v >> 64;
    }
}

static int big_sign(const big_t *acc) {
    if ((int64_t)acc->w[BIG_LIMBS - 1] < 0) return -1;
    for (int i = 0; i < BIG_LIMBS; i++) if (acc->w[i]) return 1;
    return 0;
}

/* exact sign of sum_i terms[i] */
static int exact_sign_terms(const term_t *t, int n) {
    int emin = 1 << 30;
    for (int i = 0; i < n; i++) if (t[i].mant != 0 && t[i].ex < emin) emin = t[i].ex;
    if (emin == (1 << 30)) return 0;
    big_t acc;
    memset(&acc, 0, sizeof acc);
    for (int i = 0; i < n; i++) {
        if (t[i].mant == 0) continue;
        int neg = t[i].mant < 0;
        unsigned __int128 mag = neg ? (unsigned __int128)(-t[i].mant) : (unsigned __int128)t[i].mant;
        big_add_shifted(&acc, mag, neg, t[i].ex - emin);
    }
    return big_sign(&acc);
}

/* A factor is the exact difference x - y of two float32 values (y may be 0). */
typedef struct { float x, y; } fac_t;

/* append the expansion of sgn * f0 * f1 [* f2] (each factor a difference) */
static int expand_product(term_t *out, int sgn, const fac_t *f, int nf) {
    int n = 0;
    int combos = 1 << nf;
    for (int c = 0; c < combos; c++) {
        int s = sgn;
        __int128 m = 1;
        int e = 0;
        int zero = 0;
        for (int k = 0; k < nf; k++) {
            float v = (c >> k & 1) ? f[k].y : f[k].x;
            if ((c >> k) & 1) s = -s;
            int64_t mm; int ee;
            split_f32(v, &mm, &ee);
            if (mm == 0) { zero = 1; break; }
            m *= mm; e += ee;
        }
        if (zero) continue;
        out[n].mant = s < 0 ? -m : m;
        out[n].ex = e;
        n++;
    }
    return n;
}

static const int PERM3[6][3] = {{0,1,2},{1,2,0},{2,0,1},{0,2,1},{2,1,0},{1,0,2}};
static const int PSGN3[6] = {1, 1, 1, -1, -1, -1};

/* exact sign of det[A-P, B-P, D] */
static int exact_det_abd(const float *A, const float *B, const float *P, const float *D) {
    term_t t[6 * 8];
    int n = 0;
    for (int k = 0; k < 6; k++) {
        const int *s = PERM3[k];
        fac_t f[3] = {{A[s[0]], P[s[0]]}, {B[s[1]], P[s[1]]}, {D[s[2]], 0.0f}};
        n += expand_product(t + n, PSGN3[k], f, 3);
    }
    return exact_sign_terms(t, n);
}

/* exact sign of ((A-P) x (B-P))_k */
static int exact_cross_comp(const float *A, const float *B, const float *P, int k) {
    int i = (k + 1) % 3, j = (k + 2) % 3;
    term_t t[8];
    int n = 0;
    fac_t f1[2] = {{A[i], P[i]}, {B[j], P[j]}};
    fac_t f2[2] = {{A[j], P[j]}, {B[i], P[i]}};
    n += expand_product(t + n, 1, f1, 2);
    n += expand_product(t + n, -1, f2, 2);
    return exact_sign_terms(t, n);
}

/* exact sign of ((X-P) x D)_k */
static int exact_cross_xd(const float *X, const float *P, const float *D, int k) {
    int i = (k + 1) % 3, j = (k + 2) % 3;
    term_t t[4];
    int n = 0;
    fac_t f1[2] = {{X[i], P[i]}, {D[j], 0.0f}};
    fac_t f2[2] = {{X[j], P[j]}, {D[i], 0.0f}};
    n += expand_product(t + n, 1, f1, 2);
    n += expand_product(t + n, -1, f2, 2);
    return exact_sign_terms(t, n);
}

/* X lies exactly on the forward ray from P: (X-P) x D = 0 and (X-P).D > 0 */
static int on_forward_ray(const float *X, const float *P, const float *D) {
    double dot = ((double)X[0] - P[0]) * D[0] + ((double)X[1] - P[1]) * D[1] + ((double)X[2] - P[2]) * D[2];
    if (!(dot > 0.0)) return 0;
    for (int k = 0; k < 3; k++)
        if (exact_cross_xd(X, P, D, k) != 0) return 0;
    return 1;
}

/* exact sign of det[V0-P, V1-P, V2-P] */
static int exact_orient(const float *V0, const float *V1, const float *V2, const float *P) {
    term_t t[6 * 8];
    int n = 0;
    for (int k = 0; k < 6; k++) {
        const int *s = PERM3[k];
        fac_t f[3] = {{V0[s[0]], P[s[0]]}, {V1[s[1]], P[s[1]]}, {V2[s[2]], P[s[2]]}};
        n += expand_product(t + n, PSGN3[k], f, 3);
    }
    return exact_sign_terms(t, n);
}

/* ---- float64 filters: accept the float64 sign only when |value| exceeds a
 * generous bound (16 ulp of the permanent); otherwise use the exact sign. */
static const double FILTER_U = 16.0 * 1.1102230246251565e-16;

static int sign_det_abd(const float *A, const float *B, const float *P, const float *D) {
    double a[3], b[3], d[3];
    for (int i = 0; i < 3; i++) {
        a[i] = (double)A[i] - (double)P[i];
        b[i] = (double)B[i] - (double)P[i];
        d[i] = (double)D[i];
    }
    double c0 = a[1] * b[2] - a[2] * b[1];
    double c1 = a[2] * b[0] - a[0] * b[2];
    double c2 = a[0] * b[1] - a[1] * b[0];
    double det = d[0] * c0 + d[1] * c1 + d[2] * c2;
    double perm = fabs(d[0]) * (fabs(a[1] * b[2]) + fabs(a[2] * b[1]))
                + fabs(d[1]) * (fabs(a[2] * b[0]) + fabs(a[0] * b[2]))
                + fabs(d[2]) * (fabs(a[0] * b[1]) + fabs(a[1] * b[0]));
    if (fabs(det) > FILTER_U * perm && perm > 1e-280) return det > 0 ? 1 : -1;
    return exact_det_abd(A, B, P, D);
}

static int sign_orient(const float *V0, const float *V1, const float *V2, const float *P) {
    double a[3], b[3], c[3];
    for (int i = 0; i < 3; i++) {
        a[i] = (double)V0[i] - (double)P[i];
        b[i] = (double)V1[i] - (double)P[i];
        c[i] = (double)V2[i] - (double)P[i];
    }
    double det = a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2])
               + a[2] * (b[0] * c[1] - b[1] * c[0]);
    double perm = fabs(a[0]) * (fabs(b[1] * c[2]) + fabs(b[2] * c[1]))
                + fabs(a[1]) * (fabs(b[2] * c[0]) + fabs(b[0] * c[2]))
                + fabs(a[2]) * (fabs(b[0] * c[1]) + fabs(b[1] * c[0]));
    if (fabs(det) > FILTER_U * perm && perm > 1e-280) return det > 0 ? 1 : -1;
    return exact_orient(V0, V1, V2, P);
}

/* Sign of det[A-P, B-P, d_eps] with d_eps = d + eps e_x + eps^2 e_y + eps^3 e_z
 * (symbolic perturbation of the ray direction): the first nonzero of
 * det[a,b,d], (a x b)_x, (a x b)_y, (a x b)_z.  Zero only when P lies on the
 * line through A and B. */
static int sos_edge(const float *A, const float *B, const float *P, const float *D) {
    int s = sign_det_abd(A, B, P, D);
    if (s) return s;
    for (int k = 0; k < 3; k++) {
        s = exact_cross_comp(A, B, P, k);
        if (s) return s;
    }
    return 0;
}

ORACLE_API int oracle_sign_edge(const float *A, const float *B, const float *P, const float *D) {
    return sos_edge(A, B, P, D);
}
ORACLE_API int oracle_exact_det_abd(const float *A, const float *B, const float *P, const float *D) {
    return exact_det_abd(A, B, P, D);
}
ORACLE_API int oracle_sign_orient(const float *V0, const float *V1, const float *V2, const float *P) {
    return sign_orient(V0, V1, V2, P);
}
ORACLE_API int oracle_exact_orient(const float *V0, const float *V1, const float *V2, const float *P) {
    return exact_orient(V0, V1, V2, P);
}

/* ======================================================================== */
/* thread pool helper: static partition of [0, n) over nthreads             */
/* ======================================================================== */
typedef void (*range_fn)(void *ctx, int64_t lo, int64_t hi);
typedef struct { range_fn fn; void *ctx; int64_t lo, hi; } job_t;

static void *job_main(void *p) {
    job_t *j = (job_t *)p;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

static void parallel_for(int64_t n, int nthreads, range_fn fn, void *ctx) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n < nthreads) nthreads = (int)(n > 0 ? n : 1);
    if (nthreads == 1) { fn(ctx, 0, n); return; }
    pthread_t th[256];
    job_t jobs[256];
    int created[256];
    int64_t chunk = (n + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; t++) {
        jobs[t].fn = fn;
        jobs[t].ctx = ctx;
        jobs[t].lo = t * chunk < n ? t * chunk : n;
        jobs[t].hi = (t + 1) * chunk < n ? (t + 1) * chunk : n;
        created[t] = 0;
        if (jobs[t].lo >= jobs[t].hi) continue;
        if (pthread_create(&th[t], NULL, job_main, &jobs[t]) == 0) created[t] = 1;
        else job_main(&jobs[t]);               /* no thread: run inline */
    }
    for (int t = 0; t < nthreads; t++)
        if (created[t]) pthread_join(th[t], NULL);
}

/* ======================================================================== */
/* 3D definition: w(p) = (1/4pi) sum_T Omega_T(p)                           */
/* ======================================================================== */
/* Solid angle of triangle (a, b, c) seen from the origin, by the
 * Van Oosterom-Strackee half-angle formula. */
static double solid_angle(const double *a, const double *b, const double *c) {
    double la = sqrt(a[0]*a[0] + a[1]*a[1] + a[2]*a[2]);
    double lb = sqrt(b[0]*b[0] + b[1]*b[1] + b[2]*b[2]);
    double lc = sqrt(c[0]*c[0] + c[1]*c[1] + c[2]*c[2]);
    double num = a[0] * (b[1]*c[2] - b[2]*c[1]) + a[1] * (b[2]*c[0] - b[0]*c[2])
               + a[2] * (b[0]*c[1] - b[1]*c[0]);
    double ab = a[0]*b[0] + a[1]*b[1] + a[2]*b[2];
    double ac = a[0]*c[0] + a[1]*c[1] + a[2]*c[2];
    double bc = b[0]*c[0] + b[1]*c[1] + b[2]*c[2];
    double den = la * lb * lc + ab * lc + ac * lb + bc * la;
    return 2.0 * atan2(num, den);
}

ORACLE_API double oracle_solid_angle(const double *a, const double *b, const double *c) {
    return solid_angle(a, b, c);
}

typedef struct {
    const float *V; const int32_t *F; int64_t nf;
    const float *P; double *w;
} vos_ctx;

static void vos_range(void *p, int64_t lo, int64_t hi) {
    vos_ctx *c = (vos_ctx *)p;
    for (int64_t q = lo; q < hi; q++) {
        const float *pp = c->P + 3 * q;
        double acc = 0.0;
        for (int64_t t = 0; t < c->nf; t++) {
            double v[3][3];
            for (int k = 0; k < 3; k++) {
                const float *x = c->V + 3 * (int64_t)c->F[3 * t + k];
                for (int i = 0; i < 3; i++) v[k][i] = (double)x[i] - (double)pp[i];
            }
            acc += solid_angle(v[0], v[1], v[2]);
        }
        c->w[q] = acc / (4.0 * M_PI);
    }
}

ORACLE_API void oracle_w3d_vos(const float *V, const int32_t *F, int64_t nf, const float *P,
                               int64_t nq, double *w, int nthreads) {
    vos_ctx c = {V, F, nf, P, w};
    parallel_for(nq, nthreads, vos_range, &c);
}

/* ======================================================================== */
/* Signed crossing count chi_d(p) (Eq. chi), brute force over triangles     */
/* ======================================================================== */
/* Triangle T = (v0, v1, v2) with normal n = (v1-v0) x (v2-v0).  The ray
 * p + t d_eps (t > 0) crosses T iff the three edge orientations
 * det[vi-p, vj-p, d_eps] share one sign s, and det[v0-p, v1-p, v2-p] has the
 * same sign s (t > 0).  The three edge determinants sum to d_eps . n, so the
 * contribution sign(d_eps . n) equals s.  det[v0-p, v1-p, v2-p] = 0 means p
 * lies in the plane of T: such a triangle is not counted. */
static int tri_crossing(const float *v0, const float *v1, const float *v2, const float *p,
                        const float *d) {
    int s0 = sos_edge(v0, v1, p, d);
    if (s0 == 0) return 0;
    int s1 = sos_edge(v1, v2, p, d);
    if (s1 != s0) return 0;
    int s2 = sos_edge(v2, v0, p, d);
    if (s2 != s0) return 0;
    int o = sign_orient(v0, v1, v2, p);
    return o == s0 ? s0 : 0;
}

ORACLE_API int oracle_tri_crossing(const float *v0, const float *v1, const float *v2,
                                   const float *p, const float *d) {
    return tri_crossing(v0, v1, v2, p, d);
}

typedef struct {
    const float *V; const int32_t *F; int64_t nf;
    const float *P; const float *d; int32_t *chi;
} chi_ctx;

static void chi_range(void *p, int64_t lo, int64_t hi) {
    chi_ctx *c = (chi_ctx *)p;
    for (int64_t q = lo; q < hi; q++) {
        const float *pp = c->P + 3 * q;
        int acc = 0;
        for (int64_t t = 0; t < c->nf; t++) {
            const float *v0 = c->V + 3 * (int64_t)c->F[3 * t];
            const float *v1 = c->V + 3 * (int64_t)c->F[3 * t + 1];
            const float *v2 = c->V + 3 * (int64_t)c->F[3 * t + 2];
            /* cheap exact rejection: the triangle lies entirely on one side of
             * the ray's supporting planes is not used; every triangle is tested
             * with the exact predicates (plain brute force). */
            acc += tri_crossing(v0, v1, v2, pp, c->d);
        }
        c->chi[q] = acc;
    }
}

ORACLE_API void oracle_chi3d(const float *V, const int32_t *F, int64_t nf, const float *P,
                             int64_t nq, const float *d, int32_t *chi, int nthreads) {
    chi_ctx c = {V, F, nf, P, d, chi};
    parallel_for(nq, nthreads, chi_range, &c);
}

/* ======================================================================== */
/* Boundary edges with multiplicity                                         */
/* ======================================================================== */
/* Each triangle (i, j, k) contributes directed edges i->j, j->k, k->i.  The
 * net multiplicity of the undirected pair {u < v} is (#u->v) - (#v->u); a
 * pair with nonzero net multiplicity is a boundary edge, reported as
 * u->v with m > 0 or v->u with m > 0.  A face with a repeated index has a
 * zero-length edge u->u; it bounds nothing (its solid angle is 0) and is
 * skipped. */
typedef struct { int32_t u, v; int32_t s; } dedge_t;

static int cmp_dedge(const void *x, const void *y) {
    const dedge_t *a = (const dedge_t *)x, *b = (const dedge_t *)y;
    if (a->u != b->u) return a->u < b->u ? -1 : 1;
    if (a->v != b->v) return a->v < b->v ? -1 : 1;
    return 0;
}

ORACLE_API int64_t oracle_boundary_edges(const int32_t *F, int64_t nf, int32_t *src,
                                         int32_t *dst, int32_t *mult) {
    dedge_t *e = (dedge_t *)malloc(sizeof(dedge_t) * 3 * (size_t)(nf > 0 ? nf : 1));
    if (!e) return -1;
    int64_t ne = 0;
    for (int64_t t = 0; t < nf; t++) {
        for (int k = 0; k < 3; k++) {
            int32_t a = F[3 * t + k], b = F[3 * t + (k + 1) % 3];
            if (a == b) continue;          /* zero-length edge of a degenerate face */
            dedge_t *x = &e[ne++];
            if (a < b) { x->u = a; x->v = b; x->s = 1; }
            else { x->u = b; x->v = a; x->s = -1; }
        }
    }
    qsort(e, (size_t)ne, sizeof(dedge_t), cmp_dedge);
    int64_t n = 0;
    for (int64_t i = 0; i < ne;) {
        int64_t j = i;
        int32_t m = 0;
        while (j < ne && e[j].u == e[i].u && e[j].v == e[i].v) { m += e[j].s; j++; }
        if (m > 0) { src[n] = e[i].u; dst[n] = e[i].v; mult[n] = m; n++; }
        else if (m < 0) { src[n] = e[i].v; dst[n] = e[i].u; mult[n] = -m; n++; }
        i = j;
    }
    free(e);
    return n;
}

/* ======================================================================== */
/* Boundary term relative to direction d                                    */
/* ======================================================================== */
/* Closing M with the curtain {x - s d : x in dM, s >= 0} gives a closed
 * surface whose winding number at p is the signed crossing count of the ray
 * p + t d with M (the curtain is never met by that ray).  Hence
 *     w(p) = chi_d(p) - w_curtain(p),
 * and the curtain's solid angle is the sum over directed boundary edges A->B
 * of the solid angle of the spherical triangle (A-p, B-p, -d) with a minus
 * sign, giving
 *     B_d(p) = (1/4pi) sum_e m_e Omega(A_e - p, B_e - p, -d).
 * Omega jumps by 4pi where the ray p + t d crosses the edge; there the sign of
 * the numerator (= -det[A-p, B-p, d]/|d|) is taken from the exact, perturbed
 * predicate whenever the float64 value is within its error bound, so the jump
 * sits exactly where chi_d changes.
 * A boundary vertex lying exactly on the forward ray (ray through a vertex)
 * makes its two spherical triangles degenerate (0/0).  The crossing count
 * resolves that case with the perturbed direction d_eps; the boundary term
 * takes the limit under the same perturbation: the perturbed ray sees the
 * vertex in the direction -dp (dp = the first of e_x, e_y, e_z not parallel
 * to d, projected orthogonally to d), which gives the closed-form limits
 * below. */
typedef struct {
    const float *V; const int32_t *src, *dst, *mult; int64_t ne;
    const float *P; const float *d; double *B;
} bterm_ctx;

static void bterm_range(void *p, int64_t lo, int64_t hi) {
    bterm_ctx *c = (bterm_ctx *)p;
    double dn = sqrt((double)c->d[0] * c->d[0] + (double)c->d[1] * c->d[1]
                     + (double)c->d[2] * c->d[2]);
    double dh[3] = {(double)c->d[0] / dn, (double)c->d[1] / dn, (double)c->d[2] / dn};
    double cdir[3] = {-dh[0], -dh[1], -dh[2]};
    /* perturbation direction: the first of e_x, e_y, e_z not parallel to d,
     * minus its component along d */
    double dp[3] = {0, 0, 0};
    for (int k = 0; k < 3; k++) {
        double e[3] = {0, 0, 0};
        e[k] = 1.0;
        double t = e[0] * dh[0] + e[1] * dh[1] + e[2] * dh[2];
        double q[3] = {e[0] - t * dh[0], e[1] - t * dh[1], e[2] - t * dh[2]};
        if (fabs(q[0]) + fabs(q[1]) + fabs(q[2]) > 1e-12) { dp[0] = q[0]; dp[1] = q[1]; dp[2] = q[2]; break; }
    }
    for (int64_t q = lo; q < hi; q++) {
        const float *pp = c->P + 3 * q;
        double acc = 0.0;
        for (int64_t e = 0; e < c->ne; e++) {
            const float *A = c->V + 3 * (int64_t)c->src[e];
            const float *Bv = c->V + 3 * (int64_t)c->dst[e];
            double a[3], b[3];
            for (int i = 0; i < 3; i++) {
                a[i] = (double)A[i] - (double)pp[i];
                b[i] = (double)Bv[i] - (double)pp[i];
            }
            int ra = on_forward_ray(A, pp, c->d), rb = on_forward_ray(Bv, pp, c->d);
            double num, den, perm;
            if (ra && rb) {
                num = 0.0; den = 1.0; perm = 1.0;      /* edge along the ray: limit 0 */
            } else if (ra) {
                /* A on the ray: the perturbed ray sees A in direction -dp, so
                 * Omega/2 -> atan2(dp.(b x dh), -(b.dp)) */
                double bx[3] = {b[1] * dh[2] - b[2] * dh[1], b[2] * dh[0] - b[0] * dh[2], b[0] * dh[1] - b[1] * dh[0]};
                num = dp[0] * bx[0] + dp[1] * bx[1] + dp[2] * bx[2];
                den = -(b[0] * dp[0] + b[1] * dp[1] + b[2] * dp[2]);
                perm = fabs(dp[0]) * (fabs(b[1] * dh[2]) + fabs(b[2] * dh[1]))
                     + fabs(dp[1]) * (fabs(b[2] * dh[0]) + fabs(b[0] * dh[2]))
                     + fabs(dp[2]) * (fabs(b[0] * dh[1]) + fabs(b[1] * dh[0]));
            } else if (rb) {
                /* B on the ray: Omega/2 -> atan2(det[a, dp, dh], -(a.dp)) */
                double px[3] = {dp[1] * dh[2] - dp[2] * dh[1], dp[2] * dh[0] - dp[0] * dh[2], dp[0] * dh[1] - dp[1] * dh[0]};
                num = a[0] * px[0] + a[1] * px[1] + a[2] * px[2];
                den = -(a[0] * dp[0] + a[1] * dp[1] + a[2] * dp[2]);
                perm = fabs(a[0]) * fabs(px[0]) + fabs(a[1]) * fabs(px[1]) + fabs(a[2]) * fabs(px[2]) + 1e-300;
            } else {
                double la = sqrt(a[0]*a[0] + a[1]*a[1] + a[2]*a[2]);
                double lb = sqrt(b[0]*b[0] + b[1]*b[1] + b[2]*b[2]);
                double x0 = a[1]*b[2] - a[2]*b[1], x1 = a[2]*b[0] - a[0]*b[2], x2 = a[0]*b[1] - a[1]*b[0];
                num = cdir[0]*x0 + cdir[1]*x1 + cdir[2]*x2;
                perm = fabs(cdir[0]) * (fabs(a[1]*b[2]) + fabs(a[2]*b[1]))
                     + fabs(cdir[1]) * (fabs(a[2]*b[0]) + fabs(a[0]*b[2]))
                     + fabs(cdir[2]) * (fabs(a[0]*b[1]) + fabs(a[1]*b[0]));
                double ab = a[0]*b[0] + a[1]*b[1] + a[2]*b[2];
                double ac = a[0]*cdir[0] + a[1]*cdir[1] + a[2]*cdir[2];
                double bc = b[0]*cdir[0] + b[1]*cdir[1] + b[2]*cdir[2];
                den = la * lb + ab + ac * lb + bc * la;
            }
            if (den < 0.0 && fabs(num) <= 4.0 * FILTER_U * perm + 1e-300) {
                int s = sos_edge(A, Bv, pp, c->d);      /* sign(num) = -s */
                if (s > 0) num = -fabs(num);
                else if (s < 0) num = fabs(num);
            }
            acc += (double)c->mult[e] * 2.0 * atan2(num, den);
        }
        c->B[q] = acc / (4.0 * M_PI);
    }
}

ORACLE_API void oracle_bterm3d(const float *V, const int32_t *src, const int32_t *dst,
                               const int32_t *mult, int64_t ne, const float *P, int64_t nq,
                               const float *d, double *B, int nthreads) {
    bterm_ctx c = {V, src, dst, mult, ne, P, d, B};
    parallel_for(nq, nthreads, bterm_range, &c);
}

/* ======================================================================== */
/* Gradient of the 3D definition                                            */
/* ======================================================================== */
/* Omega = 2 atan2(N, D) with N = a.(b x c), D = |a||b||c| + (a.b)|c| +
 * (a.c)|b| + (b.c)|a|, a = v0 - p, b = v1 - p, c = v2 - p.
 * dOmega = 2 (D dN - N dD) / (N^2 + D^2);  d/dp = -(d/da + d/db + d/dc). */
static void solid_angle_grad(const double *a, const double *b, const double *c,
                             double *ga, double *gb, double *gc) {
    double la = sqrt(a[0]*a[0] + a[1]*a[1] + a[2]*a[2]);
    double lb = sqrt(b[0]*b[0] + b[1]*b[1] + b[2]*b[2]);
    double lc = sqrt(c[0]*c[0] + c[1]*c[1] + c[2]*c[2]);
    double bxc[3] = {b[1]*c[2] - b[2]*c[1], b[2]*c[0] - b[0]*c[2], b[0]*c[1] - b[1]*c[0]};
    double cxa[3] = {c[1]*a[2] - c[2]*a[1], c[2]*a[0] - c[0]*a[2], c[0]*a[1] - c[1]*a[0]};
    double axb[3] = {a[1]*b[2] - a[2]*b[1], a[2]*b[0] - a[0]*b[2], a[0]*b[1] - a[1]*b[0]};
    double N = a[0]*bxc[0] + a[1]*bxc[1] + a[2]*bxc[2];
    double ab = a[0]*b[0] + a[1]*b[1] + a[2]*b[2];
    double ac = a[0]*c[0] + a[1]*c[1] + a[2]*c[2];
    double bc = b[0]*c[0] + b[1]*c[1] + b[2]*c[2];
    double D = la * lb * lc + ab * lc + ac * lb + bc * la;
    double k = 2.0 / (N * N + D * D);
    for (int i = 0; i < 3; i++) {
        double dDa = a[i] / la * (lb * lc + bc) + b[i] * lc + c[i] * lb;
        double dDb = b[i] / lb * (la * lc + ac) + a[i] * lc + c[i] * la;
        double dDc = c[i] / lc * (la * lb + ab) + a[i] * lb + b[i] * la;
        ga[i] = k * (D * bxc[i] - N * dDa);
        gb[i] = k * (D * cxa[i] - N * dDb);
        gc[i] = k * (D * axb[i] - N * dDc);
    }
}

typedef struct {
    const float *V; int64_t nv; const int32_t *F; int64_t nf;
    const float *P; int64_t nq; const double *gw;
    double *grad_p; double *grad_V_parts; int nparts;
} grad_ctx;

static void grad_range(void *p, int64_t lo, int64_t hi) {
    grad_ctx *c = (grad_ctx *)p;
    int64_t chunk = (c->nq + c->nparts - 1) / c->nparts;
    int part = (int)(chunk > 0 ? lo / chunk : 0);
    double *gV = c->grad_V_parts ? c->grad_V_parts + (size_t)part * 3 * c->nv : NULL;
    for (int64_t q = lo; q < hi; q++) {
        const float *pp = c->P + 3 * q;
        double g = c->gw ? c->gw[q] : 1.0;
        double gp[3] = {0, 0, 0};
        for (int64_t t = 0; t < c->nf; t++) {
            double v[3][3], gr[3][3];
            for (int k = 0; k < 3; k++) {
                const float *x = c->V + 3 * (int64_t)c->F[3 * t + k];
                for (int i = 0; i < 3; i++) v[k][i] = (double)x[i] - (double)pp[i];
            }
            solid_angle_grad(v[0], v[1], v[2], gr[0], gr[1], gr[2]);
            for (int k = 0; k < 3; k++) {
                for (int i = 0; i < 3; i++) {
                    gp[i] -= gr[k][i];
                    if (gV) gV[3 * (int64_t)c->F[3 * t + k] + i] += g * gr[k][i] / (4.0 * M_PI);
                }
            }
        }
        if (c->grad_p)
            for (int i = 0; i < 3; i++) c->grad_p[3 * q + i] = g * gp[i] / (4.0 * M_PI);
    }
}

/* grad_p[q] = gw[q] * dw_q/dp ; grad_V = sum_q gw[q] * dw_q/dV (gw NULL = 1).
 * Either output may be NULL. */
ORACLE_API int oracle_grad3d_vos(const float *V, int64_t nv, const int32_t *F, int64_t nf,
                                 const float *P, int64_t nq, const double *gw, double *grad_p,
                                 double *grad_V, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nq < nthreads) nthreads = (int)(nq > 0 ? nq : 1);
    double *parts = NULL;
    if (grad_V) {
        parts = (double *)calloc((size_t)nthreads * 3 * (size_t)nv, sizeof(double));
        if (!parts) return -1;
    }
    grad_ctx c = {V, nv, F, nf, P, nq, gw, grad_p, parts, nthreads};
    parallel_for(nq, nthreads, grad_range, &c);
    if (grad_V) {
        for (int64_t i = 0; i < 3 * nv; i++) {
            double s = 0.0;
            for (int t = 0; t < nthreads; t++) s += parts[(size_t)t * 3 * nv + i];
            grad_V[i] = s;
        }
        free(parts);
    }
    return 0;
}

/* ======================================================================== */
/* 2D: cubic Bezier chains                                                  */
/* ======================================================================== */
static void bez_eval(const double *c, double u, double *x, double *y) {
    double v = 1.0 - u;
    double b0 = v * v * v, b1 = 3 * u * v * v, b2 = 3 * u * u * v, b3 = u * u * u;
    *x = b0 * c[0] + b1 * c[2] + b2 * c[4] + b3 * c[6];
    *y = b0 * c[1] + b1 * c[3] + b2 * c[5] + b3 * c[7];
}

static void bez_deriv(const double *c, double u, double *dx, double *dy) {
    double v = 1.0 - u;
    *dx = 3 * (v * v * (c[2] - c[0]) + 2 * u * v * (c[4] - c[2]) + u * u * (c[6] - c[4]));
    *dy = 3 * (v * v * (c[3] - c[1]) + 2 * u * v * (c[5] - c[3]) + u * u * (c[7] - c[5]));
}

/* integrand of the subtended angle: cross(B - p, B') / |B - p|^2 */
static double angle_rate(const double *c, const double *p, double u) {
    double x, y, dx, dy;
    bez_eval(c, u, &x, &y);
    bez_deriv(c, u, &dx, &dy);
    x -= p[0]; y -= p[1];
    return (x * dy - y * dx) / (x * x + y * y);
}

/* Gauss-Kronrod 7-15 nodes/weights on [-1, 1] */
static const double GK_X[8] = {0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
                               0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
                               0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
                               0.207784955007898467600689403773245, 0.0};
static const double GK_WK[8] = {0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
                                0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
                                0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
                                0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double GK_WG[4] = {0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
                                0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

/* Gauss-Kronrod 7-15 on [a, b] with the QUADPACK-style error estimate
 * (the Kronrod-Gauss difference scaled by the integral of |f - mean|). */
static double gk15(const double *c, const double *p, double a, double b, double *err,
                   double *resabs) {
    double m = 0.5 * (a + b), h = 0.5 * (b - a);
    double fv[15];
    fv[7] = angle_rate(c, p, m);
    double k = GK_WK[7] * fv[7], g = GK_WG[3] * fv[7], ka = GK_WK[7] * fabs(fv[7]);
    for (int i = 0; i < 7; i++) {
        double f1 = angle_rate(c, p, m - h * GK_X[i]);
        double f2 = angle_rate(c, p, m + h * GK_X[i]);
        fv[i] = f1; fv[14 - i] = f2;
        k += GK_WK[i] * (f1 + f2);
        ka += GK_WK[i] * (fabs(f1) + fabs(f2));
        if (i & 1) g += GK_WG[i / 2] * (f1 + f2);
    }
    double mean = 0.5 * k;
    double asc = GK_WK[7] * fabs(fv[7] - mean);
    for (int i = 0; i < 7; i++) asc += GK_WK[i] * (fabs(fv[i] - mean) + fabs(fv[14 - i] - mean));
    double e = fabs((k - g) * h);
    asc *= fabs(h);
    if (asc != 0.0 && e != 0.0) {
        double r = pow(200.0 * e / asc, 1.5);
        e = asc * (r < 1.0 ? r : 1.0);
    }
    *err = e;
    *resabs = ka * fabs(h);
    return k * h;
}

/* Globally adaptive Gauss-Kronrod: keep a heap of subintervals ordered by
 * their error estimate, bisect the worst one, and stop when the summed error
 * estimate is below tol (or below the round-off floor, 50 ulps of the integral
 * of |f|), when the worst interval is shorter than 1e-13, or after
 * QUAD_LIMIT intervals.  The cap bounds the work for queries arbitrarily close
 * to the curve (where w is undefined and no comparison is made). */
#define QUAD_LIMIT 2048
typedef struct { double a, b, v, e, ra; } qint_t;

static void heap_push(qint_t *h, int *n, qint_t x) {
    int i = (*n)++;
    h[i] = x;
    while (i > 0) {
        int p = (i - 1) / 2;
        if (h[p].e >= h[i].e) break;
        qint_t t = h[p]; h[p] = h[i]; h[i] = t;
        i = p;
    }
}

static qint_t heap_pop(qint_t *h, int *n) {
    qint_t top = h[0];
    h[0] = h[--(*n)];
    int i = 0;
    for (;;) {
        int l = 2 * i + 1, r = l + 1, m = i;
        if (l < *n && h[l].e > h[m].e) m = l;
        if (r < *n && h[r].e > h[m].e) m = r;
        if (m == i) break;
        qint_t t = h[m]; h[m] = h[i]; h[i] = t;
        i = m;
    }
    return top;
}

static double adapt(const double *c, const double *p, double a, double b, double tol) {
    qint_t heap[QUAD_LIMIT + 2];
    int n = 0;
    qint_t x;
    x.a = a; x.b = b;
    x.v = gk15(c, p, a, b, &x.e, &x.ra);
    if (!isfinite(x.v) || !isfinite(x.e)) return x.v;
    heap_push(heap, &n, x);
    double tot = x.v, err = x.e, rabs = x.ra;
    while (n < QUAD_LIMIT) {
        if (err <= tol || err <= 50.0 * 2.220446049250313e-16 * rabs) break;
        qint_t w = heap_pop(heap, &n);
        if (w.b - w.a < 1e-13) { heap_push(heap, &n, w); break; }
        double m = 0.5 * (w.a + w.b);
        qint_t l, r;
        l.a = w.a; l.b = m; l.v = gk15(c, p, w.a, m, &l.e, &l.ra);
        r.a = m; r.b = w.b; r.v = gk15(c, p, m, w.b, &r.e, &r.ra);
        if (!isfinite(l.v) || !isfinite(r.v)) return l.v + r.v;
        tot += l.v + r.v - w.v;
        err += l.e + r.e - w.e;
        rabs += l.ra + r.ra - w.ra;
        heap_push(heap, &n, l);
        heap_push(heap, &n, r);
    }
    /* re-sum the accepted intervals (avoids drift of the running total) */
    double s = 0.0;
    for (int i = 0; i < n; i++) s += heap[i].v;
    (void)tot;
    return s;
}

typedef struct {
    const double *ctrl; int64_t nseg; const double *P; double *w; double tol;
} quad_ctx;

static void quad_range(void *p, int64_t lo, int64_t hi) {
    quad_ctx *c = (quad_ctx *)p;
    for (int64_t q = lo; q < hi; q++) {
        double acc = 0.0;
        for (int64_t s = 0; s < c->nseg; s++)
            acc += adapt(c->ctrl + 6 * s, c->P + 2 * q, 0.0, 1.0, c->tol);
        c->w[q] = acc / (2.0 * M_PI);
    }
}

/* 2D definition: w(p) = (1/2pi) sum_segments int_0^1 cross(B-p, B')/|B-p|^2 du
 * ctrl: 3*nseg+1 points (x, y) of one C0 chain. */
ORACLE_API void oracle_w2d_quad(const double *ctrl, int64_t nseg, const double *P, int64_t nq,
                                double *w, double tol, int nthreads) {
    quad_ctx c = {ctrl, nseg, P, w, tol};
    parallel_for(nq, nthreads, quad_range, &c);
}

/* Real roots in [0, 1] of g(u) = sum_k g_k B_k(u) (cubic Bernstein), sorted,
 * found by splitting [0,1] at the roots of g' into monotone intervals and
 * bisecting each interval whose end values straddle zero.  With the
 * half-open rule of a ray perturbed towards g > 0 (the ray is taken as
 * g = 0+): an interval from g(u0) to g(u1) holds a crossing iff
 * min(g0, g1) <= 0 < max(g0, g1).  Returns the number of crossings; for
 * each, the parameter, the direction (+1 when g increases) and a
 * certification radius in u: the exact root lies within rad[i] of us[i]
 * (INFINITY when that cannot be bounded, or when the interval's end value at
 * an interior cut is within its evaluation error of zero, so that even the
 * existence of the crossing is uncertain). */
static double bern3(const double *g, double u) {
    double v = 1.0 - u;
    return v * v * v * g[0] + 3 * u * v * v * g[1] + 3 * u * u * v * g[2] + u * u * u * g[3];
}

/* derivative of the cubic Bernstein polynomial, and a bound on |second
 * derivative| over [0, 1] */
static double bern3_d(const double *g, double u) {
    double v = 1.0 - u;
    return 3.0 * ((g[1] - g[0]) * v * v + 2.0 * (g[2] - g[1]) * u * v + (g[3] - g[2]) * u * u);
}
static double bern3_d2max(const double *g) {
    double a = fabs(g[2] - 2.0 * g[1] + g[0]), b = fabs(g[3] - 2.0 * g[2] + g[1]);
    return 6.0 * (a > b ? a : b);
}
/* bound on the float64 evaluation error of bern3 (and of forming the
 * coefficients by one subtraction each) */
static double bern3_err(const double *g) {
    return 12.0 * DBL_EPSILON * (fabs(g[0]) + fabs(g[1]) + fabs(g[2]) + fabs(g[3]));
}

static int monotone_crossings(const double *g, double *us, int *dirs, double *rad) {
    /* derivative coefficients (quadratic Bernstein, times 3) */
    double d0 = g[1] - g[0], d1 = g[2] - g[1], d2 = g[3] - g[2];
    /* power basis of d(u) = d0 (1-u)^2 + 2 d1 u (1-u) + d2 u^2 */
    double A = d0 - 2 * d1 + d2, B = 2 * (d1 - d0), C = d0;
    double cuts[4];
    int nc = 0;
    cuts[nc++] = 0.0;
    double r[2];
    int nr = 0;
    if (fabs(A) < 1e-300 * (fabs(B) + fabs(C) + 1e-300)) {
        if (B != 0.0) r[nr++] = -C / B;
    } else {
        double disc = B * B - 4 * A * C;
        if (disc > 0) {
            double sq = sqrt(disc);
            double qq = -0.5 * (B + (B >= 0 ? sq : -sq));
            r[nr++] = qq / A;
            if (qq != 0.0) r[nr++] = C / qq;
        }
    }
    if (nr == 2 && r[0] > r[1]) { double t = r[0]; r[0] = r[1]; r[1] = t; }
    for (int i = 0; i < nr; i++) if (r[i] > 0.0 && r[i] < 1.0) cuts[nc++] = r[i];
    cuts[nc++] = 1.0;
    const double eg = bern3_err(g), m2 = bern3_d2max(g);
    int n = 0;
    for (int i = 0; i + 1 < nc; i++) {
        double u0 = cuts[i], u1 = cuts[i + 1];
        double g0 = bern3(g, u0), g1 = bern3(g, u1);
        if (i == 0) g0 = g[0];
        if (i + 2 == nc) g1 = g[3];
        /* an end at an interior cut (an extremum of g) is only known to eg:
         * whether the interval crosses zero there is uncertain, and so are the
         * crossings within du of the cut, du the half-width of the
         * neighbourhood where |g| <= 2 eg (found by doubling) */
        double uc = -1.0, du = 0.0;
        if (i > 0 && fabs(g0) <= eg) uc = u0;
        else if (i + 2 < nc && fabs(g1) <= eg) uc = u1;
        if (uc >= 0.0) {
            du = 1e-17;
            while (du < 1.0 && (fabs(bern3(g, uc - du)) <= 2.0 * eg || fabs(bern3(g, uc + du)) <= 2.0 * eg))
                du *= 2.0;
        }
        double lo = g0 < g1 ? g0 : g1, hi = g0 < g1 ? g1 : g0;
        if (!(lo <= 0.0 && 0.0 < hi)) {
            if (uc >= 0.0) {            /* a crossing the rounding may have hidden */
                us[n] = uc;
                dirs[n] = 0;
                rad[n] = du;
                n++;
            }
            continue;
        }
        double a = u0, b = u1;
        int inc = g1 > g0;
        for (int it = 0; it < 200 && b - a > 0.0; it++) {
            double m = 0.5 * (a + b);
            if (m <= a || m >= b) break;
            double gm = bern3(g, m);
            if ((gm > 0.0) == inc) b = m; else a = m;
        }
        double u = 0.5 * (a + b);
        us[n] = u;
        dirs[n] = inc ? 1 : -1;
        /* the exact root: g changes by at least |g'(u)|/2 per unit of u within
         * del of u when m2 del <= |g'(u)|/2, so it lies within
         * del = 2 (|g(u)| + eg) / |g'(u)| of u (the derivative's own error
         * taken off first) */
        double dg = fabs(bern3_d(g, u)) - 12.0 * DBL_EPSILON * (fabs(d0) + fabs(d1) + fabs(d2)) * 3.0;
        double del = dg > 0.0 ? 2.0 * (fabs(bern3(g, u)) + eg) / dg : INFINITY;
        if (!(m2 * del <= 0.5 * dg)) del = INFINITY;
        if (del < b - a) del = b - a;
        if (uc >= 0.0) {                /* the crossing itself may be spurious */
            double r2 = fabs(u - uc) + du;
            if (r2 > del) del = r2;
        }
        rad[n] = del;
        n++;
    }
    return n;
}

/* signed crossings of the ray p + t q (t > 0) with one cubic segment; the
 * ray is perturbed to its left (towards cross(q, x - p) > 0).  *unc is set
 * when a crossing lies within its certification bound of p along the ray (or
 * its existence is uncertain): the count is then not certified. */
static int seg_ray_crossings(const double *c, const double *p, const double *q, int *unc) {
    double g[4], h[4];
    for (int k = 0; k < 4; k++) {
        double x = c[2 * k] - p[0], y = c[2 * k + 1] - p[1];
        g[k] = q[0] * y - q[1] * x;            /* cross(q, B_k - p) */
        h[k] = q[0] * x + q[1] * y;            /* (B_k - p) . q: position along the ray */
    }
    double us[3], rad[3];
    int dirs[3];
    int n = monotone_crossings(g, us, dirs, rad);
    const double eh = bern3_err(h), m2h = bern3_d2max(h);
    int chi = 0;
    for (int i = 0; i < n; i++) {
        double t = bern3(h, us[i]);
        double band = (fabs(bern3_d(h, us[i])) + m2h * rad[i]) * rad[i] + eh;
        if (unc && !(fabs(t) > band)) *unc = 1;
        if (t > 0.0) chi += dirs[i];
    }
    return chi;
}

static int chain_ray_crossings(const double *ctrl, int64_t nseg, const double *p, const double *q, int *unc) {
    int chi = 0;
    for (int64_t s = 0; s < nseg; s++) chi += seg_ray_crossings(ctrl + 6 * s, p, q, unc);
    return chi;
}

typedef struct {
    const double *ctrl; int64_t nseg; const double *P; double *w; int32_t *chi;
} alg1_ctx;

/* Algorithm 1 in 2D.  The boundary of an open chain is its end points s, e;
 * their directions from p split the unit circle into two arcs:
 * A1 from e counter-clockwise to s, A2 from s counter-clockwise to e.  One
 * ray through the middle of the larger arc gives its chi; crossing the
 * direction of e counter-clockwise lowers chi by one (the in-plane normal
 * rule of Lemma 2 for the positively oriented end point), so
 * chi(A1) = chi(A2) - 1.  w = (|A1| chi(A1) + |A2| chi(A2)) / 2pi. */
static void alg1_range(void *pv, int64_t lo, int64_t hi) {
    alg1_ctx *c = (alg1_ctx *)pv;
    const double *s = c->ctrl;
    const double *e = c->ctrl + 6 * c->nseg;
    for (int64_t qi = lo; qi < hi; qi++) {
        const double *p = c->P + 2 * qi;
        double as = atan2(s[1] - p[1], s[0] - p[0]);
        double ae = atan2(e[1] - p[1], e[0] - p[0]);
        double L1 = fmod(as - ae, 2 * M_PI);
        if (L1 < 0) L1 += 2 * M_PI;
        double L2 = 2 * M_PI - L1;
        double mid;
        int chi1, chi2;
        if (L1 >= L2) {
            mid = ae + 0.5 * L1;
            double q[2] = {cos(mid), sin(mid)};
            chi1 = chain_ray_crossings(c->ctrl, c->nseg, p, q, NULL);
            chi2 = chi1 + 1;
        } else {
            mid = as + 0.5 * L2;
            double q[2] = {cos(mid), sin(mid)};
            chi2 = chain_ray_crossings(c->ctrl, c->nseg, p, q, NULL);
            chi1 = chi2 - 1;
        }
        c->w[qi] = (L1 * chi1 + L2 * chi2) / (2 * M_PI);
        if (c->chi) c->chi[qi] = L1 >= L2 ? chi1 : chi2;
    }
}

ORACLE_API void oracle_w2d_alg1(const double *ctrl, int64_t nseg, const double *P, int64_t nq,
                                double *w, int nthreads) {
    alg1_ctx c = {ctrl, nseg, P, w, NULL};
    parallel_for(nq, nthreads, alg1_range, &c);
}

/* Closed form relative to the +x ray (ray perturbed towards +y, i.e. a
 * crossing counts when the curve's y range is [lo, hi) around y_p):
 *   w = chi_x(C) + chi_x(chord e->s) + atan2(cross(s-p, e-p), dot(s-p, e-p))/2pi.
 * chi_out receives chi_x(C) + chi_x(chord). */
typedef struct {
    const double *ctrl; int64_t nseg; const double *P; double *w; int32_t *chi; int8_t *unc;
} cx_ctx;

static int chord_crossing_x(const double *e, const double *s, const double *p, int *unc) {
    /* segment e -> s against the ray p + t(1,0), perturbed to y_p + 0 */
    double y0 = e[1] - p[1], y1 = s[1] - p[1];
    double lo = y0 < y1 ? y0 : y1, hi = y0 < y1 ? y1 : y0;
    if (!(lo <= 0.0 && 0.0 < hi)) return 0;
    /* x at y = y_p on the segment, compared with x_p via the orientation;
     * the sign of cr is certified beyond its rounding bound */
    double t1 = (e[0] - p[0]) * (s[1] - p[1]), t2 = (e[1] - p[1]) * (s[0] - p[0]);
    double cr = t1 - t2;
    if (unc && !(fabs(cr) > 8.0 * DBL_EPSILON * (fabs(t1) + fabs(t2)))) *unc = 1;
    int up = y1 > y0;
    /* the crossing is to the right of p iff p is left of the upward segment */
    int right = up ? (cr > 0) : (cr < 0);
    return right ? (up ? 1 : -1) : 0;
}

static void cx_range(void *pv, int64_t lo, int64_t hi) {
    cx_ctx *c = (cx_ctx *)pv;
    const double *s = c->ctrl;
    const double *e = c->ctrl + 6 * c->nseg;
    const double q[2] = {1.0, 0.0};
    for (int64_t qi = lo; qi < hi; qi++) {
        const double *p = c->P + 2 * qi;
        int unc = 0;
        int chi = chain_ray_crossings(c->ctrl, c->nseg, p, q, &unc) + chord_crossing_x(e, s, p, &unc);
        if (c->unc) c->unc[qi] = (int8_t)unc;
        double sx = s[0] - p[0], sy = s[1] - p[1], ex = e[0] - p[0], ey = e[1] - p[1];
        double ang = atan2(sx * ey - sy * ex, sx * ex + sy * ey);
        c->w[qi] = (double)chi + ang / (2 * M_PI);
        if (c->chi) c->chi[qi] = chi;
    }
}

ORACLE_API void oracle_w2d_closed_x(const double *ctrl, int64_t nseg, const double *P, int64_t nq,
                                    double *w, int32_t *chi, int8_t *unc, int nthreads) {
    cx_ctx c = {ctrl, nseg, P, w, chi, unc};
    parallel_for(nq, nthreads, cx_range, &c);
}

/* signed crossings of an arbitrary ray with a chain (exposed for tests) */
ORACLE_API int oracle_chain_ray_crossings(const double *ctrl, int64_t nseg, const double *p,
                                          const double *q) {
    return chain_ray_crossings(ctrl, nseg, p, q, NULL);
}

/* ======================================================================== */
/* Distances (test filtering only: w is undefined on M)                     */
/* ======================================================================== */
static double dot3(const double *a, const double *b) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }

/* squared distance from p to triangle (a, b, c): closest point by Voronoi
 * region classification of the triangle's vertices, edges and face. */
static double tri_dist2(const double *a, const double *b, const double *c, const double *p) {
    double ab[3], ac[3], ap[3], q[3];
    for (int i = 0; i < 3; i++) { ab[i] = b[i] - a[i]; ac[i] = c[i] - a[i]; ap[i] = p[i] - a[i]; }
    double d1 = dot3(ab, ap), d2 = dot3(ac, ap);
    if (d1 <= 0 && d2 <= 0) { for (int i = 0; i < 3; i++) q[i] = a[i]; goto done; }
    double bp[3];
    for (int i = 0; i < 3; i++) bp[i] = p[i] - b[i];
    double d3 = dot3(ab, bp), d4 = dot3(ac, bp);
    if (d3 >= 0 && d4 <= d3) { for (int i = 0; i < 3; i++) q[i] = b[i]; goto done; }
    double vc = d1 * d4 - d3 * d2;
    if (vc <= 0 && d1 >= 0 && d3 <= 0) {
        double v = d1 / (d1 - d3);
        for (int i = 0; i < 3; i++) q[i] = a[i] + v * ab[i];
        goto done;
    }
    double cp[3];
    for (int i = 0; i < 3; i++) cp[i] = p[i] - c[i];
    double d5 = dot3(ab, cp), d6 = dot3(ac, cp);
    if (d6 >= 0 && d5 <= d6) { for (int i = 0; i < 3; i++) q[i] = c[i]; goto done; }
    double vb = d5 * d2 - d1 * d6;
    if (vb <= 0 && d2 >= 0 && d6 <= 0) {
        double w = d2 / (d2 - d6);
        for (int i = 0; i < 3; i++) q[i] = a[i] + w * ac[i];
        goto done;
    }
    double va = d3 * d6 - d5 * d4;
    if (va <= 0 && (d4 - d3) >= 0 && (d5 - d6) >= 0) {
        double w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        for (int i = 0; i < 3; i++) q[i] = b[i] + w * (c[i] - b[i]);
        goto done;
    }
    {
        double den = 1.0 / (va + vb + vc);
        double v = vb * den, w = vc * den;
        for (int i = 0; i < 3; i++) q[i] = a[i] + ab[i] * v + ac[i] * w;
    }
done:;
    double r = 0;
    for (int i = 0; i < 3; i++) r += (p[i] - q[i]) * (p[i] - q[i]);
    return r;
}

typedef struct { const float *V; const int32_t *F; int64_t nf; const float *P; double *out; } dist_ctx;

static void dist_range(void *pv, int64_t lo, int64_t hi) {
    dist_ctx *c = (dist_ctx *)pv;
    for (int64_t q = lo; q < hi; q++) {
        double p[3] = {c->P[3*q], c->P[3*q+1], c->P[3*q+2]};
        double best = INFINITY;
        for (int64_t t = 0; t < c->nf; t++) {
            double v[3][3];
            for (int k = 0; k < 3; k++)
                for (int i = 0; i < 3; i++) v[k][i] = c->V[3 * (int64_t)c->F[3*t+k] + i];
            double d2 = tri_dist2(v[0], v[1], v[2], p);
            if (d2 < best) best = d2;
        }
        c->out[q] = sqrt(best);
    }
}

ORACLE_API void oracle_dist3d(const float *V, const int32_t *F, int64_t nf, const float *P,
                              int64_t nq, double *out, int nthreads) {
    dist_ctx c = {V, F, nf, P, out};
    parallel_for(nq, nthreads, dist_range, &c);
}

typedef struct { const double *ctrl; int64_t nseg; const double *P; double *out; } dist2_ctx;

static void dist2_range(void *pv, int64_t lo, int64_t hi) {
    dist2_ctx *c = (dist2_ctx *)pv;
    for (int64_t q = lo; q < hi; q++) {
        const double *p = c->P + 2 * q;
        double best = INFINITY;
        for (int64_t s = 0; s < c->nseg; s++) {
            const double *cc = c->ctrl + 6 * s;
            int ns = 256;
            double bu = 0, bd = INFINITY;
            for (int k = 0; k <= ns; k++) {
                double x, y, u = (double)k / ns;
                bez_eval(cc, u, &x, &y);
                double d2 = (x - p[0]) * (x - p[0]) + (y - p[1]) * (y - p[1]);
                if (d2 < bd) { bd = d2; bu = u; }
            }
            /* golden-section refinement around the best sample */
            double a = bu - 1.0 / ns, b = bu + 1.0 / ns;
            if (a < 0) a = 0;
            if (b > 1) b = 1;
            for (int it = 0; it < 80; it++) {
                double m1 = a + 0.381966 * (b - a), m2 = b - 0.381966 * (b - a);
                double x1, y1, x2, y2;
                bez_eval(cc, m1, &x1, &y1);
                bez_eval(cc, m2, &x2, &y2);
                double f1 = (x1 - p[0]) * (x1 - p[0]) + (y1 - p[1]) * (y1 - p[1]);
                double f2 = (x2 - p[0]) * (x2 - p[0]) + (y2 - p[1]) * (y2 - p[1]);
                if (f1 < f2) b = m2; else a = m1;
                if (f1 < bd) bd = f1;
                if (f2 < bd) bd = f2;
            }
            if (bd < best) best = bd;
        }
        c->out[q] = sqrt(best);
    }
}

ORACLE_API void oracle_dist2d(const double *ctrl, int64_t nseg, const double *P, int64_t nq,
                              double *out, int nthreads) {
    dist2_ctx c = {ctrl, nseg, P, out};
    parallel_for(nq, nthreads, dist2_range, &c);
}

/* ======================================================================== */
/* 3D Algorithm 1 by a spherical arrangement (tiny inputs)                  */
/* ======================================================================== */
/* The one-shot algorithm as the paper states it (Algorithm 1, with the
 * region structure of Lemma 1 and Lemma 2 and the discrete sum of
 * Eq. wn_discrete_sum): project the boundary of M onto the unit sphere around
 * p (each boundary edge A->B becomes the minor great-circle arc a->b), build
 * the arrangement of these arcs, take the area of every region, shoot ONE ray
 * into the largest region to get its crossing count, propagate the counts to
 * all regions across the arcs (Lemma 2), and return
 *     w(p) = (1/4 pi) sum_i Area(A_i) chi_i.
 * It is a third, independent evaluation (no boundary-term formula) used to
 * pin the other two on tiny inputs.
 *
 * Details of this implementation:
 *   - arrangement: all pairwise proper intersections of the arcs (float64),
 *     each arc split at its intersections; the planar map is a half-edge
 *     structure whose faces are the cycles of next(h) = the out-edge at the
 *     head of h immediately clockwise (seen from outside) from the reverse of
 *     h, so every face lies on the left of its half-edges;
 *   - separate components of the projected boundary (several loops whose
 *     images do not meet) are joined by arcs of weight zero, across which
 *     chi does not change, so every region is bounded by one cycle;
 *   - area of a region from its corners (Gauss-Bonnet for a geodesic
 *     polygon): A = 2 pi - sum_i (pi - alpha_i), alpha_i the interior angle;
 *     the printed formula in the implementation section has the sign of the
 *     corner term reversed (it gives the complement), so the standard form is
 *     used;
 *   - across a boundary arc a->b of multiplicity m, chi on its left exceeds
 *     chi on its right by m: a ray just on the triangle's side of the arc
 *     hits the triangle next to edge A->B and the hit counts sign(d . n) =
 *     sign(n . (A - p)), while the triangle's image lies on the left of a->b
 *     exactly when n . (A - p) > 0 (both cases give +m);
 *   - the ray into the largest region starts at the midpoint of its longest
 *     side, offset into the region by a small angle checked to cross no arc,
 *     and its direction rounded to float32 for the exact crossing count.
 * Inputs must be generic: no two arcs on one great circle, no endpoint
 * antipodal to another, no three arcs through one point.
 * Returns 0, or -1 (degenerate input), -2 (inconsistent arrangement),
 * -3 (out of memory). */
typedef struct { int a, b, w; } sarc_t;
typedef struct { int arc, other; double t; int vid; } sxing_t;
typedef struct { int u, v, w; } spiece_t;

static void cross3d(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3d(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static int normalize3d(double *a) {
    double n = sqrt(dot3d(a, a));
    if (!(n > 0.0)) return -1;
    a[0] /= n; a[1] /= n; a[2] /= n;
    return 0;
}
/* angle from a to b along the great circle (both unit) */
static double arc_angle(const double *a, const double *b) {
    double c[3];
    cross3d(a, b, c);
    return atan2(sqrt(dot3d(c, c)), dot3d(a, b));
}
/* x (unit) strictly inside the minor arc a->b (n = a x b) */
static int on_minor_arc(const double *a, const double *b, const double *n, const double *x) {
    double c1[3], c2[3];
    cross3d(a, x, c1);
    cross3d(x, b, c2);
    return dot3d(c1, n) > 0.0 && dot3d(c2, n) > 0.0;
}
/* proper intersection of minor arcs (a, b) and (c, d); 1 and the point in x */
static int arcs_cross(const double *a, const double *b, const double *c, const double *d, double *x, int *degen) {
    double n1[3], n2[3], s[3];
    cross3d(a, b, n1);
    cross3d(c, d, n2);
    cross3d(n1, n2, s);
    if (sqrt(dot3d(s, s)) < 1e-14 * sqrt(dot3d(n1, n1) * dot3d(n2, n2))) { *degen = 1; return 0; }
    normalize3d(s);
    for (int k = 0; k < 2; k++) {
        double y[3] = {k ? -s[0] : s[0], k ? -s[1] : s[1], k ? -s[2] : s[2]};
        if (on_minor_arc(a, b, n1, y) && on_minor_arc(c, d, n2, y)) {
            memcpy(x, y, sizeof(y));
            return 1;
        }
    }
    return 0;
}
/* tangent angle at x (unit) of the great circle toward y, in a frame at x */
static double tangent_angle(const double *x, const double *y) {
    double e1[3], e2[3], ax[3] = {1.0, 0.0, 0.0};
    if (fabs(x[0]) > 0.6) { ax[0] = 0.0; ax[1] = 1.0; }
    cross3d(x, ax, e1);
    normalize3d(e1);
    cross3d(x, e1, e2);
    double t[3], xy = dot3d(x, y);
    for (int k = 0; k < 3; k++) t[k] = y[k] - xy * x[k];
    return atan2(dot3d(t, e2), dot3d(t, e1));
}

static int uf_find(int *par, int i) {
    while (par[i] != i) { par[i] = par[par[i]]; i = par[i]; }
    return i;
}

static int cmp_xing(const void *x, const void *y) {
    const sxing_t *a = (const sxing_t *)x, *b = (const sxing_t *)y;
    if (a->arc != b->arc) return a->arc < b->arc ? -1 : 1;
    return a->t < b->t ? -1 : (a->t > b->t ? 1 : 0);
}

typedef struct { int h; double ang; } sout_t;
static int cmp_out(const void *x, const void *y) {
    const sout_t *a = (const sout_t *)x, *b = (const sout_t *)y;
    return a->ang < b->ang ? -1 : (a->ang > b->ang ? 1 : 0);
}

ORACLE_API int oracle_w3d_alg1(const float *V, int64_t nv, const int32_t *F, int64_t nf, const float *p,
                               double *w_out, double *info) {
    (void)nv;
    int rc = 0;
    int32_t *src = NULL, *dst = NULL, *mul = NULL, *vmap = NULL, *par = NULL, *vis = NULL;
    double *pts = NULL, *area = NULL;
    sarc_t *arcs = NULL;
    sxing_t *xs = NULL;
    spiece_t *pc = NULL;
    int *hnext = NULL, *hface = NULL, *ostart = NULL, *ocnt = NULL, *chi = NULL, *queue = NULL;
    sout_t *outs = NULL;
    int64_t ncap = 3 * (nf > 0 ? nf : 1);
    src = (int32_t *)malloc(sizeof(int32_t) * ncap);
    dst = (int32_t *)malloc(sizeof(int32_t) * ncap);
    mul = (int32_t *)malloc(sizeof(int32_t) * ncap);
    if (!src || !dst || !mul) { rc = -3; goto done; }
    int64_t ne = oracle_boundary_edges(F, nf, src, dst, mul);
    if (ne < 0) { rc = -3; goto done; }
    const double P3[3] = {p[0], p[1], p[2]};
    const double fourpi = 4.0 * M_PI;
    if (ne == 0) {
        /* closed: one region, the whole sphere; chi of any ray */
        float d[3] = {0.48f, 0.6f, 0.64f};
        int c = 0;
        for (int64_t t = 0; t < nf; t++)
            c += tri_crossing(V + 3 * (int64_t)F[3 * t], V + 3 * (int64_t)F[3 * t + 1], V + 3 * (int64_t)F[3 * t + 2],
                              p, d);
        *w_out = (double)c;
        if (info) { info[0] = 1; info[1] = fourpi; info[2] = c; }
        goto done;
    }
    /* 1. projected boundary vertices (one point per mesh vertex) */
    int64_t nvm = 0;
    for (int64_t e = 0; e < ne; e++) { if (src[e] + 1 > nvm) nvm = src[e] + 1; if (dst[e] + 1 > nvm) nvm = dst[e] + 1; }
    vmap = (int32_t *)malloc(sizeof(int32_t) * nvm);
    if (!vmap) { rc = -3; goto done; }
    for (int64_t i = 0; i < nvm; i++) vmap[i] = -1;
    int npt = 0;
    for (int64_t e = 0; e < ne; e++) {
        if (vmap[src[e]] < 0) vmap[src[e]] = npt++;
        if (vmap[dst[e]] < 0) vmap[dst[e]] = npt++;
    }
    int narc_b = (int)ne, ncomp_max = npt;
    int pt_cap = npt + 4 * (narc_b + ncomp_max) * (narc_b + ncomp_max) + 16;
    pts = (double *)malloc(sizeof(double) * 3 * pt_cap);
    arcs = (sarc_t *)malloc(sizeof(sarc_t) * (narc_b + ncomp_max));
    par = (int32_t *)malloc(sizeof(int32_t) * npt);
    if (!pts || !arcs || !par) { rc = -3; goto done; }
    for (int64_t i = 0; i < nvm; i++) {
        if (vmap[i] < 0) continue;
        double *x = pts + 3 * vmap[i];
        for (int k = 0; k < 3; k++) x[k] = (double)V[3 * i + k] - P3[k];
        if (normalize3d(x)) { rc = -1; goto done; }         /* p on a boundary vertex */
    }
    int narc = 0;
    for (int64_t e = 0; e < ne; e++) {
        arcs[narc].a = vmap[src[e]]; arcs[narc].b = vmap[dst[e]]; arcs[narc].w = mul[e];
        if (dot3d(pts + 3 * arcs[narc].a, pts + 3 * arcs[narc].b) < -1.0 + 1e-12) { rc = -1; goto done; }
        narc++;
    }
    /* 2. join separate components with arcs of weight zero */
    for (int i = 0; i < npt; i++) par[i] = i;
    for (int i = 0; i < narc; i++) {
        int ra = uf_find(par, arcs[i].a), rb = uf_find(par, arcs[i].b);
        if (ra != rb) par[ra] = rb;
    }
    int root0 = uf_find(par, 0);
    for (int i = 1; i < npt; i++) {
        int ri = uf_find(par, i);
        if (ri == root0) continue;
        /* bridge from point 0 to the first point of this component that is not antipodal to it */
        int j = -1;
        for (int k = i; k < npt; k++)
            if (uf_find(par, k) == ri && dot3d(pts, pts + 3 * k) > -1.0 + 1e-6) { j = k; break; }
        if (j < 0) { rc = -1; goto done; }
        arcs[narc].a = 0; arcs[narc].b = j; arcs[narc].w = 0;
        narc++;
        par[ri] = root0;
    }
    /* 3. pairwise proper intersections */
    int xcap = 2 * narc * narc + 2;
    xs = (sxing_t *)malloc(sizeof(sxing_t) * xcap);
    if (!xs) { rc = -3; goto done; }
    int nx = 0;
    for (int i = 0; i < narc; i++)
        for (int j = i + 1; j < narc; j++) {
            const sarc_t *A = &arcs[i], *B = &arcs[j];
            if (A->a == B->a || A->a == B->b || A->b == B->a || A->b == B->b) continue;
            double x[3];
            int degen = 0;
            if (arcs_cross(pts + 3 * A->a, pts + 3 * A->b, pts + 3 * B->a, pts + 3 * B->b, x, &degen)) {
                if (npt >= pt_cap) { rc = -3; goto done; }
                int vid = npt++;
                memcpy(pts + 3 * vid, x, sizeof(x));
                xs[nx].arc = i; xs[nx].other = j; xs[nx].t = arc_angle(pts + 3 * A->a, x); xs[nx].vid = vid; nx++;
                xs[nx].arc = j; xs[nx].other = i; xs[nx].t = arc_angle(pts + 3 * B->a, x); xs[nx].vid = vid; nx++;
            } else if (degen) { rc = -1; goto done; }
        }
    qsort(xs, (size_t)nx, sizeof(sxing_t), cmp_xing);
    /* 4. arc pieces */
    int npc = 0, pcap = narc + nx;
    pc = (spiece_t *)malloc(sizeof(spiece_t) * pcap);
    if (!pc) { rc = -3; goto done; }
    for (int i = 0, k = 0; i < narc; i++) {
        int prev = arcs[i].a;
        while (k < nx && xs[k].arc == i) {
            pc[npc].u = prev; pc[npc].v = xs[k].vid; pc[npc].w = arcs[i].w; npc++;
            prev = xs[k].vid;
            k++;
        }
        pc[npc].u = prev; pc[npc].v = arcs[i].b; pc[npc].w = arcs[i].w; npc++;
    }
    /* 5. half-edges (2k: u->v, 2k+1: v->u), out-edges sorted by tangent angle */
    int nh = 2 * npc;
    hnext = (int *)malloc(sizeof(int) * nh);
    hface = (int *)malloc(sizeof(int) * nh);
    ostart = (int *)calloc((size_t)npt + 1, sizeof(int));
    ocnt = (int *)calloc((size_t)npt, sizeof(int));
    outs = (sout_t *)malloc(sizeof(sout_t) * nh);
    int *hpos = (int *)malloc(sizeof(int) * nh);
    if (!hnext || !hface || !ostart || !ocnt || !outs || !hpos) { free(hpos); rc = -3; goto done; }
#define H_ORIG(h) (((h) & 1) ? pc[(h) >> 1].v : pc[(h) >> 1].u)
#define H_DEST(h) (((h) & 1) ? pc[(h) >> 1].u : pc[(h) >> 1].v)
    for (int h = 0; h < nh; h++) ostart[H_ORIG(h) + 1]++;
    for (int i = 0; i < npt; i++) ostart[i + 1] += ostart[i];
    for (int h = 0; h < nh; h++) {
        int o = H_ORIG(h);
        int slot = ostart[o] + ocnt[o]++;
        outs[slot].h = h;
        outs[slot].ang = tangent_angle(pts + 3 * o, pts + 3 * H_DEST(h));
    }
    for (int i = 0; i < npt; i++) {
        qsort(outs + ostart[i], (size_t)(ostart[i + 1] - ostart[i]), sizeof(sout_t), cmp_out);
        for (int s = ostart[i]; s < ostart[i + 1]; s++) hpos[outs[s].h] = s;
    }
    /* next(h): at the head v of h, the out-edge just clockwise from twin(h) */
    for (int h = 0; h < nh; h++) {
        int v = H_DEST(h), tw = h ^ 1;
        int s = hpos[tw], lo = ostart[v], n = ostart[v + 1] - ostart[v];
        int sp = lo + ((s - lo) - 1 + n) % n;
        hnext[h] = outs[sp].h;
    }
    /* 6. faces and their areas */
    for (int h = 0; h < nh; h++) hface[h] = -1;
    int nfc = 0;
    area = (double *)malloc(sizeof(double) * nh);
    if (!area) { free(hpos); rc = -3; goto done; }
    for (int h0 = 0; h0 < nh; h0++) {
        if (hface[h0] >= 0) continue;
        double turn = 0.0;
        int h = h0, guard = 0;
        do {
            hface[h] = nfc;
            int hn = hnext[h], v = H_DEST(h);
            /* interior angle at v: from the outgoing direction counter-clockwise to the reversed incoming one */
            double a_out = outs[hpos[hn]].ang, a_in = outs[hpos[h ^ 1]].ang;
            double alpha = fmod(a_in - a_out + 4.0 * M_PI, 2.0 * M_PI);
            if (alpha <= 0.0) alpha += 2.0 * M_PI;
            turn += M_PI - alpha;
            (void)v;
            h = hn;
            if (++guard > nh + 1) { free(hpos); rc = -2; goto done; }
        } while (h != h0);
        area[nfc++] = 2.0 * M_PI - turn;
    }
    double asum = 0.0;
    int big = 0;
    for (int f = 0; f < nfc; f++) {
        asum += area[f];
        if (area[f] > area[big]) big = f;
    }
    if (fabs(asum - fourpi) > 1e-9) { free(hpos); rc = -2; goto done; }
    /* 7. one ray into the largest region: midpoint of its longest side,
     *    offset to the left by an angle that crosses no arc */
    int hl = -1;
    double best = -1.0;
    for (int h = 0; h < nh; h++)
        if (hface[h] == big) {
            double L = arc_angle(pts + 3 * H_ORIG(h), pts + 3 * H_DEST(h));
            if (L > best) { best = L; hl = h; }
        }
    double m[3], t[3], l[3], q[3];
    {
        const double *u = pts + 3 * H_ORIG(hl), *v = pts + 3 * H_DEST(hl);
        for (int k = 0; k < 3; k++) m[k] = u[k] + v[k];
        normalize3d(m);
        double vm = 0.0;
        for (int k = 0; k < 3; k++) t[k] = v[k] - u[k];
        vm = dot3d(t, m);
        for (int k = 0; k < 3; k++) t[k] -= vm * m[k];
        normalize3d(t);
        cross3d(m, t, l);
    }
    double delta = 0.25 * best;
    int ok = 0;
    for (int it = 0; it < 60 && !ok; it++, delta *= 0.5) {
        for (int k = 0; k < 3; k++) q[k] = cos(delta) * m[k] + sin(delta) * l[k];
        normalize3d(q);
        ok = 1;
        for (int k = 0; k < npc && ok; k++) {
            if (k == (hl >> 1)) continue;
            double x[3];
            int degen = 0;
            if (arcs_cross(m, q, pts + 3 * pc[k].u, pts + 3 * pc[k].v, x, &degen) || degen) ok = 0;
        }
        if (delta < 1e-5) break;
    }
    if (!ok) { free(hpos); rc = -1; goto done; }
    float dq[3] = {(float)q[0], (float)q[1], (float)q[2]};
    int c0 = 0;
    for (int64_t tr = 0; tr < nf; tr++)
        c0 += tri_crossing(V + 3 * (int64_t)F[3 * tr], V + 3 * (int64_t)F[3 * tr + 1], V + 3 * (int64_t)F[3 * tr + 2],
                           p, dq);
    /* 8. chi of every region from the largest one across the arcs (Lemma 2):
     *    chi(left of a piece) - chi(right of it) = its weight */
    chi = (int *)malloc(sizeof(int) * nfc);
    vis = (int32_t *)calloc((size_t)nfc, sizeof(int32_t));
    queue = (int *)malloc(sizeof(int) * nfc);
    if (!chi || !vis || !queue) { free(hpos); rc = -3; goto done; }
    int qh = 0, qt = 0;
    chi[big] = c0; vis[big] = 1; queue[qt++] = big;
    while (qh < qt) {
        int f = queue[qh++];
        for (int h = 0; h < nh; h++) {
            if (hface[h] != f) continue;
            int g = hface[h ^ 1];
            int wgt = (h & 1) ? -pc[h >> 1].w : pc[h >> 1].w;    /* along the arc: f is its left side */
            int cg = chi[f] - wgt;
            if (!vis[g]) { vis[g] = 1; chi[g] = cg; queue[qt++] = g; }
            else if (chi[g] != cg) { free(hpos); rc = -2; goto done; }
        }
    }
    if (qt != nfc) { free(hpos); rc = -2; goto done; }
    /* 9. the area-weighted sum */
    double acc = 0.0;
    for (int f = 0; f < nfc; f++) acc += area[f] * (double)chi[f];
    *w_out = acc / fourpi;
    if (info) { info[0] = nfc; info[1] = area[big]; info[2] = c0; }
    free(hpos);
#undef H_ORIG
#undef H_DEST
done:
    free(src); free(dst); free(mul); free(vmap); free(par); free(vis); free(pts); free(area); free(arcs); free(xs);
    free(pc); free(hnext); free(hface); free(ostart); free(ocnt); free(chi); free(queue); free(outs);
    return rc;
}

/* ======================================================================== */
/* 3D definition for bicubic Bezier patches (parametric surfaces)           */
/* ======================================================================== */
/* w(p) = (1/4 pi) sum_patches int_0^1 int_0^1 (f - p) . (f_u x f_v) / |f - p|^3 du dv
 * (Background: w_M(p) = (1/4 pi) int_M dOmega; for a parametric patch f(u, v)
 * the solid-angle element is (f - p) . (f_u x f_v) du dv / |f - p|^3).
 * f(u, v) = sum_ij B_i(u) B_j(v) P_ij with cubic Bernstein B; ctrl holds
 * P_ij at ((patch * 4 + i) * 4 + j) * 3, float32 promoted exactly.
 * Quadrature: tensor 8-point Gauss-Legendre on a cell, accepted when it agrees
 * with the sum over the cell's four quarters to tol (scaled by the cell's
 * share of the domain), else the quarters are refined (depth <= 12). */
static const double GL8X[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290, -0.1834346424956498,
                               0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
static const double GL8W[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873, 0.3626837833783620,
                               0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};

static void bern3_basis(double u, double *b, double *db) {
    double v = 1.0 - u;
    b[0] = v * v * v; b[1] = 3.0 * u * v * v; b[2] = 3.0 * u * u * v; b[3] = u * u * u;
    db[0] = -3.0 * v * v; db[1] = 3.0 * v * v - 6.0 * u * v; db[2] = 6.0 * u * v - 3.0 * u * u; db[3] = 3.0 * u * u;
}

static double patch_integrand(const double *P, const double *p, double u, double v) {
    double bu[4], dbu[4], bv[4], dbv[4];
    bern3_basis(u, bu, dbu);
    bern3_basis(v, bv, dbv);
    double f[3] = {0, 0, 0}, fu[3] = {0, 0, 0}, fv[3] = {0, 0, 0};
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            const double *q = P + 3 * (4 * i + j);
            double w0 = bu[i] * bv[j], w1 = dbu[i] * bv[j], w2 = bu[i] * dbv[j];
            for (int k = 0; k < 3; k++) { f[k] += w0 * q[k]; fu[k] += w1 * q[k]; fv[k] += w2 * q[k]; }
        }
    double r[3] = {f[0] - p[0], f[1] - p[1], f[2] - p[2]}, n[3];
    cross3d(fu, fv, n);
    double r2 = dot3d(r, r);
    return dot3d(r, n) / (r2 * sqrt(r2));
}

static double patch_cell_gl8(const double *P, const double *p, double u0, double v0, double h) {
    double s = 0.0;
    for (int a = 0; a < 8; a++) {
        double u = u0 + 0.5 * h * (1.0 + GL8X[a]);
        for (int b = 0; b < 8; b++) {
            double v = v0 + 0.5 * h * (1.0 + GL8X[b]);
            s += GL8W[a] * GL8W[b] * patch_integrand(P, p, u, v);
        }
    }
    return s * 0.25 * h * h;
}

static double patch_adapt(const double *P, const double *p, double u0, double v0, double h, double whole,
                          double tol, int depth) {
    double hh = 0.5 * h;
    double q[4] = {patch_cell_gl8(P, p, u0, v0, hh), patch_cell_gl8(P, p, u0 + hh, v0, hh),
                   patch_cell_gl8(P, p, u0, v0 + hh, hh), patch_cell_gl8(P, p, u0 + hh, v0 + hh, hh)};
    double fine = q[0] + q[1] + q[2] + q[3];
    if (fabs(fine - whole) <= tol * h * h || depth >= 12) return fine;
    return patch_adapt(P, p, u0, v0, hh, q[0], tol, depth + 1) + patch_adapt(P, p, u0 + hh, v0, hh, q[1], tol, depth + 1) +
           patch_adapt(P, p, u0, v0 + hh, hh, q[2], tol, depth + 1) +
           patch_adapt(P, p, u0 + hh, v0 + hh, hh, q[3], tol, depth + 1);
}

typedef struct {
    const float *ctrl; int64_t npatch; const float *P; double *w; double tol;
} pq_ctx;

static void patch_quad_range(void *vp, int64_t lo, int64_t hi) {
    pq_ctx *c = (pq_ctx *)vp;
    double Pd[48];
    for (int64_t q = lo; q < hi; q++) {
        double p[3] = {c->P[3 * q], c->P[3 * q + 1], c->P[3 * q + 2]};
        double acc = 0.0;
        for (int64_t t = 0; t < c->npatch; t++) {
            for (int k = 0; k < 48; k++) Pd[k] = (double)c->ctrl[48 * t + k];
            double whole = patch_cell_gl8(Pd, p, 0.0, 0.0, 1.0);
            acc += patch_adapt(Pd, p, 0.0, 0.0, 1.0, whole, c->tol, 0);
        }
        c->w[q] = acc / (4.0 * M_PI);
    }
}

ORACLE_API void oracle_w3d_patches_quad(const float *ctrl, int64_t npatch, const float *P, int64_t nq, double *w,
                                        double tol, int nthreads) {
    pq_ctx c = {ctrl, npatch, P, w, tol};
    parallel_for(nq, nthreads, patch_quad_range, &c);
}
