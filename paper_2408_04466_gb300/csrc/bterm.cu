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
// * a boundary vertex close to the forward ray: its azimuth around the ray
//   must be accurate to well inside the 0.01 cut band, or a branch flip
//   could hide from it.  Each vertex enters both of its edges only through
//   its stereographic coordinate zeta = (a1 + i a2)/s_a, so rounding acts as
//   one perturbation of its direction shared by both edges; only the azimuth
//   error matters.  The main pass forms (a1, a2, a_n) as double-float
//   differences (project below): azimuth error ~2u + u^2 (|A|+|p|)/|a_perp|,
//   so it flags only vertices within T = 1e-6 rad (margin ~100 for
//   |a| >= 1e-4).  The careful pass uses plain float32 projections of A - p
//   (azimuth error ~4u/delta) with T = 2e-4 (error <= 1.2e-3) and recomputes
//   the edges of such vertices in float64.  Edges are flagged by
//   |num + i den| < 1.01 T |a||b|, which every edge of such a vertex
//   satisfies since |z|/(|a||b|) <= sin(delta) + 2 sin^2(delta) for an
//   endpoint at angle delta from the ray.  A vertex exactly on the ray
//   (decided exactly) is
//   seen by the perturbed ray d_eps in the direction -dp (dp = the first of
//   e_x, e_y, e_z not parallel to d, projected orthogonally to d), and its
//   edges take the limit of Omega under that perturbation.
//
// Arithmetic: two queries per 64-bit register pair; plain add/mul/fma run as
// packed f32x2 instructions (Blackwell), min/max, MUFU (rsqrt, reciprocal),
// compares and selects per element.  atan2(num, den) uses the half-angle
// identity (see edge_theta) so that a single odd polynomial on [-1, 1]
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

#include "bterm.cuh"

namespace gwn {

template <int KP, int MINB>   // KP query pairs per thread, MINB blocks per SM
__global__ void __launch_bounds__(256, MINB) bterm3d_kernel(const float4 *__restrict__ bframe, int nb, Frame fr,
                                                            const __grid_constant__ PackedConsts Kp, QuerySrc q,
                                                            const int32_t *__restrict__ chi,
                                                            float *__restrict__ w_out, float *__restrict__ b_out,
                                                            uint8_t *__restrict__ in_out,
                                                            int32_t *__restrict__ defer, int32_t *defer_count) {
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * (2 * KP) + threadIdx.x;
    const int64_t gofs = 0;
#include "bterm_main_pass.inc"
}

// Boundary records in the frame of d as double-float values: for record k,
// out[2k] = (hi of A.e1, A.e2, A.n, w), out[2k + 1] = (lo parts, 0).
__global__ void bframe_kernel(const float4 *__restrict__ bseq, int64_t n, Frame fr, float4 *__restrict__ out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float4 v = bseq[k];
    const float *e[3] = {fr.e1, fr.e2, fr.n};
    float h[3], l[3];
    for (int c = 0; c < 3; c++) {
        double x = (double)v.x * e[c][0] + (double)v.y * e[c][1] + (double)v.z * e[c][2];
        h[c] = (float)x;
        l[c] = (float)(x - (double)h[c]);
    }
    out[2 * k] = make_float4(h[0], h[1], h[2], v.w);
    out[2 * k + 1] = make_float4(l[0], l[1], l[2], 0.f);
}

cudaError_t launch_bframe(const float4 *bseq, int64_t n, const Frame &fr, float4 *out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    bframe_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(bseq, n, fr, out);
    return cudaGetLastError();
}


// The careful pass: one block of 128 threads per deferred query
// (careful_block_B), persistent grid over the list.
__global__ void __launch_bounds__(128) bterm3d_careful_kernel(const float4 *__restrict__ bseq, int nb, Frame fr,
                                                              Frame64 f64, QuerySrc q, const int32_t *chi,
                                                              float *w_out, float *b_out, uint8_t *in_out,
                                                              const int32_t *__restrict__ defer,
                                                              const int32_t *defer_count, unsigned long long *cnt,
                                                              int *status) {
    int64_t n = *defer_count;
    if (n > q.n) n = q.n;
    if (cnt && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&cnt[CNT_DEFER_BTERM], (unsigned long long)n);
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {   // block-uniform loop
        int64_t idx = defer[i];
        if (idx < 0 || idx >= q.n) {
            if (threadIdx.x == 0) atomicOr(status, ST_BAD_INPUT);
            continue;
        }
        const float Bv = careful_block_B(bseq, nb, fr, f64, query_point3(q, idx), cnt, status);
        if (threadIdx.x == 0) {
            float wv = __fadd_rn(Bv, chi ? (float)chi[idx] : 0.f);
            if (b_out) b_out[idx] = Bv;
            if (w_out) w_out[idx] = wv;
            if (in_out) in_out[idx] = wv >= 0.5f ? 1 : 0;
        }
        __syncthreads();
    }
}

PackedConsts bterm_consts() {
    PackedConsts K;
    auto dup = [](float x) { return make_float2(x, x); };
    const float c[9] = {GWN_AT_C0, GWN_AT_C1, GWN_AT_C2, GWN_AT_C3, GWN_AT_C4, GWN_AT_C5, GWN_AT_C6, GWN_AT_C7,
                        GWN_AT_C8};
    for (int i = 0; i < 9; i++) K.c[i] = dup(c[i]);
    K.pi = dup(3.14159265358979f);
    K.nearv = dup(-5e-13f);         // -T^2 / 2, T = 1e-6 (double-float projections)
    K.spin = dup(-1e-2f);           // tau
    K.cut2n = dup(-1e-4f);
    return K;
}

template <int KP, int MINB>
static cudaError_t launch_bt(const float4 *bseq, const float4 *bframe, int64_t n_bseq, const Frame &fr,
                             const Frame64 &f64, const QuerySrc &q, const int32_t *chi, float *w_out, float *b_out,
                             uint8_t *in_out, int32_t *defer, int32_t *defer_count, unsigned long long *cnt,
                             int *status, int sm_count, cudaStream_t st) {
    const int threads = 256;
    int64_t per_block = (int64_t)threads * 2 * KP;
    int64_t blocks = (q.n + per_block - 1) / per_block;
    if (blocks > 0x7fffffff || q.n > 0x7fffffff) return cudaErrorInvalidValue;
    const PackedConsts K = bterm_consts();
    cudaError_t e = cudaMemsetAsync(defer_count, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    bterm3d_kernel<KP, MINB><<<(unsigned)blocks, threads, 0, st>>>(bframe, (int)n_bseq, fr, K, q, chi, w_out, b_out,
                                                                   in_out, defer, defer_count);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // deferred queries (a fraction of a percent): persistent grid over the list
    int cblocks = (sm_count > 0 ? sm_count : 152) * 4;
    bterm3d_careful_kernel<<<cblocks, 128, 0, st>>>(bseq, (int)n_bseq, fr, f64, q, chi, w_out, b_out, in_out,
                                                    defer, defer_count, cnt, status);
    return cudaGetLastError();
}

cudaError_t launch_bterm3d(const float4 *bseq, const float4 *bframe, int64_t n_bseq, const Frame &fr,
                           const Frame64 &f64, const QuerySrc &q, const int32_t *chi, float *w_out, float *b_out,
                           int32_t *defer, int32_t *defer_count, unsigned long long *cnt, int *status, int sm_count,
                           cudaStream_t st, uint8_t *inside_out) {
    if (q.n == 0) return cudaSuccess;
    // Two query pairs per thread at two blocks per SM: the fastest of the
    // (pairs, blocks) shapes measured for 16.8M queries x 252 boundary edges.
    return launch_bt<2, 2>(bseq, bframe, n_bseq, fr, f64, q, chi, w_out, b_out, inside_out, defer, defer_count, cnt,
                           status, sm_count, st);
}

}  // namespace gwn
