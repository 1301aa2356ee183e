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

cudaError_t launch_bterm3d(const float4 *bseq, int64_t n_bseq, const Frame &fr, const QuerySrc &q,
                           const int32_t *chi, float *w_out, float *b_out, unsigned long long *cnt,
                           int *status, int sm_count, cudaStream_t st) {
    (void)sm_count;
    if (q.n == 0) return cudaSuccess;
    constexpr int K = 4;
    const int threads = 256;
    int64_t per_block = (int64_t)threads * K;
    int64_t blocks = (q.n + per_block - 1) / per_block;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    bterm3d_kernel<K><<<(unsigned)blocks, threads, 0, st>>>(bseq, (int)n_bseq, fr, q, chi, w_out, b_out,
                                                            cnt, status);
    return cudaGetLastError();
}

}  // namespace gwn
