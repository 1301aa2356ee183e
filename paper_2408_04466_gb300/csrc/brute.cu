// brute.cu -- brute-force comparator: w(p) = (1/4pi) sum over ALL triangles of
// the signed solid angle (Background: w_M = (1/4pi) int_M dOmega), one query
// per thread, triangles streamed through shared memory in tiles, float32 with
// compensated accumulation.  This is the standard method the one-shot path is
// measured against on the same GPU.
#include "gwn_internal.h"
#include "query.cuh"

namespace gwn {

constexpr int BF_TILE = 256;

__global__ void __launch_bounds__(256) bruteforce3d_kernel(const float *__restrict__ V,
                                                           const int32_t *__restrict__ F, int64_t nf,
                                                           QuerySrc q, float *__restrict__ w_out) {
    __shared__ float4 tri[BF_TILE][3];
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float3 p = idx < q.n ? query_point3(q, idx) : make_float3(0.f, 0.f, 0.f);
    float sum = 0.f, cmp = 0.f;
    for (int64_t t0 = 0; t0 < nf; t0 += BF_TILE) {
        __syncthreads();
        for (int k = threadIdx.x; k < BF_TILE; k += blockDim.x) {
            int64_t t = t0 + k;
            for (int c = 0; c < 3; c++) {
                if (t < nf) {
                    int vi = F[3 * t + c];
                    tri[k][c] = make_float4(V[3 * (int64_t)vi], V[3 * (int64_t)vi + 1], V[3 * (int64_t)vi + 2], 0.f);
                } else {
                    tri[k][c] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        }
        __syncthreads();
        int cnt = (int)(nf - t0 < BF_TILE ? nf - t0 : BF_TILE);
        for (int k = 0; k < cnt; k++) {
            float4 A = tri[k][0], B = tri[k][1], C = tri[k][2];
            float ax = A.x - p.x, ay = A.y - p.y, az = A.z - p.z;
            float bx = B.x - p.x, by = B.y - p.y, bz = B.z - p.z;
            float cx = C.x - p.x, cy = C.y - p.y, cz = C.z - p.z;
            float la = sqrtf(ax * ax + ay * ay + az * az);
            float lb = sqrtf(bx * bx + by * by + bz * bz);
            float lc = sqrtf(cx * cx + cy * cy + cz * cz);
            float num = ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx);
            float den = la * lb * lc + (ax * bx + ay * by + az * bz) * lc + (ax * cx + ay * cy + az * cz) * lb +
                        (bx * cx + by * cy + bz * cz) * la;
            float th = atan2f(num, den);
            float y = th - cmp;
            float tt = sum + y;
            cmp = (tt - sum) - y;
            sum = tt;
        }
    }
    if (idx < q.n) w_out[idx] = (sum - cmp) * 0.15915494309189535f;   // (2 theta) / 4pi
}

cudaError_t launch_bruteforce3d(const float *V, const int32_t *F, int64_t nf, const QuerySrc &q, float *w_out,
                                int sm_count, cudaStream_t st) {
    (void)sm_count;
    if (q.n == 0) return cudaSuccess;
    int64_t blocks = (q.n + 255) / 256;
    bruteforce3d_kernel<<<(unsigned)blocks, 256, 0, st>>>(V, F, nf, q, w_out);
    return cudaGetLastError();
}

}  // namespace gwn
