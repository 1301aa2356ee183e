// query.cuh -- query point generation on the device (grids and point lists).
#pragma once
#include "gwn_internal.h"

namespace gwn {

// 3D query point `i`: grid coordinates come from per-axis float32 tables
// (x fastest), point lists are float32 [n x 3] row-major.
__device__ __forceinline__ float3 query_point3(const QuerySrc &q, int64_t i) {
    if (q.kind == GWN_QUERY_GRID) {
        unsigned ii = (unsigned)i;
        unsigned nx = (unsigned)q.dims[0], ny = (unsigned)q.dims[1];
        unsigned ix = ii % nx, t = ii / nx;
        unsigned iy = t % ny, iz = t / ny;
        return make_float3(__ldg(&q.ax[0][ix]), __ldg(&q.ax[1][iy]), __ldg(&q.ax[2][iz]));
    }
    const float *p = q.pts + 3 * i;
    return make_float3(__ldg(p), __ldg(p + 1), __ldg(p + 2));
}

// Bin of coordinate v on a bin axis starting at v0 with inv = bins per unit:
// clamp(floor((v - v0) * inv), 0, nb - 1) with explicitly rounded operations,
// so it is monotone non-decreasing in v (fmaxf maps NaN to bin 0).
__device__ __forceinline__ int bin_of(float v, float v0, float inv, int nb) {
    float f = floorf(__fmul_rn(__fsub_rn(v, v0), inv));
    f = fminf(fmaxf(f, 0.f), (float)(nb - 1));
    return (int)f;
}

// Spatially coherent thread -> grid point mapping for the crossing traversal:
// a 256-thread block covers an 8 x 8 x 4 tile of the grid and each warp a
// 4 x 4 x 2 sub-tile, so the 32 rays of a warp are neighbours in the
// projection plane and traverse nearly the same nodes.  Returns the flat
// query index, or -1 for threads outside the grid.  Requires blockDim.x = 256.
__device__ __forceinline__ int64_t grid_tile_query(const QuerySrc &q) {
    unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    unsigned x = 4u * (warp & 1u) + (lane & 3u);
    unsigned y = 4u * ((warp >> 1) & 1u) + ((lane >> 2) & 3u);
    unsigned z = 2u * (warp >> 2) + (lane >> 4);
    unsigned tx = (unsigned)((q.dims[0] + 7) / 8), ty = (unsigned)((q.dims[1] + 7) / 8);
    unsigned b = blockIdx.x;
    unsigned bx = b % tx, t = b / tx, by = t % ty, bz = t / ty;
    int64_t ix = 8 * (int64_t)bx + x, iy = 8 * (int64_t)by + y, iz = 4 * (int64_t)bz + z;
    if (ix >= q.dims[0] || iy >= q.dims[1] || iz >= q.dims[2]) return -1;
    return ix + q.dims[0] * (iy + q.dims[1] * iz);
}

__host__ __forceinline__ int64_t grid_tile_blocks(const QuerySrc &q) {
    return ((q.dims[0] + 7) / 8) * ((q.dims[1] + 7) / 8) * ((q.dims[2] + 3) / 4);
}

}  // namespace gwn
