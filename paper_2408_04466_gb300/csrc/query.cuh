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

}  // namespace gwn
