// bvh.cu -- on-device LBVH over triangles in the frame of the ray direction.
//
// Steps (all on the context's stream):
//   1. per triangle: frame coordinates (e1, e2, dh) of its vertices, a padded
//      box (x0, x1, y0, y1, zmax) and its centroid;
//   2. centroid bounds (block reduction + atomics on order-preserving ints);
//   3. 63-bit Morton codes (21 bits per frame axis) of the centroids;
//   4. stable LSD radix sort of (code, triangle) pairs, 8 bits per pass,
//      passes whose digit is constant over all keys are skipped;
//   5. binary radix tree from the sorted codes (Karras 2012: each internal
//      node finds its key range by the longest-common-prefix search, ties of
//      equal codes broken by the key index);
//   6. bottom-up box refit: one thread per leaf climbs while it is the second
//      child to arrive at a node (atomic counter per node);
//   7. packing: each internal node stores both children's boxes and refs;
//      triangles are re-laid out in sorted order as 3 float4.
// The boxes are padded by a bound on the float32 rounding of the frame
// coordinates (4e-7 times the vertex's 1-norm), so culling is conservative.
#include <string.h>

#include "gwn_internal.h"
#include "query.cuh"

namespace gwn {

namespace {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int BINS = 256;

__device__ __forceinline__ unsigned f2ord(float f) {
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// bounds: [0..2] min and [3..5] max centroid, [6] min x0, [7] max x1, [8] min
// y0, [9] max y1 of the padded boxes (order-preserving unsigned)
__global__ void tri_prep_kernel(const float *__restrict__ V, const int32_t *__restrict__ F, int64_t nf, Frame fr,
                                float4 *__restrict__ box_xy, float *__restrict__ box_z,
                                float4 *__restrict__ cen, unsigned *bounds) {
    __shared__ unsigned smin[5], smax[5];
    if (threadIdx.x < 5) { smin[threadIdx.x] = 0xffffffffu; smax[threadIdx.x] = 0u; }
    __syncthreads();
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nf) {
        float x0 = 3.4e38f, x1 = -3.4e38f, y0 = 3.4e38f, y1 = -3.4e38f, z1 = -3.4e38f;
        float cx = 0.f, cy = 0.f, cz = 0.f, pad = 0.f;
        for (int k = 0; k < 3; k++) {
            int vi = F[3 * t + k];
            float vx = V[3 * (int64_t)vi], vy = V[3 * (int64_t)vi + 1], vz = V[3 * (int64_t)vi + 2];
            float a = fmaf(vz, fr.e1[2], fmaf(vy, fr.e1[1], vx * fr.e1[0]));
            float b = fmaf(vz, fr.e2[2], fmaf(vy, fr.e2[1], vx * fr.e2[0]));
            float c = fmaf(vz, fr.dh[2], fmaf(vy, fr.dh[1], vx * fr.dh[0]));
            x0 = fminf(x0, a); x1 = fmaxf(x1, a);
            y0 = fminf(y0, b); y1 = fmaxf(y1, b);
            z1 = fmaxf(z1, c);
            cx += a; cy += b; cz += c;
            pad = fmaxf(pad, fabsf(vx) + fabsf(vy) + fabsf(vz));
        }
        pad = pad * 4e-7f + 1e-30f;
        box_xy[t] = make_float4(x0 - pad, x1 + pad, y0 - pad, y1 + pad);
        atomicMin(&smin[3], f2ord(x0 - pad)); atomicMax(&smax[3], f2ord(x1 + pad));
        atomicMin(&smin[4], f2ord(y0 - pad)); atomicMax(&smax[4], f2ord(y1 + pad));
        box_z[t] = z1 + pad;
        cx *= (1.f / 3.f); cy *= (1.f / 3.f); cz *= (1.f / 3.f);
        cen[t] = make_float4(cx, cy, cz, 0.f);
        atomicMin(&smin[0], f2ord(cx)); atomicMax(&smax[0], f2ord(cx));
        atomicMin(&smin[1], f2ord(cy)); atomicMax(&smax[1], f2ord(cy));
        atomicMin(&smin[2], f2ord(cz)); atomicMax(&smax[2], f2ord(cz));
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        atomicMin(&bounds[threadIdx.x], smin[threadIdx.x]);
        atomicMax(&bounds[3 + threadIdx.x], smax[threadIdx.x]);
    } else if (threadIdx.x < 5) {
        int k = threadIdx.x - 3;
        atomicMin(&bounds[6 + 2 * k], smin[threadIdx.x]);
        atomicMax(&bounds[7 + 2 * k], smax[threadIdx.x]);
    }
}

__device__ __forceinline__ unsigned long long spread21(unsigned v) {
    unsigned long long x = v & 0x1fffffull;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__global__ void morton_kernel(const float4 *__restrict__ cen, int64_t n, const unsigned *bounds,
                              unsigned long long *__restrict__ keys, int32_t *__restrict__ vals) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    float lo[3], ext[3];
    for (int k = 0; k < 3; k++) {
        lo[k] = ord2f(bounds[k]);
        ext[k] = ord2f(bounds[3 + k]) - lo[k];
    }
    float4 c = cen[t];
    float cc[3] = {c.x, c.y, c.z};
    unsigned long long code = 0;
    for (int k = 0; k < 3; k++) {
        float u = ext[k] > 0.f ? (cc[k] - lo[k]) / ext[k] : 0.f;
        u = fminf(fmaxf(u, 0.f), 1.f);
        unsigned q = (unsigned)(u * 2097151.0f);
        code |= spread21(q) << k;
    }
    keys[t] = code;
    vals[t] = (int32_t)t;
}

// ---- stable LSD radix sort --------------------------------------------------
__global__ void hist_kernel(const unsigned long long *__restrict__ keys, int64_t n, int shift,
                            unsigned *__restrict__ hist, int nblocks) {
    __shared__ unsigned h[BINS];
    for (int i = threadIdx.x; i < BINS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    for (int r = 0; r < SORT_ITEMS; r++) {
        int64_t i = base + (int64_t)r * SORT_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < BINS; i += blockDim.x) hist[(int64_t)i * nblocks + blockIdx.x] = h[i];
}

// Exclusive scan, in place, of the BINS x nblocks digit counts (digit-major,
// hist[digit * nblocks + tile]) by one block of SCAN_THREADS threads, in steps
// of SCAN_THREADS x 8 consecutive counts: each thread takes 8 (two 16-byte
// loads, coalesced across the block; the next step's loads are issued before
// this step is scanned), a warp scan by shuffle over the threads' sums, one
// warp scanning the 32 warp totals, and a running carry.  Counts and sums fit
// in 32 bits (fewer than 2^31 keys).  Then the same block flags the pass as
// skippable when one digit value holds every key.  hist's length BINS x
// nblocks is a multiple of 4, and its start is 256-byte aligned.
constexpr int SCAN_THREADS = 1024;
__global__ void __launch_bounds__(SCAN_THREADS) scan_skip_kernel(unsigned *data, int nblocks, int64_t total,
                                                                 int *skip) {
    __shared__ unsigned wsum[2][32];                 // alternate steps: one barrier per step
    __shared__ int s_skip;
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n4 = (int64_t)BINS * nblocks / 4;
    uint4 *d4 = reinterpret_cast<uint4 *>(data);
    const uint4 Z = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) s_skip = 0;
    int64_t j4 = 2 * (int64_t)tid;
    uint4 a = j4 < n4 ? d4[j4] : Z, b = j4 + 1 < n4 ? d4[j4 + 1] : Z;
    unsigned carry = 0;                               // the same value in every thread
    for (int step = 0; j4 - 2 * (int64_t)tid < n4; step++, j4 += 2 * SCAN_THREADS) {
        const int64_t k4 = j4 + 2 * SCAN_THREADS;
        const uint4 na = k4 < n4 ? d4[k4] : Z, nb = k4 + 1 < n4 ? d4[k4 + 1] : Z;
        const unsigned v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        unsigned sum = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) sum += v[k];
        unsigned x = sum;                             // inclusive over the warp's threads
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned y = __shfl_up_sync(FULL, x, off);
            if (lane >= off) x += y;
        }
        unsigned *ws = wsum[step & 1];
        if (lane == 31) ws[warp] = x;
        __syncthreads();
        unsigned wprev = 0, wall = 0;                 // warps before this one, and all warps
        {
            unsigned w = ws[lane], wi = w;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned y = __shfl_up_sync(FULL, wi, off);
                if (lane >= off) wi += y;
            }
            wprev = __shfl_sync(FULL, wi - w, warp);
            wall = __shfl_sync(FULL, wi, 31);
        }
        unsigned r = carry + wprev + (x - sum);
        unsigned o[8];
#pragma unroll
        for (int k = 0; k < 8; k++) { o[k] = r; r += v[k]; }
        if (j4 < n4) d4[j4] = make_uint4(o[0], o[1], o[2], o[3]);
        if (j4 + 1 < n4) d4[j4 + 1] = make_uint4(o[4], o[5], o[6], o[7]);
        carry += wall;
        a = na;
        b = nb;
    }
    __syncthreads();                     // the block's global writes are visible to the block
    for (int bn = tid; bn < BINS; bn += blockDim.x) {
        const unsigned long long start = data[(int64_t)bn * nblocks];
        const unsigned long long end = bn + 1 < BINS ? data[(int64_t)(bn + 1) * nblocks] : (unsigned long long)total;
        if (end - start == (unsigned long long)total) s_skip = 1;
    }
    __syncthreads();
    if (tid == 0) *skip = s_skip;
}

__global__ void scatter_kernel(const unsigned long long *__restrict__ kin, const int32_t *__restrict__ vin,
                               unsigned long long *__restrict__ kout, int32_t *__restrict__ vout, int64_t n,
                               int shift, const unsigned *__restrict__ scanned, int nblocks, const int *skip) {
    __shared__ unsigned wcount[SORT_THREADS / 32][BINS + 1];
    __shared__ unsigned running[BINS];
    __shared__ unsigned dbase[BINS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool skip_pass = *skip != 0;
    int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    if (skip_pass) {   // copy through unchanged
        for (int r = 0; r < SORT_ITEMS; r++) {
            int64_t i = base + (int64_t)r * SORT_THREADS + threadIdx.x;
            if (i < n) { kout[i] = kin[i]; vout[i] = vin[i]; }
        }
        return;
    }
    for (int i = threadIdx.x; i < BINS; i += blockDim.x) {
        running[i] = 0;
        dbase[i] = scanned[(int64_t)i * nblocks + blockIdx.x];
    }
    for (int i = threadIdx.x; i < (SORT_THREADS / 32) * (BINS + 1); i += blockDim.x) (&wcount[0][0])[i] = 0;
    __syncthreads();
    unsigned lanemask_lt = (1u << lane) - 1u;
    for (int r = 0; r < SORT_ITEMS; r++) {
        int64_t i = base + (int64_t)r * SORT_THREADS + threadIdx.x;
        bool valid = i < n;
        unsigned long long k = valid ? kin[i] : 0ull;
        int32_t v = valid ? vin[i] : 0;
        unsigned digit = valid ? ((unsigned)(k >> shift) & 255u) : (unsigned)BINS;
        unsigned peers = __match_any_sync(0xffffffffu, digit);
        unsigned rank = __popc(peers & lanemask_lt);
        int leader = __ffs(peers) - 1;
        if (lane == leader) wcount[warp][digit] = __popc(peers);
        __syncthreads();
        if (valid) {
            unsigned off = 0;
            for (int w = 0; w < warp; w++) off += wcount[w][digit];
            unsigned pos = dbase[digit] + running[digit] + off + rank;
            if ((int64_t)pos < n) {
                kout[pos] = k;
                vout[pos] = v;
            }
        }
        __syncthreads();
        for (int b = threadIdx.x; b < BINS; b += blockDim.x) {
            unsigned s = 0;
            for (int w = 0; w < SORT_THREADS / 32; w++) { s += wcount[w][b]; wcount[w][b] = 0; }
            running[b] += s;
        }
        for (int w = 0; w < SORT_THREADS / 32; w++)
            if (threadIdx.x == 0) wcount[w][BINS] = 0;
        __syncthreads();
    }
}

// ---- Karras binary radix tree ------------------------------------------------
__device__ __forceinline__ int delta(const unsigned long long *keys, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    unsigned long long a = keys[i], b = keys[j];
    if (a == b) return 64 + __clz((unsigned)(i ^ j));
    return __clzll(a ^ b);
}

__global__ void karras_kernel(const unsigned long long *__restrict__ keys, int64_t n, int2 *__restrict__ child,
                              int32_t *__restrict__ parent_int, int32_t *__restrict__ parent_leaf) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int dr = delta(keys, n, i, i + 1), dl = delta(keys, n, i, i - 1);
    int d = dr > dl ? 1 : -1;
    int dmin = d > 0 ? dl : dr;
    int64_t lmax = 2;
    while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    int64_t j = i + l * d;
    int dnode = delta(keys, n, i, j);
    int64_t s = 0;
    int64_t t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
    int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    int left = (lo == gamma) ? ~(int)gamma : (int)gamma;
    int right = (hi == gamma + 1) ? ~(int)(gamma + 1) : (int)(gamma + 1);
    child[i] = make_int2(left, right);
    if (left < 0) parent_leaf[~left] = (int32_t)i; else parent_int[left] = (int32_t)i;
    if (right < 0) parent_leaf[~right] = (int32_t)i; else parent_int[right] = (int32_t)i;
    if (i == 0) parent_int[0] = -1;
}

struct Box5 { float x0, x1, y0, y1, z1; };

__device__ __forceinline__ bool ref_ok(int r, int64_t n) { return r < 0 ? (int64_t)(~r) < n : (int64_t)r < n - 1; }

__device__ __forceinline__ Box5 load_box(const float4 *xy, const float *z, int64_t i) {
    float4 a = __ldcg(&xy[i]);
    Box5 b = {a.x, a.y, a.z, a.w, __ldcg(&z[i])};
    return b;
}

__global__ void refit_kernel(const int32_t *__restrict__ sorted_tri, int64_t n, const float4 *__restrict__ tbox_xy,
                             const float *__restrict__ tbox_z, const int2 *__restrict__ child,
                             const int32_t *__restrict__ parent_int, const int32_t *__restrict__ parent_leaf,
                             float4 *leaf_xy, float *leaf_z, float4 *int_xy, float *int_z, unsigned *flags) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int t = sorted_tri[k];
    float4 bx = tbox_xy[t];
    float bz = tbox_z[t];
    __stcg(&leaf_xy[k], bx);
    __stcg(&leaf_z[k], bz);
    __threadfence();
    int node = parent_leaf[k];
    for (int64_t guard = 0; node >= 0 && node < n - 1 && guard < n; guard++) {
        unsigned old = atomicAdd(&flags[node], 1u);
        if (old == 0) return;          // first arrival: the sibling finishes
        __threadfence();
        int2 c = child[node];
        if (!ref_ok(c.x, n) || !ref_ok(c.y, n)) return;
        Box5 a = c.x < 0 ? load_box(leaf_xy, leaf_z, ~c.x) : load_box(int_xy, int_z, c.x);
        Box5 b = c.y < 0 ? load_box(leaf_xy, leaf_z, ~c.y) : load_box(int_xy, int_z, c.y);
        float4 u = make_float4(fminf(a.x0, b.x0), fmaxf(a.x1, b.x1), fminf(a.y0, b.y0), fmaxf(a.y1, b.y1));
        __stcg(&int_xy[node], u);
        __stcg(&int_z[node], fmaxf(a.z1, b.z1));
        __threadfence();
        node = parent_int[node];
    }
}

__global__ void pack_kernel(const int2 *__restrict__ child, int64_t n, const float4 *__restrict__ leaf_xy,
                            const float *__restrict__ leaf_z, const float4 *__restrict__ int_xy,
                            const float *__restrict__ int_z, BvhNode *__restrict__ nodes) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int2 c = child[i];
    if (!ref_ok(c.x, n) || !ref_ok(c.y, n)) {   // never dereference a corrupt reference
        BvhNode bad;
        bad.lo = bad.hi = make_float4(1.f, -1.f, 1.f, -1.f);
        bad.z = make_float4(-3.4e38f, -3.4e38f, __int_as_float(~0), __int_as_float(~0));
        nodes[i] = bad;
        return;
    }
    float4 a = c.x < 0 ? leaf_xy[~c.x] : int_xy[c.x];
    float4 b = c.y < 0 ? leaf_xy[~c.y] : int_xy[c.y];
    float za = c.x < 0 ? leaf_z[~c.x] : int_z[c.x];
    float zb = c.y < 0 ? leaf_z[~c.y] : int_z[c.y];
    BvhNode nd;
    nd.lo = a;
    nd.hi = b;
    nd.z = make_float4(za, zb, __int_as_float(c.x), __int_as_float(c.y));
    nodes[i] = nd;
}

__global__ void tris_kernel(const float *__restrict__ V, const int32_t *__restrict__ F,
                            const int32_t *__restrict__ sorted_tri, int64_t n, float4 *__restrict__ tris,
                            const float4 *__restrict__ tbox_xy, const float *__restrict__ tbox_z,
                            float4 *__restrict__ tbox) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int t = sorted_tri[k];
    tbox[2 * k] = tbox_xy[t];
    tbox[2 * k + 1] = make_float4(tbox_z[t], 0.f, 0.f, 0.f);
    for (int c = 0; c < 3; c++) {
        int vi = F[3 * (int64_t)t + c];
        tris[3 * k + c] = make_float4(V[3 * (int64_t)vi], V[3 * (int64_t)vi + 1], V[3 * (int64_t)vi + 2], 0.f);
    }
}

__global__ void radius_kernel(const float *__restrict__ V, int64_t nv, unsigned *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float r = 0.f;
    if (i < nv) {
        float x = V[3 * i], y = V[3 * i + 1], z = V[3 * i + 2];
        r = sqrtf(x * x + y * y + z * z) * 1.000001f;
    }
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(r));
}

// ---- mesh intake: checks and boundary unit edges ---------------------------
// One thread per entry of max(3 nv, 3 nf): a vertex coordinate is checked for
// being finite (flag bit 0), a face corner for indexing a vertex (bit 1), and
// face corner i = 3t + k emits the directed edge (F[i], F[3t + (k+1) mod 3])
// as the key (min << 32 | max) with value +1 if it runs from min to max, -1
// if it runs from max to min, 0 if it is degenerate.
__global__ void mesh_intake_kernel(const float *__restrict__ V, int64_t nv3, const int32_t *__restrict__ F,
                                   int64_t nf3, int64_t nv, unsigned long long *__restrict__ keys,
                                   int32_t *__restrict__ vals, unsigned *flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nv3 && !isfinite(V[i])) atomicOr(flags, 1u);
    if (i < nf3) {
        int64_t t = i / 3;
        int k = (int)(i - 3 * t);
        int32_t a = F[i], b = F[3 * t + (k == 2 ? 0 : k + 1)];
        if (a < 0 || (int64_t)a >= nv) atomicOr(flags, 2u);
        unsigned ua = (unsigned)a, ub = (unsigned)b;
        unsigned lo = ua < ub ? ua : ub, hi = ua < ub ? ub : ua;
        keys[i] = ((unsigned long long)lo << 32) | hi;
        vals[i] = a == b ? 0 : (ua < ub ? 1 : -1);
    }
}

// After the sort equal keys are adjacent: the first entry of each run adds
// the run's values, the net multiplicity m of that undirected edge, and
// emits |m| unit edges in the direction of m's sign.  The total is at most
// the number of entries; the order of the output is not fixed (atomics), the
// host sorts it.
__global__ void edge_net_kernel(const unsigned long long *__restrict__ keys, const int32_t *__restrict__ vals,
                                int64_t n, int2 *__restrict__ out, unsigned long long *count) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long k = keys[i];
    if (i > 0 && keys[i - 1] == k) return;
    long long m = 0;
    for (int64_t j = i; j < n && keys[j] == k; j++) m += vals[j];
    if (m == 0) return;
    int32_t lo = (int32_t)(k >> 32), hi = (int32_t)(k & 0xffffffffull);
    unsigned long long c = (unsigned long long)(m > 0 ? m : -m);
    unsigned long long pos = atomicAdd(count, c);
    for (unsigned long long r = 0; r < c && pos + r < (unsigned long long)n; r++)
        out[pos + r] = m > 0 ? make_int2(lo, hi) : make_int2(hi, lo);
}

// Boundary records from the chained loops: code[i] is the vertex id, or its
// complement at the first record of a loop (w = 0 there, 1 elsewhere).
__global__ void bseq_kernel(const float *__restrict__ V, const int32_t *__restrict__ code, int64_t n,
                            float4 *__restrict__ bseq, int32_t *__restrict__ bseq_vid) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = code[i];
    int32_t v = c < 0 ? ~c : c;
    bseq[i] = make_float4(V[3 * (int64_t)v], V[3 * (int64_t)v + 1], V[3 * (int64_t)v + 2], c < 0 ? 0.f : 1.f);
    bseq_vid[i] = v;
}

// zeroes the refit arrival counters and seeds the bound reductions
__global__ void build_init_kernel(unsigned *bounds, unsigned *rad, unsigned *flags, int64_t nflags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 12) bounds[i] = (i < 3 || i == 6 || i == 8) ? 0xffffffffu : 0u;
    if (i == 0) *rad = 0u;
    if (i < nflags) flags[i] = 0u;
}

// ---- 2D bins over the projection plane --------------------------------------
// All rays share d, so a ray is a point of the (e1, e2) plane and the
// crossing search is a 2D point location plus a depth test.  The bounding
// rectangle of the padded triangle boxes is cut into nbx x nby bins (about
// BIN_TRIS triangles per bin); bin (i, j) lists every triangle whose padded box
// overlaps it, by decreasing zmax.  bin_of (query.cuh) is monotone in its
// argument, which makes the lookup exact (see chi_bins_kernel).
constexpr int BIN_TRIS = 2;

// number of (bin, triangle) entries: the bins of each padded box, summed
__global__ void bin_count_kernel(const float4 *__restrict__ tbox, int64_t n, BinParams bp,
                                 unsigned long long *total) {
    __shared__ unsigned long long s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        float4 b = tbox[2 * t];
        unsigned long long c = (unsigned long long)(bin_of(b.y, bp.x0, bp.invx, bp.nbx) -
                                                    bin_of(b.x, bp.x0, bp.invx, bp.nbx) + 1) *
                               (unsigned long long)(bin_of(b.w, bp.y0, bp.invy, bp.nby) -
                                                    bin_of(b.z, bp.y0, bp.invy, bp.nby) + 1);
        atomicAdd(&s, c);
    }
    __syncthreads();
    if (threadIdx.x == 0 && s) atomicAdd(total, s);
}

// one (key, triangle) per entry: key = bin << 32 | ~order(zmax), so the sort
// puts each bin's triangles by decreasing zmax; triangles in sorted order.
// Space is taken with one atomic per warp (the warp's entries counted by a
// shuffle scan), not one per triangle on the single counter.  Launched with
// whole warps; the order of the entries is fixed only by the sort.
__global__ void bin_emit_kernel(const float4 *__restrict__ tbox, int64_t n, BinParams bp, int64_t cap,
                                unsigned long long *__restrict__ keys, int32_t *__restrict__ vals,
                                unsigned long long *counter) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = t < n;
    int bx0 = 0, bx1 = -1, by0 = 0, by1 = -1;
    unsigned zk = 0;
    if (live) {
        const float4 b = tbox[2 * t];
        zk = ~f2ord(tbox[2 * t + 1].x);
        bx0 = bin_of(b.x, bp.x0, bp.invx, bp.nbx); bx1 = bin_of(b.y, bp.x0, bp.invx, bp.nbx);
        by0 = bin_of(b.z, bp.y0, bp.invy, bp.nby); by1 = bin_of(b.w, bp.y0, bp.invy, bp.nby);
    }
    const unsigned long long c = live ? (unsigned long long)(bx1 - bx0 + 1) * (unsigned long long)(by1 - by0 + 1)
                                      : 0ull;
    unsigned long long x = c;                     // inclusive over the warp's lanes
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULL, x, off);
        if (lane >= off) x += y;
    }
    unsigned long long base = 0;
    if (lane == 31 && x) base = atomicAdd(counter, x);
    base = __shfl_sync(FULL, base, 31);
    if (!live) return;
    unsigned long long pos = base + (x - c);
    for (int by = by0; by <= by1; by++)
        for (int bx = bx0; bx <= bx1; bx++, pos++)
            if ((int64_t)pos < cap) {
                keys[pos] = ((unsigned long long)((int64_t)by * bp.nbx + bx) << 32) | zk;
                vals[pos] = (int32_t)t;
            }
}

// sorted entries -> (zmax, triangle) and the padded box of each entry
__global__ void bin_pack_kernel(const int32_t *__restrict__ vals, int64_t m, const float4 *__restrict__ tbox,
                                float2 *__restrict__ zt, float4 *__restrict__ box) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int t = vals[i];
    box[i] = tbox[2 * (int64_t)t];
    zt[i] = make_float2(tbox[2 * (int64_t)t + 1].x, __int_as_float(t));
}

// start[b] = first entry of bin b (b = nbins: the entry count), by binary
// search over the sorted keys; the longest list goes to *maxlen
__global__ void bin_start_kernel(const unsigned long long *__restrict__ keys, int64_t m, int64_t nbins,
                                 int32_t *__restrict__ start, unsigned *maxlen) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nbins) return;
    auto lower = [&](unsigned long long k) {
        int64_t lo = 0, hi = m;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (keys[mid] < k) lo = mid + 1; else hi = mid;
        }
        return lo;
    };
    int64_t s = lower((unsigned long long)b << 32);
    start[b] = (int32_t)s;
    if (b < nbins) atomicMax(maxlen, (unsigned)(lower((unsigned long long)(b + 1) << 32) - s));
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Carves one scratch block into 256-byte aligned arrays; a pass with a null
// base only adds up the size.
struct Carve {
    char *base = nullptr;
    size_t off = 0;
    template <typename T>
    T *take(int64_t count) {
        off = (off + 255) & ~(size_t)255;
        T *r = base ? (T *)(base + off) : nullptr;
        off += sizeof(T) * (size_t)(count > 0 ? count : 1);
        return r;
    }
};

// Stable LSD radix sort of n (key, value) pairs by the key bytes set in
// byte_mask (bit b: byte b), one 8-bit digit per pass; three launches per
// pass (digit histogram per tile, scan + skip test, scatter).  The pairs move
// between (k0, v0) and (k1, v1); on return (k0, v0) names the sorted copy.
cudaError_t radix_sort_pairs(unsigned long long *&k0, int32_t *&v0, unsigned long long *&k1, int32_t *&v1,
                             int64_t n, unsigned *hist, int *skip, unsigned byte_mask, cudaStream_t st) {
    if (n <= 1) return cudaSuccess;
    const int nblocks = (int)((n + SORT_TILE - 1) / SORT_TILE);
    for (int b = 0; b < 8; b++) {
        if (!((byte_mask >> b) & 1u)) continue;
        const int shift = 8 * b;
        hist_kernel<<<nblocks, SORT_THREADS, 0, st>>>(k0, n, shift, hist, nblocks);
        scan_skip_kernel<<<1, SCAN_THREADS, 0, st>>>(hist, nblocks, n, skip);
        scatter_kernel<<<nblocks, SORT_THREADS, 0, st>>>(k0, v0, k1, v1, n, shift, hist, nblocks, skip);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        unsigned long long *tk = k0; k0 = k1; k1 = tk;
        int32_t *tv = v0; v0 = v1; v1 = tv;
    }
    return cudaSuccess;
}

inline size_t sort_hist_count(int64_t n) { return (size_t)BINS * (size_t)((n + SORT_TILE - 1) / SORT_TILE); }

}  // namespace

gwn_status mesh_intake_device(gwn_ctx *ctx, const float *dV, int64_t nv, const int32_t *dF, int64_t nf,
                              std::vector<std::pair<int32_t, int32_t>> &bedges) {
    bedges.clear();
    cudaStream_t st = ctx->stream;
    const int64_t nv3 = 3 * nv, nh = 3 * nf, nthr = nv3 > nh ? nv3 : nh;
    if (nthr == 0) return GWN_OK;
    Carve c;
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 1) {
            cudaError_t e;
            c.base = (char *)arena_get(ctx, 6, c.off, &e);
            if (!c.base) return cuda_fail(e, "mesh intake scratch");
            c.off = 0;
        }
        unsigned long long *hdr = c.take<unsigned long long>(2);   // edge count, flags
        unsigned long long *k0 = c.take<unsigned long long>(nh), *k1 = c.take<unsigned long long>(nh);
        int32_t *v0 = c.take<int32_t>(nh), *v1 = c.take<int32_t>(nh);
        unsigned *hist = c.take<unsigned>((int64_t)sort_hist_count(nh));
        int *skip = c.take<int>(1);
        int2 *out = c.take<int2>(nh);
        if (pass == 0) continue;
        cudaError_t e = cudaMemsetAsync(hdr, 0, 2 * sizeof(unsigned long long), st);
        if (e != cudaSuccess) return cuda_fail(e, "mesh intake");
        mesh_intake_kernel<<<blocks_for(nthr, 256), 256, 0, st>>>(dV, nv3, dF, nh, nv, k0, v0, (unsigned *)(hdr + 1));
        // only the bytes of min and max that can be nonzero take a pass
        int bits = 0;
        while (bits < 32 && ((int64_t)1 << bits) < nv) bits++;
        unsigned nb = (unsigned)((bits + 7) / 8), m = (1u << nb) - 1u;
        e = radix_sort_pairs(k0, v0, k1, v1, nh, hist, skip, m | (m << 4), st);
        if (e != cudaSuccess) return cuda_fail(e, "mesh intake sort");
        if (nh > 0) edge_net_kernel<<<blocks_for(nh, 256), 256, 0, st>>>(k0, v0, nh, out, hdr);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "mesh intake");
        // the header and the first edges come back together (boundaries are
        // usually short); a longer boundary takes a second copy
        const int64_t spec = nh < 4096 ? nh : 4096;
        unsigned long long h[2];
        std::vector<int2> he((size_t)(spec > 0 ? spec : 1));
        e = cudaMemcpyAsync(h, hdr, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && spec > 0)
            e = cudaMemcpyAsync(he.data(), out, sizeof(int2) * spec, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "mesh intake");
        if (h[1] & 1u) { set_error("gwn_mesh_create: non-finite vertex coordinate"); return GWN_E_INVALID; }
        if (h[1] & 2u) { set_error("gwn_mesh_create: face index out of range"); return GWN_E_INVALID; }
        int64_t ne = (int64_t)(h[0] < (unsigned long long)nh ? h[0] : (unsigned long long)nh);
        if (ne > spec) {
            he.resize((size_t)ne);
            e = cudaMemcpyAsync(he.data(), out, sizeof(int2) * ne, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "mesh intake");
        }
        bedges.resize((size_t)ne);
        for (int64_t j = 0; j < ne; j++) bedges[j] = std::make_pair(he[j].x, he[j].y);
    }
    return GWN_OK;
}

cudaError_t launch_bseq(const float *dV, const int32_t *code, int64_t n, float4 *bseq, int32_t *bseq_vid,
                        cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    bseq_kernel<<<blocks_for(n, 256), 256, 0, st>>>(dV, code, n, bseq, bseq_vid);
    return cudaGetLastError();
}

static void bins_free(MeshBvh &b) {
    if (b.bin_block) cudaFree(b.bin_block);
    b.bin_block = nullptr;
    b.bin_start = nullptr;
    b.bin_zt = nullptr;
    b.bin_box = nullptr;
    b.n_bin_entries = 0;
    b.bin_maxlen = 0;
    b.bins = BinParams();
}

void bvh_free(MeshBvh &b) {
    if (b.block) cudaFree(b.block);
    b.block = nullptr;
    b.tbox = nullptr;
    b.bframe = nullptr;
    b.nodes = nullptr;
    b.tris = nullptr;
    bins_free(b);
    b.bins_tried = false;
    b.queries_seen = 0;
    b.valid = false;
}

static float ord2f_host(unsigned u) {
    unsigned v = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
    memcpy(&f, &v, sizeof(f));
    return f;
}

cudaError_t bvh_build(gwn_geom *g, const Frame &fr, cudaStream_t st) {
    MeshBvh &b = g->bvh;
    bvh_free(b);
    const int64_t n = g->nf;
    b.n = n;
    b.frame = fr;
    for (int k = 0; k < 3; k++) b.dkey[k] = fr.d[k];
    cudaError_t err = cudaSuccess;
    // the structure's own arrays, in one allocation
    Carve keep;
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 1) {
            if (keep.off == 0) break;
            err = cudaMalloc(&b.block, keep.off);
            if (err != cudaSuccess) { b.block = nullptr; return err; }
            keep.base = (char *)b.block;
            keep.off = 0;
        }
        float4 *bf = g->n_bseq > 0 ? keep.take<float4>(2 * g->n_bseq) : nullptr;
        float4 *tr = n > 0 ? keep.take<float4>(3 * n) : nullptr;
        float4 *tb = n > 0 ? keep.take<float4>(2 * n) : nullptr;
        BvhNode *nd = n > 1 ? keep.take<BvhNode>(n - 1) : nullptr;
        if (pass == 1) { b.bframe = bf; b.tris = tr; b.tbox = tb; b.nodes = nd; }
    }
    if (g->n_bseq > 0) {                 // boundary records in this frame
        err = launch_bframe(g->bseq, g->n_bseq, fr, b.bframe, st);
        if (err != cudaSuccess) { bvh_free(b); return err; }
    }
    if (n == 0) {
        b.valid = true;
        return cudaSuccess;
    }
    // temporaries from the context's build scratch
    const int64_t ni = n > 1 ? n - 1 : 1;
    Carve c;
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 1) {
            c.base = (char *)arena_get(g->ctx, 6, c.off, &err);
            if (!c.base) { bvh_free(b); return err; }
            c.off = 0;
        }
        float4 *tbox_xy = c.take<float4>(n), *cen = c.take<float4>(n);
        float *tbox_z = c.take<float>(n);
        unsigned *bounds = c.take<unsigned>(12), *rad = c.take<unsigned>(1), *hist = c.take<unsigned>(sort_hist_count(n));
        unsigned long long *k0 = c.take<unsigned long long>(n), *k1 = c.take<unsigned long long>(n);
        int32_t *v0 = c.take<int32_t>(n), *v1 = c.take<int32_t>(n);
        int *skip = c.take<int>(1);
        int2 *child = c.take<int2>(ni);
        int32_t *parent_int = c.take<int32_t>(ni), *parent_leaf = c.take<int32_t>(n);
        float4 *leaf_xy = c.take<float4>(n), *int_xy = c.take<float4>(ni);
        float *leaf_z = c.take<float>(n), *int_z = c.take<float>(ni);
        unsigned *flags = c.take<unsigned>(ni);
        if (pass == 0) continue;
        build_init_kernel<<<blocks_for(ni > 12 ? ni : 12, 256), 256, 0, st>>>(bounds, rad, flags, n > 1 ? n - 1 : 0);
        radius_kernel<<<blocks_for(g->nv, 256), 256, 0, st>>>(g->dV, g->nv, rad);
        tri_prep_kernel<<<blocks_for(n, 256), 256, 0, st>>>(g->dV, g->dF, n, fr, tbox_xy, tbox_z, cen, bounds);
        morton_kernel<<<blocks_for(n, 256), 256, 0, st>>>(cen, n, bounds, k0, v0);
        err = cudaGetLastError();
        if (err == cudaSuccess) err = radix_sort_pairs(k0, v0, k1, v1, n, hist, skip, 0xffu, st);
        if (err == cudaSuccess) {
            tris_kernel<<<blocks_for(n, 256), 256, 0, st>>>(g->dV, g->dF, v0, n, b.tris, tbox_xy, tbox_z, b.tbox);
            if (n > 1) {
                karras_kernel<<<blocks_for(n - 1, 256), 256, 0, st>>>(k0, n, child, parent_int, parent_leaf);
                refit_kernel<<<blocks_for(n, 256), 256, 0, st>>>(v0, n, tbox_xy, tbox_z, child, parent_int,
                                                                parent_leaf, leaf_xy, leaf_z, int_xy, int_z, flags);
                pack_kernel<<<blocks_for(n - 1, 256), 256, 0, st>>>(child, n, leaf_xy, leaf_z, int_xy, int_z,
                                                                   b.nodes);
            }
            err = cudaGetLastError();
        }
        unsigned h[12];
        if (err == cudaSuccess) err = cudaMemcpyAsync(h, bounds, sizeof(unsigned) * 10, cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaMemcpyAsync(&h[10], rad, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaStreamSynchronize(st);
        if (err != cudaSuccess) { bvh_free(b); return err; }
        memcpy(&b.scene_radius, &h[10], sizeof(float));
        for (int k = 0; k < 4; k++) b.box_bounds[k] = ord2f_host(h[6 + k]);
    }
    b.root = n == 1 ? ~0 : 0;
    b.valid = true;
    return cudaSuccess;
}

// Bin grid for n triangles over the box bounds (x0, x1, y0, y1): about
// BIN_TRIS triangles per bin, bins near square, at most 2^22 of them.
static BinParams bin_params(const float bb[4], int64_t n) {
    double W = (double)bb[1] - bb[0], H = (double)bb[3] - bb[2];
    double T = (double)(n / BIN_TRIS > 0 ? n / BIN_TRIS : 1);
    if (T > (double)(1 << 22)) T = (double)(1 << 22);
    int nbx = 1, nby = 1;
    if (W > 0 && H > 0) {
        nbx = (int)fmin(fmax(rint(sqrt(T * W / H)), 1.0), 16384.0);
        nby = (int)fmin(fmax(rint(T / nbx), 1.0), 16384.0);
    } else if (W > 0) {
        nbx = (int)fmin(T, 65536.0);
    } else if (H > 0) {
        nby = (int)fmin(T, 65536.0);
    }
    BinParams r;
    r.x0 = bb[0]; r.x1 = bb[1]; r.y0 = bb[2]; r.y1 = bb[3];
    r.invx = W > 0 ? (float)(nbx / W) : 0.f;
    r.invy = H > 0 ? (float)(nby / H) : 0.f;
    if (!(r.invx <= 3.0e38f)) { r.invx = 0.f; nbx = 1; }   // a width too small for float bins
    if (!(r.invy <= 3.0e38f)) { r.invy = 0.f; nby = 1; }
    r.nbx = nbx; r.nby = nby;
    return r;
}

cudaError_t bins_build(gwn_geom *g, cudaStream_t st) {
    MeshBvh &b = g->bvh;
    if (!b.valid || b.bins_tried) return cudaSuccess;
    b.bins_tried = true;
    const int64_t n = b.n;
    if (n < 2 || n >= (int64_t(1) << 26)) return cudaSuccess;
    const BinParams bp = bin_params(b.box_bounds, n);
    const int64_t nbins = (int64_t)bp.nbx * bp.nby;
    cudaError_t err = cudaSuccess;
    // entry count first: it sizes everything else
    unsigned long long *dtotal = (unsigned long long *)arena_get(g->ctx, 7, 2 * sizeof(unsigned long long), &err);
    if (!dtotal) return err;
    err = cudaMemsetAsync(dtotal, 0, 2 * sizeof(unsigned long long), st);
    if (err != cudaSuccess) return err;
    bin_count_kernel<<<blocks_for(n, 256), 256, 0, st>>>(b.tbox, n, bp, dtotal);
    unsigned long long total = 0;
    err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaMemcpyAsync(&total, dtotal, sizeof(total), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return err;
    if (total == 0 || total > (unsigned long long)(12 * n + 4096)) return cudaSuccess;   // not compact: the tree
    const int64_t m = (int64_t)total;
    Carve keep;
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 1) {
            err = cudaMalloc(&b.bin_block, keep.off);
            if (err != cudaSuccess) { b.bin_block = nullptr; return err; }
            keep.base = (char *)b.bin_block;
            keep.off = 0;
        }
        int32_t *bs = keep.take<int32_t>(nbins + 1);
        float2 *bz = keep.take<float2>(m);
        float4 *bb = keep.take<float4>(m);
        if (pass == 1) { b.bin_start = bs; b.bin_zt = bz; b.bin_box = bb; }
    }
    Carve c;
    unsigned long long *bk0 = nullptr, *bk1 = nullptr, *counter = nullptr;
    int32_t *bv0 = nullptr, *bv1 = nullptr;
    unsigned *bhist = nullptr;
    int *bskip = nullptr;
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 1) {
            c.base = (char *)arena_get(g->ctx, 7, c.off, &err);
            if (!c.base) { bins_free(b); return err; }
            c.off = 0;
        }
        counter = c.take<unsigned long long>(2);
        bk0 = c.take<unsigned long long>(m); bk1 = c.take<unsigned long long>(m);
        bv0 = c.take<int32_t>(m); bv1 = c.take<int32_t>(m);
        bhist = c.take<unsigned>(sort_hist_count(m));
        bskip = c.take<int>(1);
    }
    unsigned *maxlen = (unsigned *)(counter + 1);
    err = cudaMemsetAsync(counter, 0, 2 * sizeof(unsigned long long), st);
    if (err != cudaSuccess) { bins_free(b); return err; }
    bin_emit_kernel<<<blocks_for(n, 256), 256, 0, st>>>(b.tbox, n, bp, m, bk0, bv0, counter);
    int bits = 0;
    while (bits < 40 && (int64_t(1) << bits) < nbins) bits++;
    const unsigned nb = (unsigned)((bits + 7) / 8);
    const unsigned mask = 0x0fu | (((1u << nb) - 1u) << 4);   // 4 bytes of depth, then the bin bytes
    err = cudaGetLastError();
    if (err == cudaSuccess) err = radix_sort_pairs(bk0, bv0, bk1, bv1, m, bhist, bskip, mask, st);
    if (err == cudaSuccess) {
        bin_pack_kernel<<<blocks_for(m, 256), 256, 0, st>>>(bv0, m, b.tbox, b.bin_zt, b.bin_box);
        bin_start_kernel<<<blocks_for(nbins + 1, 256), 256, 0, st>>>(bk0, m, nbins, b.bin_start, maxlen);
        err = cudaGetLastError();
    }
    unsigned hmax = 0;
    if (err == cudaSuccess) err = cudaMemcpyAsync(&hmax, maxlen, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) { bins_free(b); return err; }
    // a list far longer than the mean (a dense cluster in a sparse domain)
    // would be scanned by every query in its bin: the tree serves then
    if (hmax > 512 && (double)hmax > 64.0 * (double)m / (double)nbins) {
        bins_free(b);
        return cudaSuccess;
    }
    b.bins = bp;
    b.n_bin_entries = m;
    b.bin_maxlen = (int64_t)hmax;
    return cudaSuccess;
}

}  // namespace gwn
