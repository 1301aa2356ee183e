/*
 * gwn.h -- C ABI of the one-shot generalized winding number library (sm_103a).
 *
 * The library evaluates the generalized winding number w(p) of a triangle
 * mesh or of open cubic Bezier chains at many query points, by the one-shot
 * method: w(p) is the signed number of crossings of ONE ray p + t d (t > 0)
 * with the geometry plus a closed-form term over the boundary only.
 *
 *   3D:  w(p) = chi_d(p) + (1/4pi) sum_{boundary edges A->B} Omega(A-p, B-p, -d)
 *   2D:  w(p) = chi_x(p) + chi_x(chord e->s; p)
 *               + (1/2pi) atan2(cross(s-p, e-p), dot(s-p, e-p))   (per chain)
 *
 * Definitions followed (paper: "One-Shot Method for Computing Generalized
 * Winding Numbers"):
 *   - w for a surface / curve:          Background section (w_M, w_C).
 *   - chi, sign convention (+1 when the ray is aligned with the normal):
 *                                       Background, Eq. chi.
 *   - chi is constant on each region of the sphere cut by the projected
 *     boundary; adjacent regions differ by one, normals point to higher chi:
 *                                       Lemma 1, Lemma 2, Algorithm 1.
 *   - one ray serves all points on it:  One-shot algorithm, "Optimization".
 *   - w undefined on M:                 Background (p in M excluded).
 * The closed form above is Algorithm 1's area-weighted sum with the regions
 * and their areas eliminated: the surface is closed by the half-infinite
 * curtain swept by its boundary in direction -d (the closure used in the proof
 * of Appendix A), which the ray p + t d never meets.
 *
 * Conventions shared by every entry point
 *   - Status: every function returning gwn_status returns GWN_OK (0) or a
 *     negative code; nothing aborts or throws across the ABI.  The message of
 *     the last error on the calling thread is available from gwn_last_error().
 *   - Ownership: inputs are copied into library-owned memory at creation;
 *     output buffers are owned by the caller and must be large enough.
 *   - Memory kinds: GWN_MEM_HOST pointers are ordinary host memory,
 *     GWN_MEM_DEVICE pointers are device memory of the context's device.
 *     Output pointers of gwn_eval / gwn_backward are device pointers.
 *   - Ordering: all device work is enqueued on the context's stream; outputs
 *     are complete when that stream is synchronised.  Functions that take a
 *     gwn_stats* synchronise the stream when the pointer is non-NULL.
 *   - Orientation: triangle (i, j, k) has normal (V[j]-V[i]) x (V[k]-V[i]);
 *     w > 0 behind the surface (the side the normal points away from).
 *   - Precision: 3D inputs are float32; the boundary term runs in float32
 *     with compensated accumulation, crossing counts are exact (filtered
 *     float32 / float64 predicates with exact expansion arithmetic as the last
 *     resort, and a symbolic perturbation of d).  2D chains are float32 or
 *     float64; the float64 path computes in float64.
 *   - Queries ON the geometry have no defined w; they return a finite value.
 */
#ifndef GWN_H
#define GWN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GWN_API __attribute__((visibility("default")))
#else
#define GWN_API
#endif

typedef enum gwn_status {
    GWN_OK = 0,
    GWN_E_INVALID = -1,        /* bad argument (NULL, size, NaN, index out of range) */
    GWN_E_OOM = -2,            /* device or host allocation failed */
    GWN_E_CUDA = -3,           /* a CUDA runtime call failed */
    GWN_E_STACK_OVERFLOW = -4, /* a traversal exceeded its stack (results invalid) */
    GWN_E_TIMEOUT = -5,        /* a bounded device loop hit its iteration limit */
    GWN_E_UNSUPPORTED = -6,    /* valid request this build does not implement */
    GWN_E_INTERNAL = -7        /* internal consistency check failed */
} gwn_status;

enum { GWN_MEM_HOST = 0, GWN_MEM_DEVICE = 1 };
enum { GWN_F32 = 0, GWN_F64 = 1 };
enum { GWN_QUERY_POINTS = 0, GWN_QUERY_GRID = 1 };
enum { GWN_GEOM_MESH = 1, GWN_GEOM_BEZIER2D = 2, GWN_GEOM_PATCHES = 3 };

typedef struct gwn_ctx gwn_ctx;
typedef struct gwn_geom gwn_geom;

/* Query set.
 *   POINTS: pts holds n points of `dim` coordinates, row-major, of type
 *           `dtype` (GWN_F32 for meshes; the chain's dtype for 2D), in
 *           memory `mem_kind`.
 *   GRID:   dims[0] x dims[1] (x dims[2] in 3D) samples; coordinate i of axis
 *           k is lo[k] + i * ((hi[k] - lo[k]) / (dims[k] - 1)) evaluated in
 *           float64 and rounded to the working precision (lo[k] when
 *           dims[k] == 1).  Flat index = i + dims[0] * (j + dims[1] * k).
 */
typedef struct gwn_queries {
    int32_t kind;
    int32_t dtype;
    int32_t mem_kind;
    int32_t dim;
    const void *pts;
    int64_t n;
    double lo[3];
    double hi[3];
    int64_t dims[3];
} gwn_queries;

/* Counters and timings of one evaluation (filled when non-NULL). */
typedef struct gwn_stats {
    int64_t n_queries;
    int64_t n_pairs;            /* query x boundary-edge (3D) or row x piece (2D) pairs */
    int64_t n_cut_sign;         /* boundary-term pairs taken off the float32 path (exact branch or float64) */
    int64_t n_fp64_filter;      /* predicates settled by the float64 filter */
    int64_t n_exact;            /* predicates settled by exact expansion arithmetic */
    int64_t n_stack_overflow;   /* traversals that overflowed (result invalid); patches: queries within the
                                   subdivision limit of the surface (w undefined there) */
    int64_t n_tri_tests;        /* exact ray/triangle tests (3D) or roots (2D) */
    float ms_prepare;           /* per-direction preparation (BVH build, crossing bins) if it ran in this call */
    float ms_traverse;          /* crossing counts */
    float ms_boundary;          /* boundary term + epilogue */
    float ms_total;
    int64_t n_deferred_traverse;  /* (query, triangle) pairs the float32 filter left unsettled, settled with the
                                     full predicates (plus any query recounted whole when the pair list is full) */
    int64_t n_deferred_boundary;  /* queries whose boundary term was recomputed by the careful pass */
    int64_t n_root_iters;         /* 2D: safeguarded Newton steps over all roots (n_tri_tests counts the roots) */
    int64_t n_cert;               /* 2D: crossings (or rows at a rounded extremum value) decided again in float64
                                     because a query lies within their float error bound */
    int64_t n_cert_fixed;         /* 2D: query counts that float64 decision changed */
} gwn_stats;

/* Geometry summary. */
typedef struct gwn_geom_info {
    int32_t kind;               /* GWN_GEOM_MESH, GWN_GEOM_BEZIER2D or GWN_GEOM_PATCHES */
    int32_t dtype;
    int64_t n_vertices;         /* mesh vertices / 2D control points */
    int64_t n_primitives;       /* triangles / cubic segments */
    int64_t n_boundary_edges;   /* 3D: unit-multiplicity boundary edges; 2D: chains */
    int64_t n_loops;            /* 3D: boundary loops; 2D: chains */
    int64_t n_pieces;           /* 2D: y-monotone pieces; 3D: 0 */
    int64_t n_chains;           /* 2D: chains; 3D: 0 */
    int64_t n_bins;             /* mesh, after preparation: bins of the 2D crossing index (0: tree only) */
    int64_t n_bin_entries;      /* (bin, triangle) entries */
    int64_t bin_maxlen;         /* longest bin list */
} gwn_geom_info;

/* Library version string (static storage). */
GWN_API const char *gwn_version(void);

/* Message of the last failed call on this thread (thread-local storage owned
 * by the library; valid until the next failing call on the same thread). */
GWN_API const char *gwn_last_error(void);

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (NULL: the legacy default stream).  The stream is borrowed, not owned. */
GWN_API gwn_status gwn_ctx_create(gwn_ctx **out, int device, void *cuda_stream);
GWN_API gwn_status gwn_ctx_set_stream(gwn_ctx *ctx, void *cuda_stream);
/* Synchronise the context's stream and report any device-side error flag
 * raised by earlier evaluations since the last check (then clear it). */
GWN_API gwn_status gwn_ctx_check(gwn_ctx *ctx);
/* Geometries created on ctx keep it alive: its resources are released when
 * both this call has been made and its last geometry has been destroyed, in
 * either order. */
GWN_API void gwn_ctx_destroy(gwn_ctx *ctx);

/* Triangle mesh: V float32 [nv x 3], F int32 [nf x 3] in `mem_kind` memory.
 * Defining passages: the boundary of the surface is what the method sums
 * over -- segments that belong to only one loop are boundary, interior
 * segments are traversed once in each direction and cancel (Curve Networks,
 * Preprocessing); several disconnected boundaries enter one and the same sum
 * (Implementation Details, "Multiple Boundaries").
 * Copies the inputs to the device and extracts the boundary there: V is
 * checked finite and F in range, every directed edge becomes a key (smaller
 * id, larger id), a device radix sort groups the keys and each run's net
 * multiplicity m = #(A->B) - #(B->A) is taken; an edge with |m| > 1 is split
 * into |m| unit edges.  Only the unit boundary edges are copied back to the
 * host, which chains them into loops (walk of unused out-edges); the loop
 * records are gathered on the device.  The call synchronises the context's
 * stream.  Fails with GWN_E_INVALID on a non-finite coordinate or an index
 * outside [0, nv).  The ray-crossing hierarchy is built per direction d on
 * first use (or by gwn_mesh_prepare). */
GWN_API gwn_status gwn_mesh_create(gwn_ctx *ctx, const float *V, int64_t nv, const int32_t *F,
                                   int64_t nf, int mem_kind, gwn_geom **out);

/* Crossing index of a mesh.  All rays share d, so the crossing search is a
 * 2D point location in the plane normal to d plus a depth test.
 *   AUTO (the default): once the evaluations of a (mesh, d) have asked for
 *     at least 4 queries per triangle in total (grid queries with d parallel
 *     to a grid axis, which reuse rays per grid line, do not count), the
 *     evaluation reaching that total builds once, besides the LBVH, a bin
 *     grid over the projected triangle boxes (lists by decreasing depth) and
 *     uses it when it is compact: at most 12 entries per triangle + 4096, and
 *     no list longer than both 512 and 64 times the mean.  Without device
 *     memory for the bins the tree serves.
 *   TREE: always the LBVH traversal.
 * Both test exactly the same (query, triangle) pairs, so the crossing counts
 * are identical.  Takes effect at the next evaluation. */
enum { GWN_INDEX_AUTO = 0, GWN_INDEX_TREE = 1 };
GWN_API gwn_status gwn_mesh_set_index(gwn_geom *g, int index);

/* Build (or reuse) the on-device LBVH of the mesh in the frame of direction
 * d (float32[3], any nonzero length).  Optional: gwn_eval prepares lazily. */
GWN_API gwn_status gwn_mesh_prepare(gwn_geom *g, const float d[3]);

/* Cubic Bezier chains.  Defining passage: the winding number of a 2D curve,
 * w_C(p) = (1/2pi) * (angle swept by the curve around p), and its crossing
 * count form with one ray (Background, 2D winding number; Validation and
 * Results, 2D parametric geometry: cubic Bezier curves on regular grids).
 * ctrl [n_ctrl x 2] of type dtype (GWN_F32|GWN_F64);
 * chain c owns control points chain_offsets[c] .. chain_offsets[c+1]-1, a
 * C0 chain of (count-1)/3 cubic segments (count = 3k+1, k >= 1).
 * chain_offsets is a host array of n_chains + 1 int64.  Each chain is split
 * on the host into y-monotone pieces. */
GWN_API gwn_status gwn_bezier2d_create(gwn_ctx *ctx, const void *ctrl, int dtype,
                                       const int64_t *chain_offsets, int64_t n_chains,
                                       int mem_kind, gwn_geom **out);

/* Surfaces of bicubic Bezier patches (parametric surfaces, "Parametric
 * Surfaces" in the paper's implementation section): ctrl [n_patches][4][4][3]
 * float32, control point P_ij of a patch at [i][j] (i along u, j along v),
 * normal f_u x f_v.  The crossing count is taken on the patches themselves
 * (no surface discretisation); the boundary term on the boundary curves (the
 * patch edge curves that no other patch cancels: a curve and its reverse,
 * bit for bit, cancel) sampled at `segments` intervals each (1 .. 65536),
 * which perturbs w by O(segments^-2) near the boundary.  Copies the input.
 * gwn_eval takes float32 points or a 3D grid and a direction d.  Fails with
 * GWN_E_INVALID on a non-finite control point. */
GWN_API gwn_status gwn_patches_create(gwn_ctx *ctx, const float *ctrl, int64_t n_patches, int segments,
                                      int mem_kind, gwn_geom **out);

GWN_API gwn_status gwn_geom_info_get(const gwn_geom *g, gwn_geom_info *out);
GWN_API void gwn_geom_destroy(gwn_geom *g);

/* Boundary loops of a mesh as extracted (host copies).  loop_offsets gets
 * n_loops + 1 entries; vert_ids gets n_boundary_edges vertex indices (loop j
 * is vert_ids[loop_offsets[j] .. loop_offsets[j+1]-1], closing back to its
 * first vertex).  Either pointer may be NULL. */
GWN_API gwn_status gwn_mesh_boundary(const gwn_geom *g, int64_t *loop_offsets, int32_t *vert_ids);

/* Host-only boundary extraction (no device needed), same result as the one
 * gwn_mesh_create performs.  Capacities: loop_offsets >= 3*nf+1 entries,
 * vert_ids >= 3*nf entries (upper bounds).  Returns counts through n_loops
 * and n_edges. */
GWN_API gwn_status gwn_boundary_extract_host(const int32_t *F, int64_t nf, int64_t nv,
                                             int64_t *loop_offsets, int32_t *vert_ids,
                                             int64_t *n_loops, int64_t *n_edges);

/* Host-only y-monotone split of one cubic segment (4 control points x, y in
 * float64): writes up to 3 parameter intervals [u0, u1] (6 doubles) and
 * returns their count through n_out.  Interval ends are 0, 1 and the roots of
 * dy/du in (0, 1). */
GWN_API gwn_status gwn_bezier_monotone_split_host(const double ctrl[8], double u_out[6],
                                                  int32_t *n_out);

/* Evaluate w at the queries.
 *   q:      mesh: a 3D grid or float32 points.  2D: a grid (one +x ray per
 *           grid row, Optimization of Alg. 1) or points in the chain's dtype
 *           (one +x ray per point, through a y-bucket index of the pieces).
 *           Mesh grids with d parallel to a grid axis traverse once per grid
 *           line.
 *   d:      ray direction.  Mesh: float32[3], nonzero (need not be unit).
 *           2D: must be NULL or (1, 0) (the +x ray).
 *   w_out:  device buffer of n_queries values: float32 for meshes and float32
 *           chains, float64 for float64 chains.
 *   chi_out (optional, device int32[n]): the signed crossing count.
 *   b_out   (optional, device, same dtype as w_out): the boundary term
 *           (3D: B_d; 2D: chord term).
 *   stats   (optional): counters; synchronises the stream.
 * A mesh evaluation for a new d first builds the LBVH (gwn_mesh_prepare), and
 * one evaluation per (mesh, d) may build the crossing bins
 * (gwn_mesh_set_index); those one-time builds synchronise the stream, so an
 * evaluation that must only enqueue work (e.g. under stream capture) needs a
 * prepared mesh and GWN_INDEX_TREE or bins already built. */
GWN_API gwn_status gwn_eval(gwn_geom *g, const gwn_queries *q, const float *d, void *w_out,
                            int32_t *chi_out, void *b_out, gwn_stats *stats);

/* Inside test (voxelization: the paper's voxel figure in Sec. Curve Networks
 * marks winding number 1 occupied and 0 empty; the threshold taken is the
 * midpoint): inside_out[i] = 1 if the float32 w(q_i) of gwn_eval is
 * >= 0.5, else 0; uint8, device memory, one byte per query, written by the
 * boundary-term kernels in place of w (no float w array is stored).  Meshes
 * and patch surfaces; GWN_E_UNSUPPORTED for 2D chains.  Asynchronous like
 * gwn_eval. */
GWN_API gwn_status gwn_eval_inside(gwn_geom *g, const gwn_queries *q, const float *d, uint8_t *inside_out);

/* Same, reading queries from HOST memory and writing w to HOST memory:
 * copies in, evaluates, copies back, synchronises.  (End-to-end entry point.)
 * For meshes and patches, a page-locked w_host (cudaHostAlloc /
 * cudaHostRegister) is written directly by the kernels instead of through a
 * device buffer and a copy; the result is the same.  w_host is complete when
 * the call returns. */
GWN_API gwn_status gwn_eval_host(gwn_geom *g, const gwn_queries *q, const float *d, void *w_host);

/* Tuning plan for batched evaluation. */
typedef struct gwn_plan {
    int32_t threads_per_block;  /* 2D: 32..256, a multiple of 32; 0 = autotuned (128 or 256) */
    int32_t rows_per_item;      /* 2D work item height in grid rows, 1..256, with rows x (widest grid's
                                   columns rounded up to 256) x 4 bytes at most 227 KB (the item's
                                   difference cells in shared memory); 0 = autotuned (4..64) */
    int32_t pieces_per_item;    /* reserved, 0 */
    int32_t use_graph;          /* 1 = capture the launch sequence in a CUDA graph */
} gwn_plan;

/* Evaluate many 2D chain sets (one geometry, chain c with its own grid
 * queries[c]) in one persistent launch.  Defining passage: the 2D experiment
 * of Validation and Results evaluates a thousand random curves, each on its
 * own regular grid in the curve's bounding box; here they are one launch
 * whose work items (chain, block of grid rows, run of pieces) are claimed
 * from an atomic counter.  w_out is one device buffer holding
 * chain c's grid at offset out_offsets[c] (host int64[n_chains]).  plan may be
 * NULL (autotuned and cached per shape).  The launch sequence is captured
 * once in a CUDA graph and replayed on later calls with the same shapes. */
GWN_API gwn_status gwn_eval_batch(gwn_geom *g, const gwn_queries *queries, int64_t n_chains,
                                  const int64_t *out_offsets, void *w_out, const gwn_plan *plan,
                                  gwn_stats *stats);

/* Work-item shape chosen for the most recent batched plan of g
 * (threads per block, grid rows per work item). */
GWN_API gwn_status gwn_batch_plan_get(gwn_geom *g, int32_t *threads, int32_t *rows);

/* Evaluate many meshes, each at its own queries, in one persistent launch.
 * Defining passage: the winding number of each mesh as gwn_eval computes it;
 * batching many inputs of uneven sizes follows the 2D experiment of
 * Validation and Results (many random inputs, each on its own grid), here for
 * meshes.  Work items are (mesh, run of 1024-query tiles), ordered by
 * boundary size and claimed from an atomic counter; a block counts the
 * crossings of its tile and runs the boundary term's main pass; list-driven
 * kernels then settle deferred work and form w.  Each query gets the same
 * bits as from gwn_eval on its mesh with the same d.
 *   meshes: n mesh geometries of ctx, each already prepared for d
 *           (gwn_mesh_prepare; GWN_E_INVALID otherwise); a mesh whose
 *           crossing bins exist (and whose index is AUTO) uses them, else its
 *           LBVH.
 *   qs:     n query sets: 3D grids, or float32 points in device memory.
 *   d:      float32[3], the direction every mesh was prepared for.
 *   w_outs: n device float32 buffers, w_outs[i] holding qs[i]'s count.
 *   plan:   NULL (tile run length and blocks per SM autotuned, graph on), or
 *           rows_per_item = tiles per work item, threads_per_block = blocks
 *           per SM (1 or 2), use_graph.
 *   stats:  optional: n_queries, ms_total, deferred counts (synchronises).
 * The first call with a given (meshes, queries, outputs, d) uploads a plan,
 * times the candidate shapes and captures the launch sequence in a CUDA
 * graph (it synchronises the stream and must not run under stream capture);
 * later calls with the same arguments replay the graph and only enqueue
 * work.  Up to 2^31 - 1 queries per batch. */
GWN_API gwn_status gwn_eval_meshes(gwn_ctx *ctx, gwn_geom *const *meshes, const gwn_queries *qs, int64_t n,
                                   const float d[3], float *const *w_outs, const gwn_plan *plan, gwn_stats *stats);

/* Shape chosen for the most recent gwn_eval_meshes plan on ctx (tiles per
 * work item, blocks per SM). */
GWN_API gwn_status gwn_meshes_plan_get(gwn_ctx *ctx, int32_t *tiles_per_item, int32_t *blocks_per_sm);

/* Gradient of w (mesh, POINTS queries) w.r.t. the query points and the mesh
 * vertices, given the upstream gradient grad_w (device float32[n]).
 * Defining passage: Conclusions (moving geometry: w recomputed as the
 * geometry moves); the derivative is that of the closed form above, whose
 * crossing count is piecewise constant, so only the boundary term varies:
 * d/dp of (1/4pi) sum Omega(A-p, B-p, -d) is the Biot-Savart line integral
 * over the boundary, independent of d.
 *   grad_p (device float32[n x 3] or NULL):  grad_w[q] * dw_q/dp
 *   grad_V (device float32[nv x 3] or NULL): sum_q grad_w[q] * dw_q/dV
 *            (rows of vertices not on the boundary are 0).
 * Only the boundary term depends on the geometry continuously (chi is
 * piecewise constant), so both come from the boundary edges alone.
 * Workspace, from the context's grow-only scratch (kept for later calls):
 * with both outputs, 12 * ceil(E / 256) bytes per query (E boundary edges:
 * its sums over each block of 256 edges) plus 32 bytes per boundary record
 * per query chunk (at most a few thousand chunks); with one output, at most
 * the second part.  A request that does not fit returns GWN_E_OOM without
 * computing anything (grad_V may already have been cleared): split the
 * queries over several calls (grad_V is then the sum of the calls' results). */
GWN_API gwn_status gwn_backward(gwn_geom *g, const gwn_queries *q, const float *d,
                                const float *grad_w, float *grad_p, float *grad_V);

/* Mesh evaluation that allocates no device memory (no counterpart in the
 * paper: a deployment variant of gwn_eval for device-resident points).
 *
 * For callers that reserve all device memory up front and cannot call
 * cudaMalloc afterwards -- it can stall the whole device and can fail under
 * memory pressure in the middle of a request.  gwn_eval keeps the per-query
 * crossing counts (scratch between the traversal and the boundary-term
 * kernel) and the boundary term's deferred-query list in buffers it
 * allocates on demand; this entry point keeps both in a fixed array inside
 * the library instead (the list length in a counter the context allocated at
 * creation) and calls no cudaMalloc, cudaFree or allocating library
 * routine.
 *   pts:   device float32 [n x 3] query points; n <= GWN_NOALLOC_MAX_QUERIES
 *          (larger n returns GWN_E_INVALID without doing any work).
 *   d:     the direction the mesh was prepared for with gwn_mesh_prepare
 *          (preparation allocates, so it must happen earlier); otherwise
 *          GWN_E_INVALID.
 *   w_out: device float32 [n]; same values as gwn_eval on the same input.
 * The array takes 32 MiB on every GPU that loads the library, until the
 * process exits.  Every call whose stream is not capturing looks up the
 * array's device address (cudaGetSymbolAddress with the device current; it
 * allocates nothing), so a device reset between calls is picked up; the
 * first call on a device must come before any stream capture, and a call on
 * a capturing stream reuses the last address looked up on that device.  All
 * calls share the one array and it keeps
 * the last call's contents: calls whose work overlaps on the GPU (other
 * streams or contexts on the same device) race on it -- serialise them. */
#define GWN_NOALLOC_MAX_QUERIES 4194304
GWN_API gwn_status gwn_eval_points_noalloc(gwn_geom *g, const float *pts, int64_t n, const float d[3],
                                           float *w_out);

/* Brute-force comparator on the same device: 3D, the sum of per-triangle
 * solid angles over every triangle (float32); 2D, per-segment angle integral
 * by fixed-order Gauss-Legendre on an adaptive subdivision.  w_out as for
 * gwn_eval. */
GWN_API gwn_status gwn_eval_bruteforce(gwn_geom *g, const gwn_queries *q, void *w_out);

#ifdef __cplusplus
}
#endif
#endif /* GWN_H */
