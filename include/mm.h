/*
 * mm.h -- C-ABI of the GB300 MulMent library (libmm.so).
 *
 * MulMent: multilevel maxent-stress graph layout (Meyerhenke, Noellenburg,
 * Schulz, arXiv 1506.04383).  The library computes a 2-D layout x of an
 * undirected connected graph by iterating the local update of Eq. 2 on every
 * level of a coarsening hierarchy (Sec. 3), with the long-range entropy term
 * approximated by a Barnes-Hut quadtree rebuilt on the GPU every iteration.
 *
 * Conventions for every call:
 *   - Positions are float32 pairs, x[2*v] = x-coordinate, x[2*v+1] = y.
 *   - Graphs are symmetric CSR: row_ptr[n+1] (int64), col[nnz] (int32), rows
 *     sorted strictly ascending, no self-loops, every edge stored in both
 *     directions.  The paper's input model (Sec. 2.1) is an undirected,
 *     connected graph with unit node weights, unit edge weights and target
 *     edge lengths d (default 1).
 *   - "device" pointers are CUDA device memory of the current device; "host"
 *     pointers are ordinary CPU memory.  The caller owns every buffer it
 *     passes; inputs are only read during the call (the hierarchy copies what
 *     it keeps); the library owns mm_hierarchy objects.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All device work is ordered on it.  Calls that write host
 *     outputs synchronise the stream before returning.
 *   - Every call returns an mm_status; no exception or exit crosses the ABI.
 *     mm_last_error() gives a message for the last failure on this thread.
 *   - There is no CPU fallback: without a usable GPU the calls return
 *     MM_ERR_CUDA.
 */
#ifndef MM_H
#define MM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mm_status;
#define MM_OK 0
#define MM_ERR_INVALID_ARG 1   /* malformed graph, bad level, bad sizes      */
#define MM_ERR_NOT_CONNECTED 2 /* the input graph is not connected (Sec. 2.1)*/
#define MM_ERR_CUDA 3          /* a CUDA runtime call failed                 */
#define MM_ERR_OOM 4           /* device allocation failed                   */
#define MM_ERR_NONFINITE 5     /* a sweep produced NaN or Inf coordinates    */
#define MM_ERR_TIMEOUT 6       /* a bounded device wait gave up              */
#define MM_ERR_UNSUPPORTED 7   /* valid request outside the implemented range*/

#define MM_PARAMS_VERSION 1u
#define MM_MAX_LEVELS 64

/*
 * Algorithm parameters.  Defaults (mm_default_params) are the paper's
 * configuration (Sec. 4, "Algorithm Configuration"): f = 20, b = 2,
 * alpha0 = 1, alpha := 0.3 alpha down to alpha_min = 0.008, at most a = 2
 * iterations per alpha, at alpha_min iterate until the relative change is
 * below 1e-4.  k, theta and coarsest_n select the general model and the
 * Barnes-Hut approximation.
 */
typedef struct mm_params {
  uint32_t struct_version;  /* must be MM_PARAMS_VERSION                      */
  int32_t k;                /* S = pairs within k hops (1 or 2); k=1 is S=E   */
  float theta;              /* Barnes-Hut opening parameter; 0 = exact via tree*/
  int32_t exact_repulsion;  /* 1: exact O(n^2) entropy sum on every level     */
  int32_t coarsest_n;       /* coarsen while n > coarsest_n (>= 2)            */
  float f, b;               /* SCLaP W = min(b^(h+1), |V|/f) (Sec. 3.1)       */
  int32_t lp_rounds;        /* SCLaP rounds l                                 */
  int32_t iters_per_alpha;  /* a: iterations per alpha round                  */
  double alpha0, alpha_factor, alpha_min;
  double eps;               /* early alpha reduction threshold                */
  double eps_final;         /* convergence threshold at alpha_min             */
  int32_t max_iters_at_min; /* cap on iterations at alpha_min                 */
  int32_t early_exit;       /* 0: run exactly a / max_iters_at_min iterations */
  uint64_t seed;            /* Philox key for prolongation and clustering     */
  int32_t max_levels;       /* hierarchy depth cap (<= MM_MAX_LEVELS)         */
  int32_t max_stalls;       /* retries of a contraction that merged nothing   */
  int32_t gather_lanes;     /* lanes per vertex in the S gather; 0 = auto     */
  int32_t heavy_degree;     /* rows above this use a block each; 0 = auto     */
  int32_t traverse_warps;   /* warps per block in the tree walk; 0 = auto     */
  int32_t fused_max_n;      /* levels with n <= this run in one single-CTA    */
                            /* kernel; 0 = auto (2048, the maximum), -1 = off */
  int32_t learned_prolong;  /* 1: prolongate with the network attached by     */
                            /* mm_hierarchy_set_net (single-graph layouts)    */
  int32_t leaf_size;        /* Barnes-Hut: a cell with at most this many      */
                            /* points is a leaf; an opened leaf is summed     */
                            /* exactly (1 = single-point leaves; 0 = 1)       */
  int32_t bh_group;         /* Barnes-Hut acceptance: 0 = per point (the      */
                            /* classic test), 1 = per group of 32 Morton-     */
                            /* consecutive points (a cell far from all of     */
                            /* them; refines each point's per-point sum)      */
  int32_t approx_levels;    /* h of MulMent_h: 0 = Barnes-Hut / exact as set  */
                            /* above; h > 0 = the entropy sum of Eq. 3 with   */
                            /* the level h levels down (or the coarsest) on   */
                            /* every level but the coarsest (Sec. 3.2); those */
                            /* levels run the sweep kernels (no fused level   */
                            /* kernel); single graphs only (batches: error)   */
  int32_t level_order;      /* 1: mm_build_hierarchy renumbers every level so */
                            /* that clusters are consecutive, in the order of */
                            /* the coarser level (memory locality of the      */
                            /* sweeps; level-0 positions still cross the ABI  */
                            /* in the caller's numbering); 0: input numbering */
  int32_t exact_max_n;      /* multilevel layouts: levels with at most this   */
                            /* many vertices (other than Eq. 3 levels) take   */
                            /* the exact O(n^2) entropy sum (the coarsest     */
                            /* level always does); 0 = only the coarsest;    */
                            /* default 16384 (below it the O(n^2) sum costs  */
                            /* less than the tree build and walk)             */
} mm_params;

/* A graph on the device (the input of mm_build_hierarchy). */
typedef struct mm_graph {
  int32_t n;                /* vertices                                       */
  int64_t nnz;              /* CSR entries (2 x edges)                        */
  const int64_t* row_ptr;   /* device [n+1]                                   */
  const int32_t* col;       /* device [nnz]                                   */
  const float* edge_len;    /* device [nnz] target lengths d, or NULL for 1   */
  int32_t num_graphs;       /* 1, or >1 for a block-diagonal batch            */
  const int32_t* graph_ptr; /* host [num_graphs+1] vertex offsets, or NULL    */
} mm_graph;

/* Per-layout statistics written by mm_layout (host struct). */
typedef struct mm_layout_stats {
  int32_t num_levels;
  int32_t total_sweeps;
  int64_t vertex_updates;              /* sum over sweeps of the level size   */
  int32_t level_n[MM_MAX_LEVELS];
  int32_t level_sweeps[MM_MAX_LEVELS];
  double final_alpha;
  double final_rel_change;
  double final_stress;                 /* stress over S of the finest level   */
  int64_t kernel_launches;             /* library kernels launched by the call*/
  float level_rel_change[MM_MAX_LEVELS]; /* relative change |x'-x|/|x| of each */
                                       /* level's last sweep (Sec. 3.2): below */
                                       /* eps_final = converged, else the level*/
                                       /* stopped at max_iters_at_min; batches:*/
                                       /* the largest over the graphs          */
} mm_layout_stats;

typedef struct mm_hierarchy mm_hierarchy;

/* Fills p with the paper's defaults (see mm_params). */
void mm_default_params(mm_params* p);

/* Static description of a status code; never NULL. */
const char* mm_status_string(mm_status s);

/* Message for the last failing call on this thread ("" if none). */
const char* mm_last_error(void);

/*
 * Builds the coarsening hierarchy of Sec. 3.1 on the device: level 0 is the
 * input graph; level h+1 is the contraction of a size-constrained label
 * propagation clustering of level h with U = max(max c, min(b^(h+1), |V|/f)),
 * |V| the input graph's vertex count.
 * A contraction that shrinks the graph by at most 10 percent sets f := 0.7f.
 * For every level it also builds the pair set S (k hops) with target
 * distances d (Sec. 3.2: sqrt(c_u) + sqrt(c_v) per edge on coarse levels)
 * and rho_u = sum_S d^-2 (Eq. 2), and sizes the per-sweep workspaces.
 *   g       device graph (validated: CSR shape, symmetry, connectivity)
 *   p       parameters (k, coarsest_n, f, b, lp_rounds, seed, ...)
 *   out     receives the hierarchy; free with mm_free_hierarchy
 * Errors: MM_ERR_INVALID_ARG (malformed graph or params),
 * MM_ERR_NOT_CONNECTED, MM_ERR_OOM, MM_ERR_UNSUPPORTED (k not 1 or 2,
 * more than 2^31 - 1 pair entries, approx_levels > 0 with num_graphs > 1),
 * MM_ERR_CUDA.  Synchronises `stream`.
 */
mm_status mm_build_hierarchy(const mm_graph* g, const mm_params* p,
                             void* stream, mm_hierarchy** out);

/* One level of a caller-supplied hierarchy (device pointers). */
typedef struct mm_level_desc {
  int32_t n;
  int64_t nnz;
  const int64_t* row_ptr;   /* device [n+1]                                   */
  const int32_t* col;       /* device [nnz], symmetric CSR as for mm_graph    */
  const float* omega;       /* device [nnz] edge weights, or NULL for 1       */
  const float* node_c;      /* device [n] node weights c, or NULL for 1       */
  const int32_t* map;       /* device [n] -> vertex of level+1; NULL on the   */
                            /* last level                                     */
} mm_level_desc;

/*
 * Same as mm_build_hierarchy, but the coarsening (Sec. 3.1) is supplied by
 * the caller instead of computed: level 0 is the input graph (target lengths
 * edge_len0, device [nnz] or NULL for 1); each coarser level's pairs use
 * d = sqrt(c_u) + sqrt(c_v) (Sec. 3.2).  Every level's CSR is validated and
 * every map entry must lie in [0, n of the next level).
 */
mm_status mm_build_hierarchy_levels(int32_t num_levels,
                                    const mm_level_desc* levels,
                                    const float* edge_len0, const mm_params* p,
                                    void* stream, mm_hierarchy** out);

/* Releases a hierarchy and its device memory.  NULL is ignored. */
void mm_free_hierarchy(mm_hierarchy* h);

/* Number of levels (level 0 = input graph). */
mm_status mm_hierarchy_levels(const mm_hierarchy* h, int32_t* num_levels);

/* Sizes of one level: vertices, CSR entries of E, entries of S (host out). */
mm_status mm_level_info(const mm_hierarchy* h, int32_t level, int32_t* n,
                        int64_t* nnz_E, int64_t* nnz_S);

/*
 * Copies one level's data into caller device buffers (each may be NULL):
 * the level's CSR (row_ptr int64 [n+1], col [nnzE], omega [nnzE] edge
 * weights of Sec. 3.1), node weights c [n], the map to the next coarser
 * level [n] (undefined on the coarsest), and S (s_ptr int64 [n+1], s_col
 * [nnzS], s_d [nnzS], rho [n]).
 */
mm_status mm_level_export(const mm_hierarchy* h, int32_t level,
                          int64_t* row_ptr, int32_t* col, float* omega,
                          float* c, int32_t* map, int64_t* s_ptr,
                          int32_t* s_col, float* s_d, float* rho,
                          void* stream);

/*
 * One Jacobi iteration of Eq. 2 on `level` (Sec. 3.2), general model over S:
 *   x'_u = (1/rho_u) sum_{v in S_u} w_uv (x_v + d_uv (x_u-x_v)/|x_u-x_v|)
 *        + (alpha/rho_u) sum_{v not in S_u, v != u} r(u,v),
 * r(u,v) = (x_u-x_v)/|x_u-x_v|^2.  The entropy sum is the Barnes-Hut total
 * over all v (quadtree rebuilt from x_in, opening parameter theta from the
 * build parameters) minus the exact r-values over S, or the exact O(n^2) sum
 * when the hierarchy was built with exact_repulsion = 1.  A coincident pair
 * contributes a zero unit vector and a zero r-value.
 *   x_in, x_out  device [2n], must not overlap
 *   stats        host [3] or NULL: sum|x'-x|^2, sum|x|^2 and the stress of
 *                x_in over the unordered pairs of S (Eq. 1); non-NULL
 *                synchronises the stream.
 * Errors: MM_ERR_INVALID_ARG, MM_ERR_NONFINITE (stats requested and the
 * result is not finite), MM_ERR_CUDA.
 */
mm_status mm_sweep(mm_hierarchy* h, int32_t level, double alpha,
                   const float* x_in, float* x_out, double* stats,
                   void* stream);

/*
 * The first two sums of Eq. 3 (Sec. 3.2, "Faster Local Improvement") on
 * `level` of a hierarchy built with approx_levels = h > 0: exact r-values
 * between u and the other vertices with the same representative M(u) on
 * level min(level + h, coarsest), plus nu(v') r(x_u, x'_{v'}) for every
 * other representative v', with nu(v') its number of vertices on `level`
 * and x'_{v'} their midpoint (from x).  On the coarsest level M is the
 * identity and the result is the exact sum.
 *   x device [2n], F_out device [2n] (n of `level`); stream-ordered.
 * Errors: MM_ERR_INVALID_ARG (null pointers, level out of range, a
 * hierarchy built with approx_levels = 0, a batch hierarchy), MM_ERR_CUDA.
 */
mm_status mm_repulsion_h(mm_hierarchy* h, int32_t level, const float* x, float* F_out,
                         void* stream);

/*
 * Full stress of a layout of the input graph (level 0) and its optimal scale
 * (Sec. 4, methodology): F(x) = sum over unordered vertex pairs of
 * w (|x_u - x_v| - d)^2 with d the hop distance and w = d^-2; s minimises
 * sum w (s |x_u - x_v| - d)^2.  Breadth-first searches from every vertex on
 * the device (64 sources per pass), O(n m) work: graphs of at most 131072
 * vertices with unit edge lengths (no edge_len).
 *   x device [2n]; out host [4] = {F(x), s, F(s x), number of pairs}.
 *   Synchronises the stream.
 * Errors: MM_ERR_INVALID_ARG (null pointers, batch hierarchy),
 * MM_ERR_UNSUPPORTED (edge lengths given, n > 131072), MM_ERR_CUDA.
 */
mm_status mm_full_stress(mm_hierarchy* h, const float* x, double* out, void* stream);

/*
 * The long-range sum F_u = sum_{v != u} r(u,v) over all vertices of `level`
 * (the quantity Barnes-Hut approximates).  theta > 0: quadtree with that
 * opening parameter; theta == 0: quadtree opened completely (exact);
 * theta < 0: the tiled exact O(n^2) kernel.
 *   x device [2n], F_out device [2n].
 */
mm_status mm_repulsion(mm_hierarchy* h, int32_t level, const float* x,
                       float theta, float* F_out, void* stream);

/*
 * The multilevel layout of Sec. 3: initial layout of the coarsest level (two
 * vertices at their target distance; more than two placed around the origin
 * and refined), then for every finer level a random polar prolongation
 * (angle in [0, 2pi), radius in [0, sqrt(c(v'))), Philox keyed by p->seed)
 * followed by the alpha schedule of Sec. 3.2.  The whole schedule runs on the
 * device (CUDA graph with a device-side loop); the host waits once.
 *   p        schedule parameters (alpha0, alpha_factor, alpha_min, eps,
 *            eps_final, iters_per_alpha, max_iters_at_min, early_exit, seed);
 *            NULL = the parameters given to mm_build_hierarchy
 *   x_init   device [2 n0] or NULL.  Non-NULL runs the schedule on level 0
 *            only, starting from x_init (resume / dynamic update, Sec. 4.3).
 *   x_out    device [2 n0]
 *   stats    host or NULL
 * Errors: MM_ERR_NONFINITE, MM_ERR_INVALID_ARG, MM_ERR_CUDA.
 */
mm_status mm_layout(mm_hierarchy* h, const mm_params* p, const float* x_init,
                    float* x_out, mm_layout_stats* stats, void* stream);

/*
 * Per-stage timing of one sweep on `level` (no paper counterpart; a
 * measurement aid): one sweep of the level as the multilevel layout runs it
 * (the exact O(n^2) sum on the coarsest level, on levels of at most
 * exact_max_n vertices and with exact_repulsion; else the tree) is run `reps`
 * times from x with CUDA events between its stages, and the mean
 * milliseconds per stage are written to stage_ms (host [8]): bbox, Morton
 * keys + digit histograms, sort passes, radix tree + prefix sums, node
 * records, traverse (or the exact kernel), gather, controller.  work (host
 * [4]) receives the walk's warp node visits and lane interactions (from one
 * instrumented walk), |S| and n.  alpha = 0.3.  x device [2n], unchanged.
 */
mm_status mm_sweep_profile(mm_hierarchy* h, int32_t level, const float* x,
                           int32_t reps, double* stage_ms, int64_t* work,
                           void* stream);

/*
 * Allocation-free Barnes-Hut long-range sum (the paper has no counterpart;
 * this is a deployment variant of the quadtree build and walk behind
 * mm_repulsion).  For callers that cannot call cudaMalloc/cudaFree on their
 * path -- a custom or pool allocator that forbids outside allocations, a
 * real-time loop that cannot take the device synchronisation of cudaFree, a
 * fixed device-memory budget: the caller passes inputs and outputs and the
 * tree workspace lives in one fixed static device array of the library
 * (under 8 MiB, held on every GPU that loads libmm.so until exit).
 *   n      number of points, 1 <= n <= 32768 (larger n: MM_ERR_INVALID_ARG)
 *   x      device [2n] positions; F_out device [2n] receives (both device
 *          memory of the current device, else MM_ERR_INVALID_ARG)
 *          F_u ~ sum_{v != u} r(u,v) with opening parameter theta >= 0
 *          (theta = 0: exact through the tree), with the walk of the
 *          default parameters (leaf_size, bh_group of mm_default_params)
 * The first call on a device (with that device current) resolves the
 * array's address; make it before any stream capture.  All calls share the
 * array: calls whose GPU work overlaps race and must be serialised by the
 * caller.  Synchronises the stream (to report a broken walk).
 */
mm_status mm_repulsion_noalloc(int32_t n, const float* x, float theta,
                               float* F_out, void* stream);

/*
 * Self-test of the timeout path of the library's bounded device waits (no
 * paper counterpart; a deployment check).  Launches one block of the radix
 * sort's look-back pass on a two-tile key set whose first tile never runs,
 * so the block waits for a status word that nothing writes.  The wait gives
 * up after spin_limit polls (1 <= spin_limit <= 2^22; the library's own
 * sorts use 2^22), the kernel finishes and the context stays usable.
 * Returns MM_ERR_TIMEOUT when the wait gave up, as intended, MM_OK if it did
 * not (a broken timeout path), MM_ERR_INVALID_ARG for a spin_limit out of
 * range.  The same MM_ERR_TIMEOUT is what mm_sweep / mm_layout /
 * mm_repulsion return when a real look-back wait gives up.  Allocates a few
 * KB with cudaMallocAsync on `stream`; synchronises it.
 */
mm_status mm_selftest_wait_timeout(int32_t spin_limit, void* stream);

/*
 * Measured FP32 FMA throughput of the current device (no paper counterpart; a
 * measurement aid): `reps` timed launches (after one warm-up) of a kernel of
 * independent FMA chains filling every SM, CUDA events on `stream`.
 * *tflops = FP32 TFLOP/s (2 flops per FMA); ms_per_launch (nullable) = mean
 * launch time.  The ALU-bound kernels' rooflines use it as their peak.
 * Synchronises the stream.
 */
mm_status mm_measure_fp32_peak(int32_t reps, double* tflops, double* ms_per_launch,
                               void* stream);

/* Result of mm_autotune (host struct). */
typedef struct mm_tune_result {
  int32_t gather_lanes[MM_MAX_LEVELS];   /* chosen lanes per S row (0: fused level) */
  int32_t traverse_warps[MM_MAX_LEVELS]; /* chosen warps per walk block (0: fused)  */
  float theta;                           /* chosen opening parameter               */
  double objective_ref;                  /* M (Eq. 1, alpha = 0.008) at the old theta */
  double objective;                      /* M at the chosen theta                  */
  double layout_ms_before;               /* one mm_layout before tuning            */
  double layout_ms_after;                /* one mm_layout after tuning             */
} mm_tune_result;

/*
 * Autotuner (no paper counterpart; a deployment aid).  For every level run by
 * the multi-kernel sweep it times the S update with 1..32 lanes per row and
 * the tree walk with 2..16 warps per block on the level's own data and keeps
 * the fastest; then it lays the graph out once per candidate opening
 * parameter and keeps the fastest theta whose final objective (Eq. 1 at
 * alpha = 0.008, summed over the graphs of a batch) stays within
 * max_rel_drift of the objective at the hierarchy's current theta.  The
 * choices are stored in the hierarchy (and cached per device and level
 * shape for later hierarchies); mm_layout uses them from then on.
 *   thetas     host [n_theta] candidates (NULL: 0.4, 0.5, 0.6, 0.7, 0.8)
 *   out        host or NULL
 * Synchronises the stream; allocates a layout buffer for the trials.
 */
mm_status mm_autotune(mm_hierarchy* h, const float* thetas, int32_t n_theta,
                      double max_rel_drift, mm_tune_result* out, void* stream);

/*
 * The tensor-core GEMM of the learned prolongation's dense layers, exposed
 * for testing (no paper counterpart): C = A * B^T on the tcgen05 tensor
 * cores with BF16 inputs and FP32 accumulation, optional bias[N] and ReLU.
 *   A device BF16 [M x K] row-major, B device BF16 [N x K] row-major,
 *   K in {16, 32, 64, 128}, N = 64 or 128, all buffers 16-byte aligned;
 *   out_f32 (device FP32 [M x N]) and/or out_bf16 (device BF16 [M x N]).
 * Synchronises the stream (reports a tensor-core wait that gave up as
 * MM_ERR_TIMEOUT).
 */
mm_status mm_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A,
                       const void* B, const float* bias, int32_t relu,
                       float* out_f32, void* out_bf16, void* stream);

/*
 * The tensor-core weight-gradient product of the learned prolongation's
 * dense layers, exposed for testing (no paper counterpart):
 *   out[R x 64] = A^T B = sum over v of A[v][r] * B[v][c]
 * on the tcgen05 tensor cores with BF16 inputs and FP32 accumulation (one
 * partial per vertex range, the partials added in a fixed order).
 *   A device BF16 [n x R] row-major, R = 16 or 128; B device BF16 [n x 64]
 *   row-major; both 16-byte aligned; out device FP32 [R x 64].
 * Allocates its partials with cudaMallocAsync on `stream`; synchronises it.
 */
mm_status mm_gemm_bf16_tn(int32_t n, int32_t R, const void* A, const void* B,
                          float* out, void* stream);

/*
 * Timing of the two tensor-core kernels of the learned prolongation at the
 * width of a hidden layer (no paper counterpart; a measurement aid): the
 * layer product [n x 128] x [128 x 64] (BF16 out) and the weight-gradient
 * partials [n x 128]^T x [n x 64], each launched `reps` times after a
 * warm-up on internally allocated operands, CUDA events on `stream`.
 * ms (host [2]) receives the mean milliseconds per launch of each.
 * Synchronises the stream.
 */
mm_status mm_net_gemm_profile(int32_t n, int32_t reps, double* ms, void* stream);

/*
 * Learned prolongation (no paper counterpart; an extension of the
 * prolongation of Sec. 3.2).  A fine vertex v of the coarse vertex p is
 * placed at x'_p + r_v + o_v: r_v is the paper's random polar offset (the
 * same Philox draws as mm_prolong) and o_v = beta_0 a_v + beta_1 b_v +
 * beta_2 r_v + beta_3 g_v a drift predicted by a 3-layer message-passing
 * network (hidden 64, mean aggregation over the fine graph, BF16 tensor-core
 * layers with FP32 accumulation) from 8 invariant features; a_v is the mean
 * direction from x'_p to the coarse positions of v's neighbours in other
 * clusters, b_v the mean direction from x'_p to p's coarse neighbours and
 * g_v = x'_p - (mean of the coarse layout), which expresses the growth of
 * the layout about its centre while a level refines.  Trained on the
 * device (Adam) to reproduce the drift that the plain layout's refinement
 * applies: loss = mean_v |o_v - t_v|^2 / c(p), t_v = x*_v - x'_p - r_v with
 * x* the converged positions of the level.
 */
typedef struct mm_prolong_net mm_prolong_net;
#define MM_NET_PARAMS 17860 /* FP32 parameters: W0[16x64] b0 W1[128x64] b1
                               W2[128x64] b2 Wo[64x4] bo, row-major */

/* One prolongation step's inputs (device pointers). */
typedef struct mm_prolong_sample {
  int32_t n;                 /* fine vertices                                 */
  const int64_t* row_ptr;    /* fine CSR [n+1]                                */
  const int32_t* col;
  const int32_t* map;        /* [n] fine -> coarse                            */
  int32_t n_coarse;
  const int64_t* crow_ptr;   /* coarse CSR [n_coarse+1]                       */
  const int32_t* ccol;
  const float* c_coarse;     /* [n_coarse] node weights c                     */
  const float* x_coarse;     /* [2 n_coarse] coarse layout                    */
  uint64_t seed;             /* Philox key of the polar offsets               */
  int32_t level;             /* level index of the fine graph (Philox counter)*/
  const float* x_target;     /* [2 n] converged fine layout, or NULL          */
} mm_prolong_sample;

/* Creates a network with the given parameters (host [MM_NET_PARAMS]). */
mm_status mm_net_create(const float* params, mm_prolong_net** out);
void mm_net_free(mm_prolong_net* net);
/* Copies the parameters out (get, host) and/or in (set, host); NULL skips. */
mm_status mm_net_params(mm_prolong_net* net, float* get, const float* set);
/* Prolongation: x_fine (device [2n]); with a target, the loss (host). */
mm_status mm_net_forward(mm_prolong_net* net, const mm_prolong_sample* smp,
                         float* x_fine, double* loss, void* stream);
/* Loss and its gradient with respect to every parameter (host outputs). */
mm_status mm_net_gradients(mm_prolong_net* net, const mm_prolong_sample* smp,
                           float* grads, double* loss, void* stream);
/* One Adam step (learning rate lr) on one sample; loss before the step. */
mm_status mm_net_train_step(mm_prolong_net* net, const mm_prolong_sample* smp,
                            float lr, double* loss, void* stream);
/* Attaches (NULL detaches) a network used by mm_layout when
 * params->learned_prolong = 1.  The network must outlive its use. */
mm_status mm_hierarchy_set_net(mm_hierarchy* h, mm_prolong_net* net);
/* mm_layout that also copies every level's final layout into level_x[l]
 * (host array of num_levels device pointers, entries may be NULL): the
 * coarse-to-converged pairs the network is trained on. */
mm_status mm_layout_levels(mm_hierarchy* h, const mm_params* p,
                           float* const* level_x, void* stream);

/*
 * Maxent-stress objective, Eq. 1, general model over S of `level`:
 *   M(x) = sum_{{u,v} in S} w_uv (|x_u-x_v| - d_uv)^2
 *        - alpha sum_{{u,v} not in S, u != v} ln|x_u - x_v|
 * over unordered pairs, exact (all O(n^2) pairs on the device, FP64
 * accumulation).  Coincident pairs contribute 0 to the ln-sum.
 *   x device [2n]; stress, lnsum, M host outputs (each may be NULL).
 * Synchronises the stream.
 */
mm_status mm_objective(mm_hierarchy* h, int32_t level, const float* x,
                       double alpha, double* stress, double* lnsum, double* M,
                       void* stream);

/*
 * The objective of Eq. 1 with the ln-sum estimated by Barnes-Hut (no exact
 * O(n^2) pass; for levels too large for mm_objective): every vertex's log
 * potential sum_{v != u} ln|x_u - x_v| comes from the quadtree walk at
 * opening parameter theta >= 0 (an accepted cell adds count x ln of the
 * centroid distance, leaves are exact, coincident points add 0; theta = 0
 * is the exact sum through the tree), the all-pairs ln-sum is half their
 * sum, and the stress and the ln-sum over S are exact, as in mm_objective.
 * x device [2n] positions of `level`; outputs as mm_objective.
 * Synchronises the stream.
 */
mm_status mm_objective_bh(mm_hierarchy* h, int32_t level, const float* x, double alpha,
                          float theta, double* stress, double* lnsum, double* M,
                          void* stream);

/*
 * The k-hop pair set S of an arbitrary graph (Sec. 2.3 footnote): for every
 * u, all v != u within k hops (k = 1 or 2), d_uv = the shortest such path
 * with edge length edge_len (or 1) -- or sqrt(c_u) + sqrt(c_v) when node_c is
 * given (coarse-level lengths, Sec. 3.2) -- and rho_u = sum d^-2.  Rows are
 * ascending in v.
 *   row_ptr/col device CSR; edge_len, node_c device or NULL.
 *   First call with s_col == NULL: writes s_ptr (device int64 [n+1]) and
 *   *nnz_S (host).  Second call with s_col [nnz_S], s_d [nnz_S], rho [n]
 *   fills S.  Synchronises the stream.
 */
mm_status mm_khop(int32_t n, const int64_t* row_ptr, const int32_t* col,
                  const float* edge_len, const float* node_c, int32_t k,
                  int64_t* s_ptr, int64_t* nnz_S, int32_t* s_col, float* s_d,
                  float* rho, void* stream);

/*
 * Size-constrained label propagation (Sec. 3.1) on the device: `rounds`
 * synchronous rounds in two seeded halves; a vertex moves to the
 * neighbouring cluster of strongest omega-connection whose weight stays
 * <= U; concurrent moves into one cluster are admitted in a seeded priority
 * order while the bound holds.  labels_out device [n].
 */
mm_status mm_cluster(int32_t n, const int64_t* row_ptr, const int32_t* col,
                     const float* omega, const float* node_c, float U,
                     int32_t rounds, uint64_t seed, int32_t level,
                     int32_t* labels_out, void* stream);

/*
 * Cluster contraction (Sec. 3.1): one coarse node per distinct label (coarse
 * id = rank of the label), c' = sum of member weights, coarse edge {a,b}
 * iff some fine edge joins the blocks, omega' = sum of the joining weights
 * (summed in fine-entry order).  Coarse rows ascending.
 *   labels device [n] in [0, n).  Outputs (device): map [n], c_out
 *   [capacity n], crow_ptr int64 [capacity n+1], ccol and comega [capacity
 *   nnz]; n_coarse and nnz_coarse are host outputs.  Synchronises.
 */
mm_status mm_contract(int32_t n, const int64_t* row_ptr, const int32_t* col,
                      const float* omega, const float* node_c,
                      const int32_t* labels, int32_t* map, float* c_out,
                      int64_t* crow_ptr, int32_t* ccol, float* comega,
                      int32_t* n_coarse, int64_t* nnz_coarse, void* stream);

/*
 * Prolongation (Sec. 3.2): x_fine[v] = x_coarse[map[v]] + rad (cos phi,
 * sin phi), phi = 2 pi U1, rad = sqrt(c_coarse[map[v]]) U2, with U1, U2 the
 * top 24 bits of words 0 and 1 of Philox4x32-10(counter = (v, level, 0, 0),
 * key = seed) scaled to [0, 1).  All pointers device.
 */
mm_status mm_prolong(int32_t n_fine, const int32_t* map,
                     const float* x_coarse, const float* c_coarse,
                     uint64_t seed, int32_t level, float* x_fine,
                     void* stream);

/*
 * One-call convenience API with HOST buffers: copies the CSR to the device,
 * builds the hierarchy, runs mm_layout and copies the layout back.
 *   row_ptr host [n+1], col host [nnz], edge_len host [nnz] or NULL,
 *   x_out host [2n], stats host or NULL.
 */
mm_status mm_layout_host(int32_t n, const int64_t* row_ptr,
                         const int32_t* col, const float* edge_len,
                         const mm_params* p, float* x_out,
                         mm_layout_stats* stats, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MM_H */
