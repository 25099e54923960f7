// Internal declarations of the GB300 MulMent library.  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <vector>

#include "mm.h"

namespace mm {

// ---------------------------------------------------------------- errors --
void set_error(const char* fmt, ...);
mm_status cuda_status(cudaError_t e, const char* what, const char* file, int line);

#define MM_CK(call)                                                          \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) return mm::cuda_status(e_, #call, __FILE__, __LINE__); \
  } while (0)

// Propagates an mm_status from a helper.
#define MM_TRY(expr)                      \
  do {                                    \
    mm_status s_ = (expr);                \
    if (s_ != MM_OK) return s_;           \
  } while (0)

// Capacity bound for buffers sized by the SM count (per-block partials);
// grids are sized by num_sms(), the device's own count (152 on GB300: two
// dies of 76 SMs), clamped to this bound.
constexpr int kMaxSMs = 256;
// Multiprocessor count of the current device (cudaDevAttrMultiProcessorCount,
// read once per device).
int num_sms();

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ------------------------------------------------------------ data types --
// One entry of the pair set S: neighbour id and target distance d_uv.
struct __align__(8) SEnt {
  int32_t col;
  float d;
};

// Device-resident state of the alpha schedule (Sec. 3.2).  The sweep kernels
// read alpha and the buffer parity from here; the controller kernel updates
// it after each sweep, so a whole level runs without host round trips.
struct SweepState {
  double alpha;        // alpha of the next sweep
  double last_rel;     // relative change of the last sweep
  double last_stress;  // stress over S of the last sweep's input
  double last_sdx, last_sx;
  int32_t it_in_round; // iterations done at the current alpha
  int32_t total;       // sweeps in this layout so far
  int32_t level_sweeps;
  int32_t parity;      // x lives in buffer [parity]
  int32_t done;
  int32_t error;       // MM_ERR_NONFINITE when a sweep went non-finite
  int32_t pad[2];
};

// Schedule constants (copied into the controller launch).
struct SchedParams {
  double alpha0, alpha_factor, alpha_min, eps, eps_final;
  int32_t iters_per_alpha, max_iters_at_min, early_exit, level_cap;
};

// Error-free float-float addition (Knuth's two-sum, then renormalise): sums
// of (hi, lo) pairs keep ~44 significant bits with FP32 arithmetic only.
// The reductions the schedule needs use it instead of FP64, whose issue rate
// on this part is a small fraction of FP32's.
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float v = s - a.x;
  float e = (a.x - (s - v)) + (b.x - v);
  e += a.y + b.y;
  const float hi = s + e;
  return make_float2(hi, e - (hi - s));
}

__device__ __forceinline__ float2 ff_shfl_xor(float2 v, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

// Block-wide float-float sums of three per-thread values, in a fixed order
// (warp trees, then the warp totals' tree in warp 0).  kT threads (a multiple
// of 32, at most 1024); every thread must call it.  Result in thread 0.
template <int kT>
__device__ __forceinline__ void block_ffsum3(float2 a, float2 b, float2 c, double out[3]) {
  __shared__ float2 sh[3][kT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a = ff_add(a, ff_shfl_xor(a, o));
    b = ff_add(b, ff_shfl_xor(b, o));
    c = ff_add(c, ff_shfl_xor(c, o));
  }
  __syncthreads();
  if (lane == 0) { sh[0][warp] = a; sh[1][warp] = b; sh[2][warp] = c; }
  __syncthreads();
  if (warp == 0) {
    const float2 z = make_float2(0.f, 0.f);
    a = lane < kT / 32 ? sh[0][lane] : z;
    b = lane < kT / 32 ? sh[1][lane] : z;
    c = lane < kT / 32 ? sh[2][lane] : z;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      a = ff_add(a, ff_shfl_xor(a, o));
      b = ff_add(b, ff_shfl_xor(b, o));
      c = ff_add(c, ff_shfl_xor(c, o));
    }
    if (lane == 0) {
      out[0] = (double)a.x + (double)a.y;
      out[1] = (double)b.x + (double)b.y;
      out[2] = (double)c.x + (double)c.y;
    }
  }
}

// One step of the alpha schedule of Sec. 3.2 after a sweep with reductions
// sdx = sum|x'-x|^2, sx = sum|x|^2 and stress: at most iters_per_alpha
// iterations per alpha (fewer when the relative change |x'-x|/|x| drops
// below eps), alpha := max(factor * alpha, alpha_min); at alpha_min iterate
// until the change is below eps_final or max_iters_at_min iterations.
// Flips the buffer parity.  Returns true when the level is done.  Single
// thread.
__device__ __forceinline__ bool schedule_step(SweepState* st, const SchedParams& sp, double sdx,
                                              double sx, double stress, float* trace,
                                              int trace_cap, int* level_sweeps_out) {
  // the relative change in FP32 (the sums are FP64; FP64 square roots and
  // divisions are long instruction sequences on this part)
  const float fsdx = (float)sdx, fsx = (float)sx;
  const double rel = fsx > 0.f ? (double)(sqrtf(fsdx) / sqrtf(fsx))
                               : (fsdx == 0.f ? 0.0 : (double)INFINITY);
  const double alpha = st->alpha;
  const int t = st->total;
  if (trace && t < trace_cap) {
    trace[3 * t] = (float)alpha;
    trace[3 * t + 1] = (float)rel;
    trace[3 * t + 2] = (float)stress;
  }
  st->total = t + 1;
  st->level_sweeps += 1;
  st->parity ^= 1;
  st->it_in_round += 1;
  st->last_rel = rel;
  st->last_stress = stress;
  st->last_sdx = sdx;
  st->last_sx = sx;
  const bool at_min = alpha <= sp.alpha_min;
  const int cap = at_min ? sp.max_iters_at_min : sp.iters_per_alpha;
  const double tol = at_min ? sp.eps_final : sp.eps;
  if ((sp.early_exit && rel < tol) || st->it_in_round >= cap) {
    if (at_min) {
      st->done = 1;
    } else {
      st->alpha = fmax(alpha * sp.alpha_factor, sp.alpha_min);
      st->it_in_round = 0;
    }
  }
  if (!isfinite(sdx) || !isfinite(sx)) {
    st->error = MM_ERR_NONFINITE;
    st->done = 1;
  }
  if (st->level_sweeps >= sp.level_cap) st->done = 1;
  if (level_sweeps_out) {
    // [0, MM_MAX_LEVELS): sweeps per level; the next MM_MAX_LEVELS words
    // hold the FP32 relative change of each level's latest sweep
    *level_sweeps_out = st->level_sweeps;
    level_sweeps_out[MM_MAX_LEVELS] = __float_as_int((float)rel);
  }
  return st->done != 0;
}

// Selects the current position buffer by the device-side parity.
struct XSel {
  const float2* b0;
  const float2* b1;
  const int32_t* parity;
  __device__ __forceinline__ const float2* cur() const { return *parity ? b1 : b0; }
  __device__ __forceinline__ float2* next() const {
    return const_cast<float2*>(*parity ? b0 : b1);
  }
};

// One level of the hierarchy (device arrays).
struct Level {
  int32_t n = 0;
  int64_t nnzE = 0, nnzS = 0;
  int32_t* rp = nullptr;     // [n+1]
  int32_t* col = nullptr;    // [nnzE]
  float* omega = nullptr;    // [nnzE] edge weights (Sec. 3.1)
  float* c = nullptr;        // [n] node weights
  float* elen = nullptr;     // [nnzE] input lengths (level 0 only, nullable)
  int32_t* map = nullptr;    // [n] -> next coarser level
  int32_t* sp = nullptr;     // [n+1]
  SEnt* s = nullptr;         // [nnzS]
  float* rho = nullptr;      // [n]
  int32_t* heavy = nullptr;  // vertices whose |S_u| > heavy_degree
  int32_t n_heavy = 0;
  int32_t max_deg = 0;       // max |S_u|
  int32_t lanes = 1;         // lanes per vertex in the light gather
  int32_t heavy_degree = 0;
  int32_t walk_warps = 0;    // warps per block in the tree walk (0 = default)
  bool fused = false;        // whole level in the single-CTA kernel
  bool split_gather = false; // sums over S beside the walk (gather_sum + update_from_sum)
  double sum_c = 0;
  // Eq. 3 (approx_levels = h > 0, all levels but the coarsest): the map to
  // the level h levels down (or the coarsest, nt vertices), the level's
  // vertices grouped by it (ascending ids) and the groups' offsets
  int32_t* hmap = nullptr;    // [n]
  int32_t* members = nullptr; // [n]
  int32_t* moff = nullptr;    // [nt+1]
  int32_t nt = 0;
};

// Hierarchy order (k_order.cu): every level of a library-built hierarchy is
// renumbered so that clusters are consecutive, in the order of the coarser
// level.  Level 0's permutation and the caller's level-0 CSR are kept.
struct LevelOrder {
  int32_t* perm0 = nullptr;      // [n0] caller's vertex -> internal index
  int32_t* inv0 = nullptr;       // [n0] internal index -> caller's vertex
  int32_t* rp_user = nullptr;    // the caller's level-0 CSR, as validated
  int32_t* col_user = nullptr;
  float* omega_user = nullptr;
  float* elen_user = nullptr;
};
mm_status renumber_levels(std::vector<Level>& levels, LevelOrder& ord, cudaStream_t s);
// out[i] = in[idx[i]]
mm_status permute_positions(int n, const int32_t* idx, const float2* in, float2* out,
                            cudaStream_t s);

// ----------------------------------------------------------- primitives --
struct SortWS {
  uint32_t* counts = nullptr;  // [256 * max_tiles]
  uint32_t* totals = nullptr;  // [256]
  int max_tiles = 0;
};
constexpr int kSortThreads = 256;
constexpr int kSortIPT = 8;
constexpr int kSortTile = kSortThreads * kSortIPT;
// The tree build's sort and prefix-sum tiles hold kSortThreads * ipt keys,
// ipt the largest of 8, 4, 2, 1 that still gives a tile per SM (small levels
// get many small tiles instead of a few large ones); workspaces are sized
// for the smallest tile.
constexpr int kSortMinTile = kSortThreads;
inline int sort_ipt(int64_t n) {
  for (int ipt = kSortIPT; ipt > 1; ipt >>= 1)
    if (ceil_div(n, (int64_t)kSortThreads * ipt) >= num_sms()) return ipt;
  return 1;
}

mm_status sort_ws_alloc(SortWS& ws, int64_t max_n);
void sort_ws_free(SortWS& ws);

// Stable LSD radix sort of (key, value) pairs on bits [begin_bit, end_bit).
// Ping-pongs between the two buffers; *keys_out / *vals_out receive the
// buffer that holds the result.
mm_status radix_sort_u32(uint32_t* k0, uint32_t* k1, int32_t* v0, int32_t* v1, int n,
                         int begin_bit, int end_bit, SortWS& ws, cudaStream_t s,
                         uint32_t** keys_out, int32_t** vals_out);
mm_status radix_sort_u64(uint64_t* k0, uint64_t* k1, int32_t* v0, int32_t* v1, int n,
                         int begin_bit, int end_bit, SortWS& ws, cudaStream_t s,
                         uint64_t** keys_out, int32_t** vals_out);

// Exclusive scan of int32 counts; out[n] receives the total.  ws needs
// scan_ws_bytes(n) bytes.
size_t scan_ws_bytes(int64_t n);
mm_status scan_exclusive_i32(const int32_t* in, int32_t* out, int n, void* ws,
                             cudaStream_t s);
mm_status scan_exclusive_i64(const int32_t* in, int64_t* out, int n, void* ws,
                             cudaStream_t s);

// Reads one small value from the device into *host through a per-thread
// pinned buffer (a copy to pageable memory goes through the driver's shared
// staging buffer, which serialises host threads building a batch), then
// synchronises the stream.
struct PinnedScratch {
  void* p = nullptr;
  ~PinnedScratch() {
    if (p) cudaFreeHost(p);
  }
};
template <typename T>
mm_status read_scalar(const void* dev, T* host, cudaStream_t s) {
  static_assert(sizeof(T) <= 64, "read_scalar reads at most 64 bytes");
  thread_local PinnedScratch buf;
  if (!buf.p) MM_CK(cudaHostAlloc(&buf.p, 64, cudaHostAllocDefault));
  MM_CK(cudaMemcpyAsync(buf.p, dev, sizeof(T), cudaMemcpyDeviceToHost, s));
  MM_CK(cudaStreamSynchronize(s));
  memcpy(host, buf.p, sizeof(T));
  return MM_OK;
}

// ------------------------------------------------------------ quadtree --
// One quadtree cell as the walk reads it: a = (cx, cy, r_crit^2, count),
// b = (first child | -1, escape | -1, first point lo, point count).  Both
// halves share one 32-byte sector, so a visit is a single 256-bit load; the
// integer count makes the point-in-cell test one subtraction and one
// unsigned comparison.
struct __align__(32) NodeRec {
  float4 a;
  int4 b;
};
static_assert(sizeof(NodeRec) == 32 && alignof(NodeRec) == 32,
              "a cell record is one aligned 32-byte sector");

// Workspace of the Barnes-Hut tree, sized for the largest level.
struct TreeWS {
  int64_t cap = 0;
  uint32_t* keys[2] = {nullptr, nullptr};
  int32_t* vals[2] = {nullptr, nullptr};
  float2* xs = nullptr;       // positions in Morton order
  int32_t* lo = nullptr;      // internal nodes [n-1]
  int32_t* hi = nullptr;
  int32_t* left = nullptr;
  int32_t* right = nullptr;
  int32_t* delta = nullptr;
  int32_t* owner = nullptr;   // owner[g] = internal node whose split is g
  int32_t* parent = nullptr;  // all nodes [2n-1]
  ulonglong2* incl = nullptr;     // [n] inclusive fixed-point position sums per sort tile
  ulonglong2* tile_sum = nullptr; // [tiles] tile totals, then their exclusive prefix
  unsigned long long* status = nullptr;  // [4][tiles][256] look-back words
  uint32_t* hist = nullptr;   // [4][256] digit counts
  uint32_t* counters = nullptr;  // [4] tile tickets of the sort passes
  unsigned* walk_next = nullptr;  // next task of the persistent walk (reset by each build)
  int walk_resident = 0;          // blocks of the persistent walk that fit on the device
  NodeRec* node = nullptr;    // [2n-1] cell records (one 32-byte sector each)
  float4* partials = nullptr; // bbox partial results
  float4* root = nullptr;     // (min x, min y, side, key scale)
  uint32_t* ticket = nullptr; // [0] last-block ticket, [1] build epoch
  int* err = nullptr;         // set by a walk that met a broken tree (1) or a
                              // sort pass whose look-back gave up (2)
  cudaStream_t aux = nullptr; // second branch of the build (radix tree); may be null
  cudaEvent_t fork = nullptr, join = nullptr;
};
constexpr int kKeyBits = 16;  // per axis -> 32-bit Morton keys, depth 16

size_t tree_status_words(int64_t n);
// Whether the tree build of n points scans its tile totals in a kernel of
// its own (else the record kernel folds them in).
bool tree_tile_scan(int64_t n);
// Sizes the persistent walk's grid (occupancy query; no allocation).
mm_status walk_setup(TreeWS& ws);
mm_status tree_ws_alloc(TreeWS& ws, int64_t n, cudaStream_t s);
void tree_ws_free(TreeWS& ws);

// Rebuilds the quadtree from the current positions (bbox, Morton keys and
// digit histograms, look-back sort passes, radix tree, 64-bit fixed-point
// prefix sums of the sorted positions, node records).
// ev (nullable, 6 events) records the stage boundaries for profiling.
// leaf: cells with at most `leaf` points become leaves (1..kMaxLeaf).
// with_bbox = false: the root square (and the zeroed sort state) was left
// by the previous sweep's update epilogue or an explicit bh_bbox.
// coarse_keys: Morton keys of 12 bits per axis (cells down to depth 12;
// points in one deepest cell form a bucket), three sort passes instead of
// four -- used with group acceptance, whose walk does not reproduce the
// oracle's per-point cells anyway.
mm_status bh_build(XSel x, int n, float theta, int leaf, TreeWS& ws, cudaStream_t s,
                   cudaEvent_t* ev = nullptr, bool with_bbox = true, bool coarse_keys = false);
// Bounding square of x into ws.root; zeroes the sort histograms and
// counters and starts a new look-back epoch.
mm_status bh_bbox(XSel x, int n, TreeWS& ws, cudaStream_t s);
// Warp-synchronous stackless walk: F[v] = sum over accepted cells / leaves.
// group = false: per-point acceptance (the oracle's Barnes-Hut); true: a
// cell is accepted for a warp's 32 points together (refines every point's
// per-point sum).
// mode: 0 = per-point walk, 1 = group acceptance over 32 Morton-consecutive
// points (one per lane)
mm_status bh_traverse(int n, const TreeWS& ws, float2* F, int warps_per_block,
                      unsigned long long* counters, cudaStream_t s, int mode = 0);

constexpr int kMaxWalkWarps = 16;  // warps per block of the tree walk

// Group acceptance of a parameter set.
inline bool group_of(const mm_params& p) { return p.bh_group != 0; }
// Tiled exact sum F[v] = sum_{u != v} r(v, u).  With part ([kExactPartCap]
// float2) and arrive ([ceil(n / 128)] counters, zero between calls) small n
// split the sources over several blocks per vertex block (partials added in
// a fixed order).
constexpr int kExactPartCap = 1 << 20;
mm_status exact_repulsion(XSel x, int n, float2* F, cudaStream_t s, float2* part = nullptr,
                          unsigned* arrive = nullptr);
// The group walk (bh_group = 1 decisions) over a built tree that also writes
// Phi[u] = sum_{v != u} ln|x_u - x_v| (accepted cells: count x ln of the
// centroid distance; leaves exact; coincident points 0), in input order.
mm_status bh_potential(int n, const TreeWS& ws, float2* F, float* Phi, int warps_per_block,
                       cudaStream_t s);
// One block of the sort pass waits on a status word that nothing publishes;
// *timed_out = 1 when the bounded wait gave up (error bit 2) as it must.
mm_status lookback_selftest(int spin_limit, int* timed_out, cudaStream_t s);

// ------------------------------------------------------ Eq. 3 (MulMent_h) --
// Builds L's map to level min(level + h, top) and its member groups.
mm_status approx_setup(Level& L, const std::vector<Level>& levels, int level, int h,
                       cudaStream_t s);
// F = the first two sums of Eq. 3 for the current positions; xc holds the
// nt midpoints and counts (x', nu) afterwards.
mm_status approx_repulsion(const Level& L, XSel x, float4* xc, float2* F, cudaStream_t s);

// ---------------------------------------------------- full stress (Sec. 4) --
// out = {F(x), s, F(s x), connected pairs} over all unordered pairs of the
// unit-length graph (rp, col) with hop distances; synchronises the stream.
mm_status full_stress(int n, const int32_t* rp, const int32_t* col, const float2* x,
                      double out[4], cudaStream_t s);
constexpr int kFullStressMaxN = 1 << 17;

// ---------------------------------------------------------------- sweep --
constexpr int kGatherThreads = 256;
constexpr int kMaxLightBlocks = kMaxSMs * 16;  // buffer bounds; grids use num_sms()
constexpr int kMaxHeavyBlocks = kMaxSMs * 8;
// Upper bound of gather_blocks() for any lanes setting (partials sizing).
constexpr int kMaxGatherBlocks = kMaxLightBlocks + kMaxHeavyBlocks;
int gather_blocks(const Level& L);
int gather_light_blocks(const Level& L);
int gather_heavy_blocks(const Level& L);
// What the last block of an update launch does once every block's partial
// sums are in (see gather_update): the controller's schedule step, and
// optionally the next sweep's bounding square.
struct SweepEpilogue {
  SweepState* st;
  SchedParams sp;
  float* trace;
  int trace_cap;
  int* lsw;
  cudaGraphConditionalHandle h;
  int use_h;
  unsigned* arrive;       // arrival counter, 0 between sweeps
  float4* box;            // [kMaxGatherBlocks] per-block boxes of x', or null
  float4* root;           // with box: the tree's root square, sort state
  uint32_t* hist;
  uint32_t* counters;
  unsigned* tree_ticket;
};
// Fused Eq. 2 update over S plus per-block partial sums (3 doubles/block);
// with `epi`, the update ends with the schedule step (no controller launch).
mm_status gather_update(const Level& L, XSel x, const float2* F, const SweepState* st,
                        float4* partials, cudaStream_t s, const SweepEpilogue* epi = nullptr);
// The same update in two launches: gather_sum stores each vertex's sums over
// S_u (acc: [n] float4 of the w-weighted targets and of r(u,v); acc_st: [n]
// stress terms) and reads only x, so it can run beside the tree build and
// walk; update_from_sum then finishes the vertices from acc/acc_st and F with
// gather_update's grid and arithmetic (bit-identical results).
mm_status gather_sum(const Level& L, XSel x, float4* acc, float* acc_st, cudaStream_t s);
mm_status update_from_sum(const Level& L, XSel x, const float2* F, const float4* acc,
                          const float* acc_st, const SweepState* st, float4* partials,
                          cudaStream_t s, const SweepEpilogue* epi = nullptr);
// Reduces the partials, applies the alpha schedule, optionally sets the
// graph loop condition.
mm_status controller(int nblocks, const float4* partials, SweepState* st, SchedParams sp,
                     float* trace, int trace_cap, int* level_sweeps_out,
                     cudaGraphConditionalHandle handle, bool use_handle, cudaStream_t s);
// Writes the prolongated positions into xf_direct, or into xc.next() when
// xf_direct is NULL.
mm_status prolong(int n_fine, const int32_t* map, XSel xc, const float* cc, uint64_t seed,
                  int level, float2* xf_direct, cudaStream_t s);
mm_status level_start(SweepState* st, double alpha0, int flip, cudaStream_t s);
mm_status init_coarsest(int n, const float* c, const SEnt* s0, uint64_t seed, int level,
                        float R, float2* x0, SweepState* st, double alpha0, cudaStream_t s);
// out[i] = current position of vertex perm[i] (perm NULL: of vertex i).
mm_status copy_current(XSel x, int n, float2* out, cudaStream_t s,
                       const int32_t* perm = nullptr);

// ------------------------------------------------- fused small levels ---
constexpr int kSmallMaxN = 2048;     // largest level the single-CTA kernel takes
constexpr int kSmallThreads = 1024;

constexpr int kMaxLeaf = 64;  // largest Barnes-Hut leaf bucket

// Leaf size of a parameter set (0 reads as 1).
inline int leaf_of(const mm_params& p) { return p.leaf_size > 0 ? p.leaf_size : 1; }

struct SmallArgs {
  int n;
  int leaf;        // Barnes-Hut leaf bucket size
  int group;       // Barnes-Hut group acceptance
  const int32_t* sp;
  const SEnt* S;
  const float* rho;
  int exact;
  float theta;
  float2* b0;
  float2* b1;
  SweepState* st;
  SchedParams sched;
  float* trace;
  int trace_cap;
  int* lsw;
  int max_sweeps;
  int lanes;       // lanes per S row in the update (power of two <= 32)
  int cluster;     // CTAs that share the level (single-level launches)
  float4* part;    // [2 kSmallMaxN] per-vertex partial sums (two buffers)
  int* err;
  long long* prof; // nullable: clock64 stamps of the first sweep's phases [10]
};
size_t small_level_smem();
mm_status small_level_setup();
int small_level_max_cluster();
// Runs sweeps of one level in one CTA until the schedule ends the level or
// max_sweeps sweeps are done; reads buffer [st->parity], flips it per sweep.
mm_status small_level(const SmallArgs& a, cudaStream_t s);
// One CTA per entry of dev_args (device array of `count` levels).
mm_status small_level_batch(const SmallArgs* dev_args, int count, cudaStream_t s);

// ------------------------------------------------------------ hierarchy --
mm_status validate_graph(int n, int64_t nnz, const int64_t* rp64, const int32_t* col,
                         int32_t* rp32_out, cudaStream_t s);
mm_status build_khop(int n, const int32_t* rp, const int32_t* col, const float* elen,
                     const float* c, int k, int32_t** sp_out, SEnt** s_out, float** rho_out,
                     int64_t* nnz_out, cudaStream_t s);
mm_status cluster_lp(int n, const int32_t* rp, const int32_t* col, const float* omega,
                     const float* c, float U, int rounds, uint64_t seed, int level,
                     int32_t* labels, cudaStream_t s);
mm_status contract(int n, const int32_t* rp, const int32_t* col, const float* omega,
                   const float* c, const int32_t* labels, int32_t* map, Level& out,
                   cudaStream_t s);
mm_status gather_config(Level& L, const mm_params& p, cudaStream_t s);

// --------------------------------------------------------- tensor cores ---
// C[M x N] = A[M x K] * B[N x K]^T on tcgen05 (BF16 in, FP32 accumulate);
// optional bias and ReLU; BF16 and/or FP32 output (row-major [M x N]).
// K in {16, ..., 128} (multiple of 16), N in {64, 128}.  err |= 4 if the
// bounded wait for the tensor cores gave up.
mm_status gemm_bf16(const void* A, int M, int K, const void* B, int N, const float* bias,
                    int relu, void* outb, float* outf, int* err, cudaStream_t s);

mm_status gemm_setup();
// part[b][r][c] = sum over the b-th of `parts` contiguous vertex ranges of
// A[v][r] * B[v][c] on the tensor cores (A BF16 [n x R], R in {16, 128};
// B BF16 [n x 64]; part FP32 [parts x R x 64]); err |= 4 on a wait timeout.
mm_status gemm_tn_partials(const void* A, int n, int R, const void* B, float* part, int parts,
                           int* err, cudaStream_t s);
// out[R x 64] = sum_v A[v]^T B[v] (partials then a fixed-order sum); part
// holds gemm_tn_parts(n) x R x 64 floats.
int gemm_tn_parts(int n);
mm_status gemm_tn_bf16(const void* A, int n, int R, const void* B, float* out, float* part,
                       int* err, cudaStream_t s);

// ------------------------------------------------- learned prolongation ---
constexpr int kNetHidden = 64;
constexpr int kNetFeatures = 8;
constexpr int kNetOut = 4;       // drift coefficients: a, b, r, g
constexpr int kNetParts = 512;   // vertex chunks of the weight-gradient sums

struct Net {
  float* P = nullptr;   // FP32 parameters (flat, see net_offsets)
  float* G = nullptr;   // gradients
  float* M1 = nullptr;  // Adam moments
  float* M2 = nullptr;
  void* Wt[3] = {nullptr, nullptr, nullptr};  // BF16 W_l^T [64 x rows]
  void* Wb[3] = {nullptr, nullptr, nullptr};  // BF16 W_l [rows x 64]
  int* err = nullptr;
  int cap = 0;
  int64_t step = 0;
  void* f = nullptr;         // BF16 features [n x 8]
  float2* basis = nullptr;   // (a, b, r, g) per vertex
  float* stat = nullptr;     // coarse layout mean (x, y) and RMS radius
  void* Hc = nullptr;        // BF16 [n x 128] concatenation
  void* H[3] = {nullptr, nullptr, nullptr};  // BF16 layer outputs [n x 64]
  float* dbeta = nullptr;
  float* dH = nullptr;
  float* dZ = nullptr;
  void* dZb = nullptr;
  float* dHc = nullptr;
  float* part = nullptr;
  double* loss_part = nullptr;
};

// One prolongation sample: fine level (CSR, map to the coarse level) and the
// coarse level (CSR, weights, positions through an XSel).
struct NetSample {
  int n = 0;
  const int32_t* rp = nullptr;
  const int32_t* col = nullptr;
  const int32_t* map = nullptr;
  XSel xc;
  const int32_t* crp = nullptr;
  const int32_t* ccol = nullptr;
  const float* cc = nullptr;
  int nc = 0;  // coarse vertices
  uint64_t seed = 0;
  int level = 0;
};

void net_offsets(int off[9]);
mm_status net_alloc(Net& net, int max_n);
void net_free(Net& net);
mm_status net_sync_weights(Net& net, cudaStream_t s);
mm_status net_forward(Net& net, const NetSample& smp, float2* xout, const float2* target,
                      cudaStream_t s);
mm_status net_backward(Net& net, const NetSample& smp, cudaStream_t s);
mm_status net_adam_step(Net& net, float lr, cudaStream_t s);

// ------------------------------------------------------------ objective --
mm_status objective_exact(const Level& L, const float2* x, double alpha, double out[3],
                          cudaStream_t s);
// As objective_exact, with the all-pairs ln-sum taken as (1/2) sum_u phi[u].
mm_status objective_from_phi(const Level& L, const float2* x, const float* phi, double alpha,
                             double out[3], cudaStream_t s);

// ---------------------------------------------------------------- philox --
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the 4x32 bijection.
__host__ __device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                        uint32_t c3, uint32_t k0, uint32_t k1,
                                                        uint32_t out[4]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

}  // namespace mm
