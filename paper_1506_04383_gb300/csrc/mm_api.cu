// C-ABI entry points and host orchestration of the multilevel layout.
//
// Sec. 3 of the paper: coarsen (SCLaP + contraction) until the coarsest
// level, lay out the coarsest graph, then prolongate level by level and run
// the alpha schedule of Eq. 2 iterations on each.  Here the whole uncoarsening
// is one CUDA graph: per level a child graph (initial layout or prolongation)
// followed by a conditional WHILE node whose body is one sweep (tree build,
// tree walk or exact sum, fused gather/update, controller).  The controller
// kernel decides on the device whether the level continues, so the host
// launches the graph once and waits once.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "mm_internal.cuh"

struct mm_prolong_net {
  int device = 0;
  mm::Net net;
  int32_t* zero = nullptr;  // device int 0 (parity of caller-given positions)
};

struct mm_hierarchy {
  mm_params p;
  mm_prolong_net* net = nullptr;  // learned prolongation (not owned)
  int device = 0;
  cudaStream_t cs = nullptr;  // capture stream (non-blocking)
  std::vector<mm::Level> levels;
  mm::TreeWS tree;
  float2* xb[2] = {nullptr, nullptr};
  float2* F = nullptr;
  mm::LevelOrder ord;                 // hierarchy order of the levels (level 0 mapped)
  float2* pbuf[2] = {nullptr, nullptr};  // level-0 positions in internal order
  float4* partials = nullptr;        // [kMaxGatherBlocks] per-block FP32 sums
  mm::SweepState* state = nullptr;   // layout schedule state
  mm::SweepState* sstate = nullptr;  // standalone calls
  float4* spart = nullptr;           // [2 kSmallMaxN] fused-level partial sums
  float4* xc = nullptr;              // Eq. 3 midpoints and counts (approx_levels > 0)
  float4* box = nullptr;             // [kMaxGatherBlocks] update-block boxes
  unsigned* arrive = nullptr;        // update epilogue arrival counter
  // Eq. 2's sums over S, computed on a parallel branch of each sweep
  float4* gacc = nullptr;            // [n0] weighted targets and r(u,v) sums per vertex
  float* gacc_st = nullptr;          // [n0] stress terms per vertex
  cudaStream_t gs = nullptr;         // stream of that branch
  cudaEvent_t gfork = nullptr, gjoin = nullptr;
  float2* xpart = nullptr;           // [kExactPartCap] chunk partials of the exact sum
  unsigned* xarrive = nullptr;       // [ceil(n0 / 128)] their arrival counters (zero between sweeps)
  int32_t* zero = nullptr;           // device int 0 (parity of standalone calls)
  int32_t* lsw = nullptr;            // [2 MM_MAX_LEVELS] sweeps, last rel. change per level
  float* trace = nullptr;
  int trace_cap = 0;
  int level_cap = 0;
  // cached uncoarsening graph
  cudaGraphExec_t gexec = nullptr;
  mm_params gparams;
  int gsingle = -1;
  // batch of independent graphs (mm_graph.num_graphs > 1): one hierarchy per
  // graph, built by the single-graph path with seed + graph index; the
  // fields above then describe none of them
  std::vector<mm_hierarchy*> subs;
  std::vector<int32_t> gptr;           // vertex offsets of the graphs
  mm::SmallArgs* batch_args = nullptr; // device, fused levels of every round
  float2* xcat = nullptr;              // concatenated result
  int64_t batch_launches = 0;          // kernels per batched layout (fixed part)
};

namespace mm {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

mm_status cuda_status(cudaError_t e, const char* what, const char* file, int line) {
  set_error("%s failed at %s:%d: %s", what, file, line, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA;
}

int gather_light_blocks(const Level& L);

namespace {

__global__ void rp_to_i32(int n, const int64_t* __restrict__ a, int32_t* b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= n) b[i] = (int32_t)a[i];
}
__global__ void i32_to_i64(int n, const int32_t* __restrict__ a, int64_t* b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}
__global__ void fill_f32(int64_t n, float v, float* a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}
__global__ void max_f32(int n, const float* __restrict__ a, int* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicMax(out, __float_as_int(a[i]));  // non-negative floats order as ints
}
__global__ void split_sent(int64_t m, const SEnt* __restrict__ S, int32_t* col, float* d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  if (col) col[i] = S[i].col;
  if (d) d[i] = S[i].d;
}
__global__ void set_state(SweepState* st, double alpha) {
  st->alpha = alpha;
  st->it_in_round = 0;
  st->level_sweeps = 0;
  st->total = 0;
  st->done = 0;
  st->error = 0;
  st->parity = 0;
}

void free_level(Level& L) {
  void* ptrs[] = {L.rp,  L.col,   L.omega, L.c,       L.elen,   L.map, L.sp,
                  L.s,   L.rho,   L.heavy, L.hmap,    L.members, L.moff};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  L = Level();
}

mm_status check_params(const mm_params* p) {
  if (!p) {
    set_error("params is NULL");
    return MM_ERR_INVALID_ARG;
  }
  if (p->struct_version != MM_PARAMS_VERSION) {
    set_error("mm_params.struct_version %u, library expects %u", p->struct_version,
              MM_PARAMS_VERSION);
    return MM_ERR_INVALID_ARG;
  }
  if (p->k != 1 && p->k != 2) {
    set_error("k = %d: the device path supports k = 1 and k = 2", p->k);
    return MM_ERR_UNSUPPORTED;
  }
  if (!(p->theta >= 0.f) || p->coarsest_n < 1 || !(p->f > 0.f) || !(p->b > 1.f) ||
      p->lp_rounds < 0 || p->iters_per_alpha < 1 || p->max_iters_at_min < 1 ||
      !(p->alpha_min > 0) || !(p->alpha0 > 0) || !(p->alpha_factor > 0 && p->alpha_factor < 1) ||
      p->max_levels < 1 || p->max_levels > MM_MAX_LEVELS || p->leaf_size < 0 ||
      p->leaf_size > kMaxLeaf || p->approx_levels < 0 || p->approx_levels > MM_MAX_LEVELS ||
      p->bh_group < 0 || p->bh_group > 1 || p->level_order < 0 || p->level_order > 1 ||
      p->exact_max_n < 0) {
    set_error("parameter out of range");
    return MM_ERR_INVALID_ARG;
  }
  return MM_OK;
}

int alpha_rounds(const mm_params& p) {
  double a = p.alpha0;
  int r = 1;
  while (a > p.alpha_min && r < 1000) {
    a = std::max(a * p.alpha_factor, p.alpha_min);
    ++r;
  }
  return r;
}

SchedParams sched_of(const mm_params& p, int level_cap) {
  SchedParams sp;
  sp.alpha0 = p.alpha0;
  sp.alpha_factor = p.alpha_factor;
  sp.alpha_min = p.alpha_min;
  sp.eps = p.eps;
  sp.eps_final = p.eps_final;
  sp.iters_per_alpha = p.iters_per_alpha;
  sp.max_iters_at_min = p.max_iters_at_min;
  sp.early_exit = p.early_exit;
  sp.level_cap = level_cap;
  return sp;
}

// Host BFS over one (small) level: the coarse graph is connected iff the
// input is, since label propagation only merges adjacent clusters.
mm_status check_connected(const Level& L, cudaStream_t s) {
  if (L.n <= 1) return MM_OK;
  std::vector<int32_t> rp(L.n + 1), col((size_t)std::max<int64_t>(L.nnzE, 1));
  MM_CK(cudaMemcpyAsync(rp.data(), L.rp, sizeof(int32_t) * (L.n + 1), cudaMemcpyDeviceToHost, s));
  if (L.nnzE)
    MM_CK(cudaMemcpyAsync(col.data(), L.col, sizeof(int32_t) * L.nnzE, cudaMemcpyDeviceToHost, s));
  MM_CK(cudaStreamSynchronize(s));
  std::vector<char> seen(L.n, 0);
  std::vector<int32_t> q;
  q.push_back(0);
  seen[0] = 1;
  for (size_t i = 0; i < q.size(); ++i)
    for (int e = rp[q[i]]; e < rp[q[i] + 1]; ++e)
      if (!seen[col[e]]) {
        seen[col[e]] = 1;
        q.push_back(col[e]);
      }
  if ((int)q.size() != L.n) {
    set_error("graph is not connected (%zu of %d coarsest vertices reachable)", q.size(), L.n);
    return MM_ERR_NOT_CONNECTED;
  }
  return MM_OK;
}

// A tree walk that met an out-of-range node id or exceeded its visit budget
// stops and raises a flag (never faults); the host reports it here.
mm_status tree_error(mm_hierarchy* h, cudaStream_t s) {
  int e = 0;
  MM_CK(cudaMemcpyAsync(&e, h->tree.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  MM_CK(cudaStreamSynchronize(s));
  if (e) {
    cudaMemsetAsync(h->tree.err, 0, sizeof(int), s);
    if (e & 2) {
      set_error("a bounded device wait gave up (the sort's look-back)");
      return MM_ERR_TIMEOUT;
    }
    set_error("internal error: Barnes-Hut walk met an inconsistent tree");
    return MM_ERR_CUDA;
  }
  return MM_OK;
}

bool level_approx(const mm_hierarchy* h, int level);

bool level_exact(const mm_hierarchy* h, int level, bool single) {
  if (h->p.exact_repulsion) return true;
  if (single) return false;
  // the coarsest level of a multilevel run is refined with the exact sum,
  // and so is every level of at most exact_max_n vertices (below that size
  // the O(n^2) sum costs less than a tree build and walk)
  if (level == (int)h->levels.size() - 1) return true;
  return !level_approx(h, level) && h->levels[level].n <= h->p.exact_max_n;
}

// The level takes its entropy sum from Eq. 3 (a map to a coarser level).
bool level_approx(const mm_hierarchy* h, int level) {
  return h->p.approx_levels > 0 && h->levels[level].hmap != nullptr;
}

// Library kernels one sweep of a layout's WHILE loop launches (mirrors
// sweep_body with in_loop = true).
int64_t kernels_per_sweep(const mm_hierarchy* h, int level, bool exact) {
  const Level& L = h->levels[level];
  const int64_t upd = 1 + (L.n_heavy > 0 ? 1 : 0);  // update (+ heavy rows), epilogue fused
  if (exact) return upd + 1;                   // tiled exact sum
  if (level_approx(h, level)) return upd + 2;  // midpoints, Eq. 3 sums
  int64_t k = L.split_gather ? 2 * upd : upd;  // sums over S on their branch, then the update
  k += 1 + (group_of(h->p) ? 3 : 4);         // Morton keys + histograms, sort passes
  if (L.n > 1) k += 1;                       // radix tree
  k += 1;                                    // position prefix sums
  if (tree_tile_scan(L.n)) k += 1;           // tile scan (else folded into records)
  return k + 1 + 1;                          // records, walk
}

// Kernels a multi-kernel level launches outside its loop: the bounding
// square before the first sweep (Barnes-Hut levels).
int64_t kernels_before_loop(const mm_hierarchy* h, int level, bool exact) {
  return exact || level_approx(h, level) ? 0 : 1;
}

SmallArgs small_args(mm_hierarchy* h, int level, bool exact, SweepState* st, SchedParams sp,
                     float* trace, int trace_cap, int* lsw, int max_sweeps) {
  const Level& L = h->levels[level];
  SmallArgs a;
  a.n = L.n;
  a.sp = L.sp;
  a.S = L.s;
  a.rho = L.rho;
  a.exact = exact ? 1 : 0;
  a.theta = h->p.theta;
  a.leaf = leaf_of(h->p);
  a.group = group_of(h->p) ? 1 : 0;
  a.b0 = h->xb[0];
  a.b1 = h->xb[1];
  a.st = st;
  a.sched = sp;
  a.trace = trace;
  a.trace_cap = trace_cap;
  a.lsw = lsw;
  a.max_sweeps = max_sweeps;
  a.lanes = L.lanes;
  // one 32-vertex task per CTA up to 16 CTAs (every CTA repeats the tree
  // build, so more CTAs only shorten the walk; measured: 1.8 % faster
  // layouts than 4 tasks per CTA)
  a.cluster = std::max(1, std::min(16, (L.n + 31) / 32));
  a.part = h->spart;
  a.err = h->tree.err;
  a.prof = nullptr;
  return a;
}

// One sweep on `level`: repulsion, fused update whose last block takes the
// schedule step.  in_loop: the sweep is the body of a layout's WHILE loop;
// the update then also leaves the next sweep's bounding square (the first
// one comes from a bh_bbox before the loop), so the tree build skips it.
mm_status sweep_body(mm_hierarchy* h, int level, bool exact, XSel x, SweepState* st,
                     SchedParams sp, float* trace, int trace_cap, int* lsw,
                     cudaGraphConditionalHandle hnd, bool use_h, cudaStream_t s,
                     bool in_loop = false) {
  const Level& L = h->levels[level];
  const bool approx = !exact && level_approx(h, level);
  if (exact) {
    MM_TRY(exact_repulsion(x, L.n, h->F, s, h->xpart, h->xarrive));
  } else if (approx) {
    MM_TRY(approx_repulsion(L, x, h->xc, h->F, s));
  } else {
    // the sums over S_u need only x: on levels where they are heavy, a
    // parallel branch beside the tree build and the walk, joined before the
    // update
    if (L.split_gather) {
      MM_CK(cudaEventRecord(h->gfork, s));
      MM_CK(cudaStreamWaitEvent(h->gs, h->gfork, 0));
      MM_TRY(gather_sum(L, x, h->gacc, h->gacc_st, h->gs));
      MM_CK(cudaEventRecord(h->gjoin, h->gs));
    }
    MM_TRY(bh_build(x, L.n, h->p.theta, leaf_of(h->p), h->tree, s, nullptr, !in_loop,
                    group_of(h->p)));
    MM_TRY(bh_traverse(L.n, h->tree, h->F, L.walk_warps > 0 ? L.walk_warps : h->p.traverse_warps,
                       nullptr, s, h->p.bh_group));
    if (L.split_gather) MM_CK(cudaStreamWaitEvent(s, h->gjoin, 0));
  }
  SweepEpilogue ep{};
  ep.st = st;
  ep.sp = sp;
  ep.trace = trace;
  ep.trace_cap = trace_cap;
  ep.lsw = lsw;
  ep.h = hnd;
  ep.use_h = use_h ? 1 : 0;
  ep.arrive = h->arrive;
  if (in_loop && !exact && !approx) {
    ep.box = h->box;
    ep.root = h->tree.root;
    ep.hist = h->tree.hist;
    ep.counters = h->tree.counters;
    ep.tree_ticket = h->tree.ticket;
  }
  if (exact || approx || !L.split_gather)
    MM_TRY(gather_update(L, x, h->F, st, h->partials, s, &ep));
  else
    MM_TRY(update_from_sum(L, x, h->F, h->gacc, h->gacc_st, st, h->partials, s, &ep));
  return MM_OK;
}

mm_status build_graph(mm_hierarchy* h, const mm_params& p, bool single,
                      float* const* level_out = nullptr) {
  cudaStream_t cs = h->cs;
  XSel x{h->xb[0], h->xb[1], &h->state->parity};
  const SchedParams sp = sched_of(p, h->level_cap);
  cudaGraph_t g = nullptr;
  MM_CK(cudaGraphCreate(&g, 0));
  cudaGraphNode_t prev = nullptr;
  mm_status st = MM_OK;
  auto fail = [&](mm_status s2) {
    cudaGraphDestroy(g);
    return s2;
  };
  auto add_child = [&](auto&& launches) -> mm_status {
    cudaGraph_t sub = nullptr;
    MM_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    mm_status r = launches(cs);
    cudaError_t e = cudaStreamEndCapture(cs, &sub);
    if (r != MM_OK) {
      if (sub) cudaGraphDestroy(sub);
      return r;
    }
    MM_CK(e);
    cudaGraphNode_t node;
    e = cudaGraphAddChildGraphNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, sub);
    cudaGraphDestroy(sub);
    MM_CK(e);
    prev = node;
    return MM_OK;
  };
  auto add_loop = [&](int level, bool exact) -> mm_status {
    if (h->levels[level].fused)
      return add_child([&](cudaStream_t s) -> mm_status {
        return small_level(small_args(h, level, exact, h->state, sp, h->trace, h->trace_cap,
                                      h->lsw + level, 1 << 30),
                           s);
      });
    if (!exact && !level_approx(h, level))  // the first sweep's bounding square; later ones
                                             // come from the update
      MM_TRY(add_child([&](cudaStream_t s) -> mm_status {
        return bh_bbox(x, h->levels[level].n, h->tree, s);
      }));
    cudaGraphConditionalHandle hnd;
    MM_CK(cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault));
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    memset(cp_raw, 0, sizeof(cp_raw));
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hnd;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    MM_CK(cudaGraphAddNode(&node, g, prev ? &prev : nullptr, nullptr, prev ? 1 : 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    MM_CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
    mm_status r = sweep_body(h, level, exact, x, h->state, sp, h->trace, h->trace_cap,
                             h->lsw + level, hnd, true, cs, true);
    cudaGraph_t out = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &out);
    if (r != MM_OK) return r;
    MM_CK(e);
    prev = node;
    return MM_OK;
  };
  const int top = (int)h->levels.size() - 1;
  if (single) {
    st = add_child([&](cudaStream_t s) -> mm_status {
      set_state<<<1, 1, 0, s>>>(h->state, p.alpha0);
      MM_CK(cudaGetLastError());
      return MM_OK;
    });
    if (st == MM_OK) st = add_loop(0, level_exact(h, 0, true));
  } else {
    const Level& C = h->levels[top];
    st = add_child([&](cudaStream_t s) -> mm_status {
      set_state<<<1, 1, 0, s>>>(h->state, p.alpha0);
      MM_CK(cudaGetLastError());
      return init_coarsest(C.n, C.c, C.s, p.seed, top, (float)std::sqrt(C.sum_c), h->xb[0],
                           h->state, p.alpha0, s);
    });
    if (st == MM_OK) st = add_loop(top, level_exact(h, top, false));
    if (st == MM_OK && level_out && level_out[top])
      st = add_child([&](cudaStream_t s) -> mm_status {
        return copy_current(x, C.n, (float2*)level_out[top], s,
                            top == 0 ? h->ord.perm0 : nullptr);
      });
    for (int lv = top - 1; lv >= 0 && st == MM_OK; --lv) {
      const Level& L = h->levels[lv];
      const Level& Cn = h->levels[lv + 1];
      // one alpha schedule spans the run: the coarsest level ends at
      // alpha_min, so every finer level refines at alpha_min
      st = add_child([&](cudaStream_t s) -> mm_status {
        if (p.learned_prolong && h->net) {
          NetSample smp;
          smp.n = L.n;
          smp.rp = L.rp;
          smp.col = L.col;
          smp.map = L.map;
          smp.xc = x;
          smp.crp = Cn.rp;
          smp.ccol = Cn.col;
          smp.cc = Cn.c;
          smp.nc = Cn.n;
          smp.seed = p.seed;
          smp.level = lv;
          MM_TRY(net_forward(h->net->net, smp, nullptr, nullptr, s));
        } else {
          MM_TRY(prolong(L.n, L.map, x, Cn.c, p.seed, lv, nullptr, s));
        }
        return level_start(h->state, p.alpha_min, 1, s);
      });
      if (st == MM_OK) st = add_loop(lv, level_exact(h, lv, false));
      if (st == MM_OK && level_out && level_out[lv])
        st = add_child([&](cudaStream_t s) -> mm_status {
          return copy_current(x, L.n, (float2*)level_out[lv], s,
                              lv == 0 ? h->ord.perm0 : nullptr);
        });
    }
  }
  if (st != MM_OK) return fail(st);
  cudaGraphExec_t ex = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  MM_CK(e);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = ex;
  h->gparams = p;
  h->gsingle = single ? 1 : 0;
  return MM_OK;
}

mm_status level_check(const mm_hierarchy* h, int level) {
  if (!h) {
    set_error("hierarchy is NULL");
    return MM_ERR_INVALID_ARG;
  }
  if (!h->subs.empty()) {
    set_error("per-level calls take a single-graph hierarchy, not a batch");
    return MM_ERR_UNSUPPORTED;
  }
  if (level < 0 || level >= (int)h->levels.size()) {
    set_error("level %d out of range [0, %zu)", level, h->levels.size());
    return MM_ERR_INVALID_ARG;
  }
  return MM_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Level-0 positions cross the C-ABI in the caller's numbering; a
// renumbered hierarchy (level_order) works in its internal order.  in:
// the caller's positions -> an internal copy in pbuf[k] (or x itself).
const float2* x_in_internal(mm_hierarchy* h, int level, const float* x, int k, cudaStream_t s,
                            mm_status* st) {
  *st = MM_OK;
  if (level != 0 || !h->ord.perm0) return (const float2*)x;
  *st = permute_positions(h->levels[0].n, h->ord.inv0, (const float2*)x, h->pbuf[k], s);
  return h->pbuf[k];
}
// out: internal positions (or forces) of level 0 -> the caller's numbering
mm_status x_out_user(mm_hierarchy* h, int level, const float2* xi, float* out, cudaStream_t s) {
  if (level != 0 || !h->ord.perm0) return MM_OK;
  return permute_positions(h->levels[0].n, h->ord.perm0, xi, (float2*)out, s);
}

__global__ void i32_to_i64_k(int n, const int32_t* __restrict__ a, int64_t* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}
__global__ void split_sent_k(int64_t m, const SEnt* __restrict__ s, int32_t* col, float* d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  if (col) col[i] = s[i].col;
  if (d) d[i] = s[i].d;
}
__global__ void map_user_k(int n, const int32_t* __restrict__ perm0,
                           const int32_t* __restrict__ map, int32_t* __restrict__ out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) out[v] = map[perm0[v]];
}
__global__ void gather_f32_k(int n, const int32_t* __restrict__ idx, const float* __restrict__ a,
                             float* __restrict__ b) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) b[v] = a[idx[v]];
}

// Level 0 of a renumbered hierarchy as the caller numbers it: the caller's
// CSR (kept), node weights and map gathered through the permutation, and
// the pair set S rebuilt on the caller's CSR (rows ascending, as
// mm_build_hierarchy builds it).
mm_status export_level0_user(const mm_hierarchy* h, int64_t* row_ptr, int32_t* col, float* omega,
                             float* c, int32_t* map, int64_t* s_ptr, int32_t* s_col, float* s_d,
                             float* rho, cudaStream_t s) {
  const Level& L = h->levels[0];
  const LevelOrder& o = h->ord;
  const int n = L.n;
  if (row_ptr) i32_to_i64_k<<<ceil_div(n + 1, 256), 256, 0, s>>>(n + 1, o.rp_user, row_ptr);
  if (col && L.nnzE)
    MM_CK(cudaMemcpyAsync(col, o.col_user, 4 * L.nnzE, cudaMemcpyDeviceToDevice, s));
  if (omega && L.nnzE)
    MM_CK(cudaMemcpyAsync(omega, o.omega_user, 4 * L.nnzE, cudaMemcpyDeviceToDevice, s));
  if (c) gather_f32_k<<<ceil_div(n, 256), 256, 0, s>>>(n, o.perm0, L.c, c);
  if (map && L.map) map_user_k<<<ceil_div(n, 256), 256, 0, s>>>(n, o.perm0, L.map, map);
  if (s_ptr || s_col || s_d || rho) {
    int32_t* sp = nullptr;
    SEnt* se = nullptr;
    float* r = nullptr;
    int64_t nnzS = 0;
    MM_TRY(build_khop(n, o.rp_user, o.col_user, o.elen_user, nullptr, h->p.k, &sp, &se, &r,
                      &nnzS, s));
    if (s_ptr) i32_to_i64_k<<<ceil_div(n + 1, 256), 256, 0, s>>>(n + 1, sp, s_ptr);
    if ((s_col || s_d) && nnzS)
      split_sent_k<<<ceil_div(nnzS, 256), 256, 0, s>>>(nnzS, se, s_col, s_d);
    if (rho) MM_CK(cudaMemcpyAsync(rho, r, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s));
    cudaFreeAsync(sp, s);
    cudaFreeAsync(se, s);
    cudaFreeAsync(r, s);
  }
  MM_CK(cudaGetLastError());
  return MM_OK;
}

mm_status finish_levels(mm_hierarchy* h, const mm_params* p, cudaStream_t s);
mm_status build_batch(const mm_graph* g, const mm_params* p, cudaStream_t s, mm_hierarchy** out);

// Level arrays and workspaces come from the stream-ordered allocator: its
// pool keeps freed memory for reuse (no release to the driver at every
// synchronisation), and allocations from many host threads building a batch
// do not serialise on the driver the way cudaMalloc does.
void keep_pool(int dev) {
  static std::mutex mu;
  static std::vector<int> done;
  std::lock_guard<std::mutex> lock(mu);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done.push_back(dev);
}

mm_status build(const mm_graph* g, const mm_params* p, cudaStream_t s, mm_hierarchy** out) {
  if (g && g->num_graphs > 1) return build_batch(g, p, s, out);
  MM_TRY(check_params(p));
  if (!g || !out || g->n < 1 || g->nnz < 0 || !g->row_ptr || (g->nnz > 0 && !g->col)) {
    set_error("invalid graph descriptor");
    return MM_ERR_INVALID_ARG;
  }
  if (g->nnz >= 0x7fffffffLL) {
    set_error("graphs with 2^31 or more CSR entries are not supported");
    return MM_ERR_UNSUPPORTED;
  }
  mm_hierarchy* h = new mm_hierarchy();
  *out = h;  // freed by the caller's wrapper on error
  h->p = *p;
  MM_CK(cudaGetDevice(&h->device));
  keep_pool(h->device);
  MM_CK(cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking));
  const int n0 = g->n;
  Level L0;
  L0.n = n0;
  L0.nnzE = g->nnz;
  MM_CK(cudaMallocAsync(&L0.rp, sizeof(int32_t) * (size_t)(n0 + 1), s));
  h->levels.push_back(L0);
  Level& l0 = h->levels[0];
  MM_TRY(validate_graph(n0, g->nnz, g->row_ptr, g->col, l0.rp, s));
  MM_CK(cudaMallocAsync(&l0.col, sizeof(int32_t) * (size_t)std::max<int64_t>(g->nnz, 1), s));
  MM_CK(cudaMallocAsync(&l0.omega, sizeof(float) * (size_t)std::max<int64_t>(g->nnz, 1), s));
  MM_CK(cudaMallocAsync(&l0.c, sizeof(float) * (size_t)n0, s));
  if (g->nnz)
    MM_CK(cudaMemcpyAsync(l0.col, g->col, sizeof(int32_t) * g->nnz, cudaMemcpyDeviceToDevice, s));
  if (g->edge_len) {
    MM_CK(cudaMallocAsync(&l0.elen, sizeof(float) * (size_t)std::max<int64_t>(g->nnz, 1), s));
    if (g->nnz)
      MM_CK(cudaMemcpyAsync(l0.elen, g->edge_len, sizeof(float) * g->nnz,
                            cudaMemcpyDeviceToDevice, s));
  }
  fill_f32<<<ceil_div(std::max<int64_t>(g->nnz, 1), 256), 256, 0, s>>>(g->nnz, 1.f, l0.omega);
  fill_f32<<<ceil_div(n0, 256), 256, 0, s>>>(n0, 1.f, l0.c);
  MM_CK(cudaGetLastError());

  // ---- coarsening (Sec. 3.1)
  double f = p->f;
  int stalls = 0;
  int* dmax = nullptr;
  int32_t* labels = nullptr;
  MM_CK(cudaMallocAsync(&dmax, sizeof(int), s));
  MM_CK(cudaMallocAsync(&labels, sizeof(int32_t) * (size_t)n0, s));
  mm_status st = MM_OK;
  while (st == MM_OK && h->levels.back().n > p->coarsest_n &&
         (int)h->levels.size() < p->max_levels && stalls < p->max_stalls) {
    Level& cur = h->levels.back();
    const int hidx = (int)h->levels.size() - 1;
    int maxc_bits = 0;
    cudaMemsetAsync(dmax, 0, sizeof(int), s);
    max_f32<<<ceil_div(cur.n, 256), 256, 0, s>>>(cur.n, cur.c, dmax);
    st = read_scalar(dmax, &maxc_bits, s);
    if (st != MM_OK) break;
    float maxc;
    memcpy(&maxc, &maxc_bits, sizeof(float));
    // |V| of Sec. 3.1 is the input graph's vertex count: W bounds a cluster's
    // weight, and the weights c count input vertices (their sum is n0 on
    // every level)
    const double W = std::min(std::pow((double)p->b, hidx + 1), n0 / f);
    const float U = (float)std::max((double)maxc, W);
    st = cluster_lp(cur.n, cur.rp, cur.col, cur.omega, cur.c, U, p->lp_rounds, p->seed, hidx,
                    labels, s);
    if (st != MM_OK) break;
    Level nxt;
    int32_t* map = nullptr;
    if (cudaMallocAsync(&map, sizeof(int32_t) * (size_t)cur.n, s) != cudaSuccess) {
      st = cuda_status(cudaErrorMemoryAllocation, "cudaMalloc(map)", __FILE__, __LINE__);
      break;
    }
    st = contract(cur.n, cur.rp, cur.col, cur.omega, cur.c, labels, map, nxt, s);
    if (st != MM_OK) {
      cudaFree(map);
      free_level(nxt);
      break;
    }
    if (nxt.n >= cur.n || nxt.n < 2) {
      cudaFree(map);
      free_level(nxt);
      f *= 0.7;
      ++stalls;
      continue;
    }
    stalls = 0;
    if (nxt.n > 0.9 * cur.n) f *= 0.7;
    cur.map = map;
    h->levels.push_back(nxt);
  }
  cudaFreeAsync(dmax, s);
  cudaFreeAsync(labels, s);
  MM_TRY(st);
  if (p->level_order) MM_TRY(renumber_levels(h->levels, h->ord, s));

  return finish_levels(h, p, s);
}

__global__ void check_map(int n, const int32_t* __restrict__ map, int nc, int* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && (map[i] < 0 || map[i] >= nc)) atomicOr(bad, 1);
}

// Copies one caller-described level into library memory (validated).
mm_status import_level(const mm_level_desc& d, const mm_level_desc* next, Level& L,
                       cudaStream_t s) {
  if (d.n < 1 || d.nnz < 0 || !d.row_ptr || (d.nnz > 0 && !d.col)) {
    set_error("invalid level descriptor");
    return MM_ERR_INVALID_ARG;
  }
  L.n = d.n;
  L.nnzE = d.nnz;
  MM_CK(cudaMalloc(&L.rp, sizeof(int32_t) * (size_t)(d.n + 1)));
  MM_TRY(validate_graph(d.n, d.nnz, d.row_ptr, d.col, L.rp, s));
  const size_t m = (size_t)std::max<int64_t>(d.nnz, 1);
  MM_CK(cudaMalloc(&L.col, sizeof(int32_t) * m));
  MM_CK(cudaMalloc(&L.omega, sizeof(float) * m));
  MM_CK(cudaMalloc(&L.c, sizeof(float) * (size_t)d.n));
  if (d.nnz) MM_CK(cudaMemcpyAsync(L.col, d.col, 4 * d.nnz, cudaMemcpyDeviceToDevice, s));
  if (d.omega && d.nnz)
    MM_CK(cudaMemcpyAsync(L.omega, d.omega, 4 * d.nnz, cudaMemcpyDeviceToDevice, s));
  else
    fill_f32<<<ceil_div((int64_t)m, 256), 256, 0, s>>>(d.nnz, 1.f, L.omega);
  if (d.node_c)
    MM_CK(cudaMemcpyAsync(L.c, d.node_c, 4 * (size_t)d.n, cudaMemcpyDeviceToDevice, s));
  else
    fill_f32<<<ceil_div(d.n, 256), 256, 0, s>>>(d.n, 1.f, L.c);
  if (next) {
    if (!d.map) {
      set_error("level map missing");
      return MM_ERR_INVALID_ARG;
    }
    MM_CK(cudaMalloc(&L.map, sizeof(int32_t) * (size_t)d.n));
    MM_CK(cudaMemcpyAsync(L.map, d.map, 4 * (size_t)d.n, cudaMemcpyDeviceToDevice, s));
    int* bad = nullptr;
    int hb = 0;
    MM_CK(cudaMalloc(&bad, sizeof(int)));
    cudaMemsetAsync(bad, 0, sizeof(int), s);
    check_map<<<ceil_div(d.n, 256), 256, 0, s>>>(d.n, L.map, next->n, bad);
    cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(bad);
    MM_CK(e);
    if (hb) {
      set_error("level map entry outside [0, %d)", next->n);
      return MM_ERR_INVALID_ARG;
    }
  }
  MM_CK(cudaGetLastError());
  return MM_OK;
}

mm_status build_explicit(int num_levels, const mm_level_desc* d, const float* elen0,
                         const mm_params* p, cudaStream_t s, mm_hierarchy** out) {
  MM_TRY(check_params(p));
  if (num_levels < 1 || num_levels > MM_MAX_LEVELS || !d || !out) {
    set_error("num_levels must lie in [1, %d]", MM_MAX_LEVELS);
    return MM_ERR_INVALID_ARG;
  }
  mm_hierarchy* h = new mm_hierarchy();
  *out = h;
  h->p = *p;
  MM_CK(cudaGetDevice(&h->device));
  keep_pool(h->device);
  MM_CK(cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking));
  for (int l = 0; l < num_levels; ++l) {
    h->levels.push_back(Level());
    MM_TRY(import_level(d[l], l + 1 < num_levels ? &d[l + 1] : nullptr, h->levels.back(), s));
  }
  if (elen0 && d[0].nnz) {
    Level& L0 = h->levels[0];
    MM_CK(cudaMalloc(&L0.elen, sizeof(float) * (size_t)d[0].nnz));
    MM_CK(cudaMemcpyAsync(L0.elen, elen0, 4 * d[0].nnz, cudaMemcpyDeviceToDevice, s));
  }
  return finish_levels(h, p, s);
}

// Connectivity, pair sets S and gather configuration per level, workspaces.
mm_status finish_levels(mm_hierarchy* h, const mm_params* p, cudaStream_t s) {
  MM_TRY(check_connected(h->levels.back(), s));
  for (size_t lv = 0; lv < h->levels.size(); ++lv) {
    Level& L = h->levels[lv];
    MM_TRY(build_khop(L.n, L.rp, L.col, lv == 0 ? L.elen : nullptr, lv == 0 ? nullptr : L.c,
                      p->k, &L.sp, &L.s, &L.rho, &L.nnzS, s));
    MM_TRY(gather_config(L, *p, s));
    const int lim = p->fused_max_n == 0 ? kSmallMaxN : std::min(p->fused_max_n, kSmallMaxN);
    L.fused = p->fused_max_n >= 0 && L.n <= lim;
  }
  // Eq. 3: every level but the coarsest takes its entropy sum from the level
  // approx_levels below (the fused kernel has no Eq. 3 path: those levels
  // run the sweep kernels)
  int max_nt = 0;
  if (p->approx_levels > 0 && !p->exact_repulsion) {
    for (size_t lv = 0; lv + 1 < h->levels.size(); ++lv) {
      Level& L = h->levels[lv];
      MM_TRY(approx_setup(L, h->levels, (int)lv, p->approx_levels, s));
      L.fused = false;
      max_nt = std::max(max_nt, L.nt);
    }
  }
  MM_TRY(small_level_setup());
  {
    Level& C = h->levels.back();
    std::vector<float> hc(C.n);
    MM_CK(cudaMemcpyAsync(hc.data(), C.c, sizeof(float) * C.n, cudaMemcpyDeviceToHost, s));
    MM_CK(cudaStreamSynchronize(s));
    double sc = 0;
    for (float v : hc) sc += v;
    C.sum_c = sc;
  }

  // ---- workspaces, sized for the largest level
  int n0 = 1;
  for (const Level& L : h->levels) n0 = std::max(n0, L.n);
  MM_TRY(tree_ws_alloc(h->tree, n0, s));
  MM_CK(cudaMallocAsync(&h->xb[0], sizeof(float2) * (size_t)n0, s));
  MM_CK(cudaMallocAsync(&h->xb[1], sizeof(float2) * (size_t)n0, s));
  MM_CK(cudaMallocAsync(&h->F, sizeof(float2) * (size_t)n0, s));
  if (h->ord.perm0) {
    MM_CK(cudaMallocAsync(&h->pbuf[0], sizeof(float2) * (size_t)h->levels[0].n, s));
    MM_CK(cudaMallocAsync(&h->pbuf[1], sizeof(float2) * (size_t)h->levels[0].n, s));
  }
  // partials for the largest grid any lanes setting (autotuner) can launch
  MM_CK(cudaMallocAsync(&h->partials, sizeof(float4) * (size_t)kMaxGatherBlocks, s));
  MM_CK(cudaMallocAsync(&h->state, sizeof(SweepState), s));
  MM_CK(cudaMallocAsync(&h->sstate, sizeof(SweepState), s));
  MM_CK(cudaMallocAsync(&h->spart, sizeof(float4) * 2 * (size_t)kSmallMaxN, s));
  if (max_nt > 0) MM_CK(cudaMallocAsync(&h->xc, sizeof(float4) * (size_t)max_nt, s));
  MM_CK(cudaMallocAsync(&h->box, sizeof(float4) * (size_t)kMaxGatherBlocks, s));
  MM_CK(cudaMallocAsync(&h->arrive, sizeof(unsigned), s));
  MM_CK(cudaMemsetAsync(h->arrive, 0, sizeof(unsigned), s));
  MM_CK(cudaMallocAsync(&h->xpart, sizeof(float2) * (size_t)kExactPartCap, s));
  MM_CK(cudaMallocAsync(&h->xarrive, sizeof(unsigned) * (size_t)ceil_div(n0, 128), s));
  MM_CK(cudaMemsetAsync(h->xarrive, 0, sizeof(unsigned) * (size_t)ceil_div(n0, 128), s));
  MM_CK(cudaMallocAsync(&h->gacc, sizeof(float4) * (size_t)n0, s));
  MM_CK(cudaMallocAsync(&h->gacc_st, sizeof(float) * (size_t)n0, s));
  MM_CK(cudaStreamCreateWithFlags(&h->gs, cudaStreamNonBlocking));
  MM_CK(cudaEventCreateWithFlags(&h->gfork, cudaEventDisableTiming));
  MM_CK(cudaEventCreateWithFlags(&h->gjoin, cudaEventDisableTiming));
  MM_CK(cudaMemsetAsync(h->state, 0, sizeof(SweepState), s));
  MM_CK(cudaMemsetAsync(h->sstate, 0, sizeof(SweepState), s));
  MM_CK(cudaMallocAsync(&h->zero, sizeof(int32_t), s));
  MM_CK(cudaMemsetAsync(h->zero, 0, sizeof(int32_t), s));
  MM_CK(cudaMallocAsync(&h->lsw, sizeof(int32_t) * 2 * MM_MAX_LEVELS, s));
  MM_CK(cudaMemsetAsync(h->lsw, 0, sizeof(int32_t) * 2 * MM_MAX_LEVELS, s));
  MM_CK(cudaStreamSynchronize(s));
  return MM_OK;
}

__global__ void slice_csr(int n, int64_t e0, int a, const int64_t* __restrict__ rp,
                          const int32_t* __restrict__ col, int64_t m, int64_t* srp,
                          int32_t* scol) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= n) srp[i] = rp[a + i] - e0;
  if (i < m) scol[i] = col[e0 + i] - a;
}

// One hierarchy per graph of a block-diagonal batch.  Graph i is built
// exactly as mm_build_hierarchy would build it alone, with seed + i, so its
// batched layout equals its own unbatched layout.
mm_status build_batch(const mm_graph* g, const mm_params* p, cudaStream_t s, mm_hierarchy** out) {
  MM_TRY(check_params(p));
  if (p->approx_levels > 0) {
    set_error("approx_levels (Eq. 3) is not available for batches of graphs");
    return MM_ERR_UNSUPPORTED;
  }
  if (!g->graph_ptr || g->n < 1 || !g->row_ptr) {
    set_error("a batch needs graph_ptr (host) and a CSR");
    return MM_ERR_INVALID_ARG;
  }
  const int G = g->num_graphs;
  std::vector<int32_t> gp(g->graph_ptr, g->graph_ptr + G + 1);
  if (gp[0] != 0 || gp[G] != g->n) {
    set_error("graph_ptr must start at 0 and end at n");
    return MM_ERR_INVALID_ARG;
  }
  for (int i = 0; i < G; ++i)
    if (gp[i + 1] <= gp[i]) {
      set_error("graph %d of the batch is empty or graph_ptr is not increasing", i);
      return MM_ERR_INVALID_ARG;
    }
  mm_hierarchy* h = new mm_hierarchy();
  *out = h;
  h->p = *p;
  h->gptr = gp;
  MM_CK(cudaGetDevice(&h->device));
  keep_pool(h->device);
  MM_CK(cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking));
  std::vector<int64_t> rp(g->n + 1);
  MM_CK(cudaMemcpyAsync(rp.data(), g->row_ptr, sizeof(int64_t) * (g->n + 1),
                        cudaMemcpyDeviceToHost, s));
  MM_CK(cudaStreamSynchronize(s));
  if (rp[g->n] != g->nnz) {
    set_error("row_ptr[n] != nnz");
    return MM_ERR_INVALID_ARG;
  }
  // the graphs are built by a pool of host threads, each on its own
  // non-blocking stream; temporaries are stream-ordered, so the builds overlap
  h->subs.assign(G, nullptr);
  std::atomic<int> next(0);
  std::atomic<int> failed(-1);
  std::string fail_msg;
  mm_status fail_st = MM_OK;
  std::mutex fail_mu;
  auto worker = [&]() {
    cudaSetDevice(h->device);
    cudaStream_t ts = nullptr;
    if (cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess) {
      std::lock_guard<std::mutex> lock(fail_mu);
      if (fail_st == MM_OK) { fail_st = MM_ERR_CUDA; fail_msg = "stream creation failed"; }
      return;
    }
    while (true) {
      const int i = next.fetch_add(1);
      if (i >= G || failed.load() >= 0) break;
      const int a = gp[i], ni = gp[i + 1] - gp[i];
      const int64_t e0 = rp[a], m = rp[gp[i + 1]] - e0;
      int64_t* srp = nullptr;
      int32_t* scol = nullptr;
      float* slen = nullptr;
      mm_status st = MM_OK;
      if (cudaMallocAsync(&srp, sizeof(int64_t) * (size_t)(ni + 1), ts) != cudaSuccess ||
          cudaMallocAsync(&scol, sizeof(int32_t) * (size_t)std::max<int64_t>(m, 1), ts) !=
              cudaSuccess ||
          (g->edge_len &&
           cudaMallocAsync(&slen, sizeof(float) * (size_t)std::max<int64_t>(m, 1), ts) !=
               cudaSuccess)) {
        st = MM_ERR_OOM;
        set_error("allocation of a graph slice failed");
      }
      if (st == MM_OK) {
        slice_csr<<<ceil_div(std::max<int64_t>(ni + 1, m), 256), 256, 0, ts>>>(
            ni, e0, a, g->row_ptr, g->col, m, srp, scol);
        if (slen && m)
          cudaMemcpyAsync(slen, g->edge_len + e0, sizeof(float) * m, cudaMemcpyDeviceToDevice,
                          ts);
        mm_graph sg;
        memset(&sg, 0, sizeof(sg));
        sg.n = ni;
        sg.nnz = m;
        sg.row_ptr = srp;
        sg.col = scol;
        sg.edge_len = slen;
        sg.num_graphs = 1;
        mm_params pi = *p;
        pi.seed = p->seed + (uint64_t)i;
        mm_hierarchy* sub = nullptr;
        st = build(&sg, &pi, ts, &sub);
        h->subs[i] = sub;
      }
      if (srp) cudaFreeAsync(srp, ts);
      if (scol) cudaFreeAsync(scol, ts);
      if (slen) cudaFreeAsync(slen, ts);
      cudaStreamSynchronize(ts);
      if (st != MM_OK) {
        std::lock_guard<std::mutex> lock(fail_mu);
        if (fail_st == MM_OK) {
          fail_st = st;
          fail_msg = "graph " + std::to_string(i) + " of the batch: " + g_err;
          failed.store(i);
        }
      }
    }
    cudaStreamDestroy(ts);
  };
  // host threads of the build (MM_BUILD_THREADS overrides the default): the
  // builds overlap up to about 8 threads (measured on 512 graphs: 13.3 s with
  // 1 thread, 4.7 s with 8, 5.2 s with 16 -- launches and synchronisations
  // then contend in the driver)
  int nthreads = 8;
  if (const char* e = std::getenv("MM_BUILD_THREADS")) nthreads = std::max(1, std::atoi(e));
  const int T = std::max(1, std::min(G, nthreads));
  std::vector<std::thread> pool;
  for (int t = 0; t < T; ++t) pool.emplace_back(worker);
  for (auto& th : pool) th.join();
  // drop empty slots (a failed build) so the hierarchy frees cleanly
  std::vector<mm_hierarchy*> built;
  for (mm_hierarchy* sub : h->subs)
    if (sub) built.push_back(sub);
  if (fail_st != MM_OK) {
    h->subs = built;
    set_error("%s", fail_msg.c_str());
    return fail_st;
  }
  MM_CK(cudaMalloc(&h->xcat, sizeof(float2) * (size_t)g->n));
  return MM_OK;
}

mm_status ensure_trace(mm_hierarchy* h, const mm_params& p) {
  const int per_level = (alpha_rounds(p) - 1) * p.iters_per_alpha + p.max_iters_at_min;
  const int cap = per_level * (int)h->levels.size();
  h->level_cap = per_level;
  if (cap > h->trace_cap) {
    if (h->trace) cudaFree(h->trace);
    h->trace = nullptr;
    MM_CK(cudaMalloc(&h->trace, sizeof(float) * 3 * (size_t)cap));
    h->trace_cap = cap;
    if (h->gexec) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
  }
  return MM_OK;
}

bool same_schedule(const mm_params& a, const mm_params& b) {
  return a.alpha0 == b.alpha0 && a.alpha_factor == b.alpha_factor && a.alpha_min == b.alpha_min &&
         a.eps == b.eps && a.eps_final == b.eps_final && a.iters_per_alpha == b.iters_per_alpha &&
         a.max_iters_at_min == b.max_iters_at_min && a.early_exit == b.early_exit &&
         a.seed == b.seed && a.learned_prolong == b.learned_prolong;
}

// Adds a child graph captured from `launches` after `deps`.
template <typename Fn>
mm_status graph_child(cudaGraph_t g, cudaStream_t cs, const std::vector<cudaGraphNode_t>& deps,
                      Fn&& launches, cudaGraphNode_t* out) {
  cudaGraph_t sub = nullptr;
  MM_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  mm_status r = launches(cs);
  cudaError_t e = cudaStreamEndCapture(cs, &sub);
  if (r != MM_OK) {
    if (sub) cudaGraphDestroy(sub);
    return r;
  }
  MM_CK(e);
  e = cudaGraphAddChildGraphNode(out, g, deps.empty() ? nullptr : deps.data(), deps.size(), sub);
  cudaGraphDestroy(sub);
  MM_CK(e);
  return MM_OK;
}

// Adds a WHILE node after `deps` whose body is one sweep of `level` of h.
mm_status graph_loop(cudaGraph_t g, cudaStream_t cs, const std::vector<cudaGraphNode_t>& deps,
                     mm_hierarchy* h, int level, bool exact, SchedParams sp,
                     cudaGraphNode_t* out) {
  std::vector<cudaGraphNode_t> pre = deps;
  if (!exact) {  // the first sweep's bounding square; later ones come from the update
    cudaGraphNode_t bb;
    XSel xb{h->xb[0], h->xb[1], &h->state->parity};
    MM_TRY(graph_child(g, cs, deps, [&](cudaStream_t s) -> mm_status {
      return bh_bbox(xb, h->levels[level].n, h->tree, s);
    }, &bb));
    pre.assign(1, bb);
  }
  cudaGraphConditionalHandle hnd;
  MM_CK(cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault));
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(raw);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hnd;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  MM_CK(cudaGraphAddNode(out, g, pre.empty() ? nullptr : pre.data(), nullptr, pre.size(), &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  MM_CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal));
  XSel x{h->xb[0], h->xb[1], &h->state->parity};
  mm_status r = sweep_body(h, level, exact, x, h->state, sp, h->trace, h->trace_cap,
                           h->lsw + level, hnd, true, cs, true);
  cudaGraph_t o = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &o);
  MM_TRY(r);
  MM_CK(e);
  return MM_OK;
}

// The batched uncoarsening: rounds aligned at each graph's coarsest level.
// Round r runs level L_g - 1 - r of every graph g that has it: the
// initial layout or prolongation kernels of all graphs, then one launch of
// the fused level kernel with a CTA per small graph-level (each CTA runs
// that level's whole schedule), and a WHILE loop per larger level, all
// larger levels of a round in parallel graph branches.
mm_status build_graph_batch(mm_hierarchy* h, const mm_params& p) {
  cudaStream_t cs = h->cs;
  const int G = (int)h->subs.size();
  int rounds = 0;
  for (mm_hierarchy* sub : h->subs) rounds = std::max(rounds, (int)sub->levels.size());
  const SchedParams sp = sched_of(p, h->subs.empty() ? 1 : h->subs[0]->level_cap);
  std::vector<SmallArgs> args;
  std::vector<int> off(rounds + 1, 0);
  for (int r = 0; r < rounds; ++r) {
    off[r] = (int)args.size();
    for (int i = 0; i < G; ++i) {
      mm_hierarchy* sub = h->subs[i];
      const int lev = (int)sub->levels.size() - 1 - r;
      if (lev < 0 || sub->levels[0].n < 2 || !sub->levels[lev].fused) continue;
      args.push_back(small_args(sub, lev, level_exact(sub, lev, false), sub->state, sp, nullptr,
                                0, sub->lsw + lev, 1 << 30));
    }
  }
  off[rounds] = (int)args.size();
  if (h->batch_args) cudaFree(h->batch_args);
  h->batch_args = nullptr;
  MM_CK(cudaMalloc(&h->batch_args, sizeof(SmallArgs) * std::max<size_t>(args.size(), 1)));
  if (!args.empty())
    MM_CK(cudaMemcpy(h->batch_args, args.data(), sizeof(SmallArgs) * args.size(),
                     cudaMemcpyHostToDevice));
  cudaGraph_t g = nullptr;
  MM_CK(cudaGraphCreate(&g, 0));
  std::vector<cudaGraphNode_t> join;
  mm_status st = MM_OK;
  int64_t launches = 0;
  for (int r = 0; r < rounds && st == MM_OK; ++r) {
    cudaGraphNode_t pre;
    st = graph_child(g, cs, join, [&](cudaStream_t s) -> mm_status {
      for (int i = 0; i < G; ++i) {
        mm_hierarchy* sub = h->subs[i];
        const int L = (int)sub->levels.size();
        const int lev = L - 1 - r;
        if (lev < 0 || sub->levels[0].n < 2) continue;
        const uint64_t seed = p.seed + (uint64_t)i;
        if (lev == L - 1) {
          const Level& C = sub->levels[lev];
          set_state<<<1, 1, 0, s>>>(sub->state, p.alpha0);
          MM_TRY(init_coarsest(C.n, C.c, C.s, seed, lev, (float)std::sqrt(C.sum_c), sub->xb[0],
                               sub->state, p.alpha0, s));
        } else {
          XSel x{sub->xb[0], sub->xb[1], &sub->state->parity};
          MM_TRY(prolong(sub->levels[lev].n, sub->levels[lev].map, x, sub->levels[lev + 1].c,
                         seed, lev, nullptr, s));
          MM_TRY(level_start(sub->state, p.alpha_min, 1, s));
        }
        launches += 2;
      }
      return MM_OK;
    }, &pre);
    if (st != MM_OK) break;
    join.clear();
    if (off[r + 1] > off[r]) {
      cudaGraphNode_t fused;
      st = graph_child(g, cs, {pre}, [&](cudaStream_t s) -> mm_status {
        return small_level_batch(h->batch_args + off[r], off[r + 1] - off[r], s);
      }, &fused);
      join.push_back(fused);
      launches += 1;
    }
    for (int i = 0; i < G && st == MM_OK; ++i) {
      mm_hierarchy* sub = h->subs[i];
      const int lev = (int)sub->levels.size() - 1 - r;
      if (lev < 0 || sub->levels[0].n < 2 || sub->levels[lev].fused) continue;
      cudaGraphNode_t loop;
      st = graph_loop(g, cs, {pre}, sub, lev, level_exact(sub, lev, false), sp, &loop);
      join.push_back(loop);
    }
    if (join.empty()) join.push_back(pre);
  }
  if (st == MM_OK) {
    cudaGraphNode_t fin;
    st = graph_child(g, cs, join, [&](cudaStream_t s) -> mm_status {
      for (int i = 0; i < G; ++i) {
        mm_hierarchy* sub = h->subs[i];
        const int n = sub->levels[0].n;
        if (n < 2) {
          MM_CK(cudaMemsetAsync(h->xcat + h->gptr[i], 0, sizeof(float2) * n, s));
          continue;
        }
        XSel x{sub->xb[0], sub->xb[1], &sub->state->parity};
        MM_TRY(copy_current(x, n, h->xcat + h->gptr[i], s, sub->ord.perm0));
        launches += 1;
      }
      return MM_OK;
    }, &fin);
  }
  if (st != MM_OK) {
    cudaGraphDestroy(g);
    return st;
  }
  cudaGraphExec_t ex = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  MM_CK(e);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = ex;
  h->gparams = p;
  h->gsingle = 0;
  h->batch_launches = launches;
  return MM_OK;
}

mm_status layout_batch(mm_hierarchy* h, const mm_params& p, const float* x_init, float* x_out,
                       mm_layout_stats* stats, cudaStream_t s) {
  if (x_init) {
    set_error("a batched hierarchy lays out from scratch only (x_init must be NULL)");
    return MM_ERR_UNSUPPORTED;
  }
  for (mm_hierarchy* sub : h->subs) MM_TRY(ensure_trace(sub, p));
  if (!h->gexec || !same_schedule(h->gparams, p)) MM_TRY(build_graph_batch(h, p));
  for (mm_hierarchy* sub : h->subs)
    MM_CK(cudaMemsetAsync(sub->lsw, 0, sizeof(int32_t) * 2 * MM_MAX_LEVELS, s));
  MM_CK(cudaGraphLaunch(h->gexec, s));
  const int64_t n = h->gptr.back();
  MM_CK(cudaMemcpyAsync(x_out, h->xcat, sizeof(float2) * n, cudaMemcpyDeviceToDevice, s));
  const int G = (int)h->subs.size();
  std::vector<SweepState> hs(G);
  // per graph: sweeps per level, then the bits of each level's last
  // relative change (2 x MM_MAX_LEVELS words)
  constexpr size_t kL = 2 * MM_MAX_LEVELS;
  std::vector<int32_t> lsw((size_t)G * kL);
  for (int i = 0; i < G; ++i) {
    MM_CK(cudaMemcpyAsync(&hs[i], h->subs[i]->state, sizeof(SweepState), cudaMemcpyDeviceToHost,
                          s));
    MM_CK(cudaMemcpyAsync(&lsw[(size_t)i * kL], h->subs[i]->lsw, sizeof(int32_t) * kL,
                          cudaMemcpyDeviceToHost, s));
  }
  MM_CK(cudaStreamSynchronize(s));
  int64_t vu = 0, kl = h->batch_launches;
  int tot = 0, err = 0, maxl = 0;
  for (int i = 0; i < G; ++i) {
    mm_hierarchy* sub = h->subs[i];
    const int nl = (int)sub->levels.size();
    maxl = std::max(maxl, nl);
    for (int l = 0; l < nl; ++l) {
      const int32_t sw = lsw[(size_t)i * kL + l];
      vu += (int64_t)sw * sub->levels[l].n;
      tot += sw;
      if (!sub->levels[l].fused) {
        const bool ex = level_exact(sub, l, false);
        kl += kernels_before_loop(sub, l, ex) + (int64_t)sw * kernels_per_sweep(sub, l, ex);
      }
    }
    if (hs[i].error) err = 1;
  }
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->num_levels = maxl;
    stats->total_sweeps = tot;
    stats->vertex_updates = vu;
    stats->kernel_launches = kl + 1;
    // per round: vertices and sweeps summed over the graphs
    for (int i = 0; i < G; ++i) {
      mm_hierarchy* sub = h->subs[i];
      const int nl = (int)sub->levels.size();
      for (int l = 0; l < nl; ++l) {
        const int r = nl - 1 - l;
        const int slot = maxl - 1 - r;
        stats->level_n[slot] += sub->levels[l].n;
        stats->level_sweeps[slot] += lsw[(size_t)i * kL + l];
        float rel;
        memcpy(&rel, &lsw[(size_t)i * kL + MM_MAX_LEVELS + l], sizeof(rel));
        if (!(rel <= stats->level_rel_change[slot])) stats->level_rel_change[slot] = rel;
      }
    }
  }
  if (err) {
    set_error("a sweep produced non-finite coordinates");
    return MM_ERR_NONFINITE;
  }
  for (mm_hierarchy* sub : h->subs) MM_TRY(tree_error(sub, s));
  return MM_OK;
}

mm_status layout(mm_hierarchy* h, const mm_params* pin, const float* x_init, float* x_out,
                 mm_layout_stats* stats, cudaStream_t s) {
  mm_params p = h->p;
  if (pin) {
    MM_TRY(check_params(pin));
    p.alpha0 = pin->alpha0; p.alpha_factor = pin->alpha_factor; p.alpha_min = pin->alpha_min;
    p.eps = pin->eps; p.eps_final = pin->eps_final; p.iters_per_alpha = pin->iters_per_alpha;
    p.max_iters_at_min = pin->max_iters_at_min; p.early_exit = pin->early_exit;
    p.seed = pin->seed;
    p.learned_prolong = pin->learned_prolong;
  }
  if (p.learned_prolong && !h->net) {
    set_error("learned_prolong = 1 but no network is attached (mm_hierarchy_set_net)");
    return MM_ERR_INVALID_ARG;
  }
  if (!x_out) {
    set_error("x_out is NULL");
    return MM_ERR_INVALID_ARG;
  }
  if (!h->subs.empty()) return layout_batch(h, p, x_init, x_out, stats, s);
  const int n0 = h->levels[0].n;
  const bool single = x_init != nullptr;
  if (stats) memset(stats, 0, sizeof(*stats));
  if (n0 == 1) {  // a single vertex sits at the origin
    MM_CK(cudaMemsetAsync(x_out, 0, sizeof(float2), s));
    MM_CK(cudaStreamSynchronize(s));
    if (stats) { stats->num_levels = 1; stats->level_n[0] = 1; }
    return MM_OK;
  }
  MM_TRY(ensure_trace(h, p));
  if (!h->gexec || h->gsingle != (single ? 1 : 0) || !same_schedule(h->gparams, p))
    MM_TRY(build_graph(h, p, single));
  if (single) {
    if (h->ord.perm0)
      MM_TRY(permute_positions(n0, h->ord.inv0, (const float2*)x_init, h->xb[0], s));
    else
      MM_CK(cudaMemcpyAsync(h->xb[0], x_init, sizeof(float2) * n0, cudaMemcpyDeviceToDevice, s));
  }
  MM_CK(cudaMemsetAsync(h->lsw, 0, sizeof(int32_t) * 2 * MM_MAX_LEVELS, s));
  MM_CK(cudaGraphLaunch(h->gexec, s));
  XSel x{h->xb[0], h->xb[1], &h->state->parity};
  MM_TRY(copy_current(x, n0, (float2*)x_out, s, h->ord.perm0));
  SweepState hs;
  int32_t lsw[2 * MM_MAX_LEVELS];
  MM_CK(cudaMemcpyAsync(&hs, h->state, sizeof(hs), cudaMemcpyDeviceToHost, s));
  MM_CK(cudaMemcpyAsync(lsw, h->lsw, sizeof(lsw), cudaMemcpyDeviceToHost, s));
  MM_CK(cudaStreamSynchronize(s));
  if (stats) {
    const int nl = (int)h->levels.size();
    stats->num_levels = nl;
    int64_t vu = 0;
    for (int i = 0; i < nl; ++i) {
      stats->level_n[i] = h->levels[i].n;
      stats->level_sweeps[i] = lsw[i];
      memcpy(&stats->level_rel_change[i], &lsw[MM_MAX_LEVELS + i], sizeof(float));
      vu += (int64_t)lsw[i] * h->levels[i].n;
    }
    stats->total_sweeps = hs.total;
    stats->vertex_updates = vu;
    stats->final_alpha = hs.alpha;
    stats->final_rel_change = hs.last_rel;
    stats->final_stress = hs.last_stress;
    int64_t kl = 1;  // copy of the result
    for (int i = 0; i < nl; ++i) {
      if (single && i > 0) break;
      // prolongation (the network's 9 kernels when learned) + schedule reset,
      // or the initial layout; then the fused kernel or the sweep loop
      const bool learned = p.learned_prolong && h->net && !single && i < nl - 1;
      const int64_t start = single ? 1 : (learned ? 10 : 2);
      const bool ex = level_exact(h, i, single);
      if (h->levels[i].fused)
        kl += start + 1;
      else
        kl += start + kernels_before_loop(h, i, ex) + (int64_t)lsw[i] * kernels_per_sweep(h, i, ex);
    }
    stats->kernel_launches = kl;
  }
  if (hs.error) {
    set_error("a sweep produced non-finite coordinates");
    return MM_ERR_NONFINITE;
  }
  return tree_error(h, s);
}

// ---------------------------------------------------------------- autotune
struct TuneKey {
  int device, n, lanes_hint;
  int64_t nnzS;
  bool operator<(const TuneKey& o) const {
    if (device != o.device) return device < o.device;
    if (n != o.n) return n < o.n;
    if (nnzS != o.nnzS) return nnzS < o.nnzS;
    return lanes_hint < o.lanes_hint;
  }
};
std::map<TuneKey, std::pair<int, int>> g_tune_cache;
std::mutex g_tune_mu;

// Mean milliseconds of `reps` launches of fn (after one warm-up).
template <typename Fn>
mm_status time_ms(cudaStream_t s, int reps, Fn&& fn, double* ms) {
  cudaEvent_t a, b;
  MM_CK(cudaEventCreate(&a));
  MM_CK(cudaEventCreate(&b));
  mm_status st = fn();
  cudaEventRecord(a, s);
  for (int r = 0; r < reps && st == MM_OK; ++r) st = fn();
  cudaEventRecord(b, s);
  cudaError_t e = cudaEventSynchronize(b);
  float t = 0.f;
  cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  MM_TRY(st);
  MM_CK(e);
  *ms = t / reps;
  return MM_OK;
}

__global__ void fill_uniform(int n, float side, uint32_t k0, float2* x) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  uint32_t z[4];
  philox4x32_10((uint32_t)v, 0u, 7u, 0u, k0, 0u, z);
  x[v] = make_float2(side * (float)(z[0] >> 8) * (1.f / 16777216.f),
                     side * (float)(z[1] >> 8) * (1.f / 16777216.f));
}

// Lanes per row and walk block shape of every multi-kernel level of h.
mm_status tune_levels(mm_hierarchy* h, cudaStream_t s) {
  for (size_t lv = 0; lv < h->levels.size(); ++lv) {
    Level& L = h->levels[lv];
    if (L.fused || L.n < 2) continue;
    const TuneKey key{h->device, L.n, 0, L.nnzS};
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        L.lanes = it->second.first;
        L.walk_warps = it->second.second;
        continue;
      }
    }
    // random positions on the level's scale, F from one real walk
    fill_uniform<<<ceil_div(L.n, 256), 256, 0, s>>>(L.n, sqrtf((float)L.n), 12345u, h->xb[0]);
    XSel x{h->xb[0], h->xb[1], h->zero};
    set_state<<<1, 1, 0, s>>>(h->sstate, 0.008);
    MM_TRY(bh_build(x, L.n, h->p.theta, leaf_of(h->p), h->tree, s, nullptr, true,
                    group_of(h->p)));
    double best = 1e30;
    int best_lanes = L.lanes;
    const int keep = L.lanes;
    for (int lanes = 1; lanes <= 32; lanes <<= 1) {
      L.lanes = lanes;
      double ms = 0;
      MM_TRY(time_ms(s, 5, [&]() { return gather_update(L, x, h->F, h->sstate, h->partials, s); },
                     &ms));
      if (ms < best) { best = ms; best_lanes = lanes; }
    }
    L.lanes = best_lanes;
    (void)keep;
    best = 1e30;
    int best_w = 4;
    for (int w = 1; w <= 16; w <<= 1) {
      double ms = 0;
      MM_TRY(time_ms(s, 5, [&]() { return bh_traverse(L.n, h->tree, h->F, w, nullptr, s, h->p.bh_group); }, &ms));
      if (ms < best) { best = ms; best_w = w; }
    }
    L.walk_warps = best_w;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = {L.lanes, L.walk_warps};
  }
  MM_TRY(tree_error(h, s));
  return MM_OK;
}

// Objective of the finest level (summed over a batch) of layout x.
mm_status layout_objective(mm_hierarchy* h, const float2* x, double* M, cudaStream_t s) {
  double out[3];
  if (h->subs.empty()) {
    MM_TRY(objective_exact(h->levels[0], x, 0.008, out, s));
    *M = out[2];
    return MM_OK;
  }
  double tot = 0;
  for (size_t i = 0; i < h->subs.size(); ++i) {
    MM_TRY(objective_exact(h->subs[i]->levels[0], x + h->gptr[i], 0.008, out, s));
    tot += out[2];
  }
  *M = tot;
  return MM_OK;
}

void set_theta(mm_hierarchy* h, float theta) {
  h->p.theta = theta;
  for (mm_hierarchy* sub : h->subs) sub->p.theta = theta;
  if (h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  for (mm_hierarchy* sub : h->subs)
    if (sub->gexec) {
      cudaGraphExecDestroy(sub->gexec);
      sub->gexec = nullptr;
    }
}

mm_status autotune(mm_hierarchy* h, const float* thetas, int n_theta, double drift,
                   mm_tune_result* out, cudaStream_t s) {
  static const float kDefault[] = {0.4f, 0.5f, 0.6f, 0.7f, 0.8f};
  if (!thetas) {
    thetas = kDefault;
    n_theta = 5;
  }
  if (n_theta < 1 || !(drift >= 0)) {
    set_error("need at least one theta and a non-negative drift bound");
    return MM_ERR_INVALID_ARG;
  }
  const int64_t n = h->subs.empty() ? h->levels[0].n : h->gptr.back();
  float2* x = nullptr;
  MM_CK(cudaMalloc(&x, sizeof(float2) * (size_t)std::max<int64_t>(n, 1)));
  auto run = [&](double* ms, double* M) -> mm_status {
    MM_TRY(layout(h, nullptr, nullptr, (float*)x, nullptr, s));  // builds the graph
    MM_TRY(time_ms(s, 1, [&]() { return layout(h, nullptr, nullptr, (float*)x, nullptr, s); }, ms));
    return layout_objective(h, x, M, s);
  };
  mm_status st = MM_OK;
  double ms0 = 0, M0 = 0;
  const float theta0 = h->p.theta;
  st = run(&ms0, &M0);
  // 1. per-level kernel shapes
  if (st == MM_OK) {
    if (h->subs.empty()) {
      st = tune_levels(h, s);
    } else {
      for (mm_hierarchy* sub : h->subs)
        if (st == MM_OK) st = tune_levels(sub, s);
    }
    set_theta(h, theta0);  // rebuild the graphs with the new shapes
  }
  // 2. theta: fastest candidate within the objective drift bound
  double best_ms = 1e30, best_M = M0;
  float best_theta = theta0;
  for (int i = 0; i < n_theta && st == MM_OK; ++i) {
    set_theta(h, thetas[i]);
    double ms = 0, M = 0;
    st = run(&ms, &M);
    if (st != MM_OK) break;
    const bool ok = std::fabs(M - M0) <= drift * std::fabs(M0);
    if (ok && ms < best_ms) {
      best_ms = ms;
      best_theta = thetas[i];
      best_M = M;
    }
  }
  if (st == MM_OK) {
    set_theta(h, best_theta);
    double ms1 = 0, M1 = 0;
    st = run(&ms1, &M1);
    if (st == MM_OK && out) {
      memset(out, 0, sizeof(*out));
      const Level* lv = h->subs.empty() ? h->levels.data() : h->subs[0]->levels.data();
      const size_t nl = h->subs.empty() ? h->levels.size() : h->subs[0]->levels.size();
      for (size_t i = 0; i < nl && i < MM_MAX_LEVELS; ++i) {
        out->gather_lanes[i] = lv[i].fused ? 0 : lv[i].lanes;
        out->traverse_warps[i] = lv[i].fused ? 0 : (lv[i].walk_warps ? lv[i].walk_warps : 4);
      }
      out->theta = best_theta;
      out->objective_ref = M0;
      out->objective = M1;
      out->layout_ms_before = ms0;
      out->layout_ms_after = ms1;
    }
    (void)best_M;
  }
  cudaFree(x);
  return st;
}

}  // namespace

int num_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 152;
  }
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
    cudaGetLastError();
    v = 152;
  }
  v = std::min(v, kMaxSMs);
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

}  // namespace mm

using namespace mm;

extern "C" {

void mm_default_params(mm_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->struct_version = MM_PARAMS_VERSION;
  p->k = 2;
  p->theta = 0.5f;
  p->exact_repulsion = 0;
  p->coarsest_n = 2;
  p->f = 20.f;
  p->b = 2.f;
  p->lp_rounds = 10;
  p->iters_per_alpha = 2;
  p->alpha0 = 1.0;
  p->alpha_factor = 0.3;
  p->alpha_min = 0.008;
  p->eps = 1e-4;
  p->eps_final = 1e-4;
  p->max_iters_at_min = 100;
  p->early_exit = 1;
  p->seed = 1506;
  p->max_levels = MM_MAX_LEVELS;
  p->max_stalls = 10;
  p->gather_lanes = 0;
  p->heavy_degree = 0;
  p->traverse_warps = 0;
  p->leaf_size = 24;
  p->bh_group = 1;
  p->level_order = 1;
  p->exact_max_n = 16384;
}

const char* mm_status_string(mm_status s) {
  switch (s) {
    case MM_OK: return "ok";
    case MM_ERR_INVALID_ARG: return "invalid argument";
    case MM_ERR_NOT_CONNECTED: return "graph not connected";
    case MM_ERR_CUDA: return "CUDA error";
    case MM_ERR_OOM: return "out of device memory";
    case MM_ERR_NONFINITE: return "non-finite coordinates";
    case MM_ERR_TIMEOUT: return "device wait timed out";
    case MM_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

const char* mm_last_error(void) { return g_err.c_str(); }


mm_status mm_selftest_wait_timeout(int32_t spin_limit, void* stream) {
  g_err.clear();
  if (spin_limit < 1 || spin_limit > (1 << 22)) {
    set_error("spin_limit must be in [1, 2^22], got %d", spin_limit);
    return MM_ERR_INVALID_ARG;
  }
  int timed_out = 0;
  MM_TRY(lookback_selftest(spin_limit, &timed_out, (cudaStream_t)stream));
  if (!timed_out) {
    set_error("the look-back wait on a status word that nothing publishes did not give up");
    return MM_OK;
  }
  set_error("a bounded device wait gave up (the sort's look-back), as the self-test intends");
  return MM_ERR_TIMEOUT;
}

mm_status mm_build_hierarchy(const mm_graph* g, const mm_params* p, void* stream,
                             mm_hierarchy** out) {
  g_err.clear();
  if (!out) {
    set_error("out is NULL");
    return MM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  mm_hierarchy* h = nullptr;
  mm_status st = build(g, p, (cudaStream_t)stream, &h);
  if (st != MM_OK) {
    mm_free_hierarchy(h);
    return st;
  }
  *out = h;
  return MM_OK;
}

mm_status mm_build_hierarchy_levels(int32_t num_levels, const mm_level_desc* levels,
                                    const float* edge_len0, const mm_params* p, void* stream,
                                    mm_hierarchy** out) {
  g_err.clear();
  if (!out) {
    set_error("out is NULL");
    return MM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  mm_hierarchy* h = nullptr;
  mm_status st = build_explicit(num_levels, levels, edge_len0, p, (cudaStream_t)stream, &h);
  if (st != MM_OK) {
    mm_free_hierarchy(h);
    return st;
  }
  *out = h;
  return MM_OK;
}

void mm_free_hierarchy(mm_hierarchy* h) {
  if (!h) return;
  DeviceGuard dg(h->device);
  cudaDeviceSynchronize();
  for (Level& L : h->levels) free_level(L);
  tree_ws_free(h->tree);
  void* ptrs[] = {h->xb[0], h->xb[1], h->F, h->partials, h->state, h->sstate, h->spart, h->xc,
                  h->box, h->arrive, h->gacc, h->gacc_st, h->xpart, h->xarrive,
                  h->zero, h->lsw, h->trace, h->pbuf[0], h->pbuf[1], h->ord.perm0,
                  h->ord.inv0, h->ord.rp_user, h->ord.col_user, h->ord.omega_user,
                  h->ord.elen_user};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->gfork) cudaEventDestroy(h->gfork);
  if (h->gjoin) cudaEventDestroy(h->gjoin);
  if (h->gs) cudaStreamDestroy(h->gs);
  if (h->cs) cudaStreamDestroy(h->cs);
  for (mm_hierarchy* sub : h->subs) mm_free_hierarchy(sub);
  if (h->batch_args) cudaFree(h->batch_args);
  if (h->xcat) cudaFree(h->xcat);
  delete h;
}

mm_status mm_hierarchy_levels(const mm_hierarchy* h, int32_t* num_levels) {
  if (!h || !num_levels) {
    set_error("NULL argument");
    return MM_ERR_INVALID_ARG;
  }
  int32_t nl = (int32_t)h->levels.size();
  for (const mm_hierarchy* sub : h->subs) nl = std::max(nl, (int32_t)sub->levels.size());
  *num_levels = nl;
  return MM_OK;
}

mm_status mm_level_info(const mm_hierarchy* h, int32_t level, int32_t* n, int64_t* nnz_E,
                        int64_t* nnz_S) {
  MM_TRY(level_check(h, level));
  const Level& L = h->levels[level];
  if (n) *n = L.n;
  if (nnz_E) *nnz_E = L.nnzE;
  if (nnz_S) *nnz_S = L.nnzS;
  return MM_OK;
}

mm_status mm_level_export(const mm_hierarchy* h, int32_t level, int64_t* row_ptr, int32_t* col,
                          float* omega, float* c, int32_t* map, int64_t* s_ptr, int32_t* s_col,
                          float* s_d, float* rho, void* stream) {
  g_err.clear();
  MM_TRY(level_check(h, level));
  DeviceGuard dg(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  const Level& L = h->levels[level];
  const int nb = ceil_div(L.n + 1, 256);
  if (level == 0 && h->ord.perm0) return export_level0_user(h, row_ptr, col, omega, c, map,
                                                           s_ptr, s_col, s_d, rho, s);
  if (row_ptr) i32_to_i64<<<nb, 256, 0, s>>>(L.n + 1, L.rp, row_ptr);
  if (col && L.nnzE) MM_CK(cudaMemcpyAsync(col, L.col, 4 * L.nnzE, cudaMemcpyDeviceToDevice, s));
  if (omega && L.nnzE)
    MM_CK(cudaMemcpyAsync(omega, L.omega, 4 * L.nnzE, cudaMemcpyDeviceToDevice, s));
  if (c) MM_CK(cudaMemcpyAsync(c, L.c, 4 * (size_t)L.n, cudaMemcpyDeviceToDevice, s));
  if (map && L.map) MM_CK(cudaMemcpyAsync(map, L.map, 4 * (size_t)L.n, cudaMemcpyDeviceToDevice, s));
  if (s_ptr) i32_to_i64<<<nb, 256, 0, s>>>(L.n + 1, L.sp, s_ptr);
  if ((s_col || s_d) && L.nnzS)
    split_sent<<<ceil_div(L.nnzS, 256), 256, 0, s>>>(L.nnzS, L.s, s_col, s_d);
  if (rho) MM_CK(cudaMemcpyAsync(rho, L.rho, 4 * (size_t)L.n, cudaMemcpyDeviceToDevice, s));
  MM_CK(cudaGetLastError());
  return MM_OK;
}

mm_status mm_sweep(mm_hierarchy* h, int32_t level, double alpha, const float* x_in, float* x_out,
                   double* stats, void* stream) {
  g_err.clear();
  MM_TRY(level_check(h, level));
  if (!x_in || !x_out || x_in == x_out) {
    set_error("x_in and x_out must be distinct device buffers");
    return MM_ERR_INVALID_ARG;
  }
  DeviceGuard dg(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  const Level& L = h->levels[level];
  mm_status cst;
  const float2* xi = x_in_internal(h, level, x_in, 0, s, &cst);
  MM_TRY(cst);
  const bool mapped = level == 0 && h->ord.perm0;
  float2* xo = mapped ? h->pbuf[1] : (float2*)x_out;
  XSel x{xi, xo, h->zero};
  set_state<<<1, 1, 0, s>>>(h->sstate, alpha);
  MM_CK(cudaGetLastError());
  SchedParams sp = sched_of(h->p, 1 << 30);
  sp.iters_per_alpha = 1 << 30;
  sp.max_iters_at_min = 1 << 30;
  sp.early_exit = 0;
  if (L.fused) {
    SmallArgs a = small_args(h, level, h->p.exact_repulsion != 0, h->sstate, sp, nullptr, 0,
                             nullptr, 1);
    a.b0 = const_cast<float2*>(xi);
    a.b1 = xo;
    MM_TRY(small_level(a, s));
  } else {
    MM_TRY(sweep_body(h, level, h->p.exact_repulsion != 0, x, h->sstate, sp, nullptr, 0,
                      nullptr, 0, false, s));
  }
  MM_TRY(x_out_user(h, level, xo, x_out, s));
  if (stats) {
    SweepState hs;
    MM_CK(cudaMemcpyAsync(&hs, h->sstate, sizeof(hs), cudaMemcpyDeviceToHost, s));
    MM_CK(cudaStreamSynchronize(s));
    stats[0] = hs.last_sdx;
    stats[1] = hs.last_sx;
    stats[2] = hs.last_stress;
    if (hs.error) {
      set_error("the sweep produced non-finite coordinates");
      return MM_ERR_NONFINITE;
    }
    return tree_error(h, s);
  }
  return MM_OK;
}

mm_status mm_repulsion(mm_hierarchy* h, int32_t level, const float* x, float theta, float* F_out,
                       void* stream) {
  g_err.clear();
  MM_TRY(level_check(h, level));
  if (!x || !F_out) {
    set_error("NULL buffer");
    return MM_ERR_INVALID_ARG;
  }
  DeviceGuard dg(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int n = h->levels[level].n;
  mm_status cst;
  const float2* xi = x_in_internal(h, level, x, 0, s, &cst);
  MM_TRY(cst);
  const bool mapped = level == 0 && h->ord.perm0;
  float2* Fi = mapped ? h->pbuf[1] : (float2*)F_out;
  XSel xs{xi, xi, h->zero};
  if (theta < 0.f) {
    MM_TRY(exact_repulsion(xs, n, Fi, s));
    return x_out_user(h, level, Fi, F_out, s);
  }
  MM_TRY(bh_build(xs, n, theta, leaf_of(h->p), h->tree, s, nullptr, true, group_of(h->p)));
  MM_TRY(bh_traverse(n, h->tree, Fi, h->p.traverse_warps, nullptr, s, h->p.bh_group));
  MM_TRY(x_out_user(h, level, Fi, F_out, s));
  return tree_error(h, s);
}

mm_status mm_full_stress(mm_hierarchy* h, const float* x, double* out, void* stream) {
  g_err.clear();
  MM_TRY(level_check(h, 0));
  if (!x || !out) {
    set_error("NULL buffer");
    return MM_ERR_INVALID_ARG;
  }
  const Level& L = h->levels[0];
  if (L.elen) {
    set_error("mm_full_stress takes unit edge lengths (hop distances); edge_len was given");
    return MM_ERR_UNSUPPORTED;
  }
  if (L.n > kFullStressMaxN) {
    set_error("mm_full_stress takes at most %d vertices (all pairs), got %d", kFullStressMaxN,
              L.n);
    return MM_ERR_UNSUPPORTED;
  }
  DeviceGuard dg(h->device);
  // the caller's numbering of x matches the caller's CSR
  const int32_t* rp = h->ord.rp_user ? h->ord.rp_user : L.rp;
  const int32_t* col = h->ord.rp_user ? h->ord.col_user : L.col;
  return full_stress(L.n, rp, col, (const float2*)x, out, (cudaStream_t)stream);
}

mm_status mm_repulsion_h(mm_hierarchy* h, int32_t level, const float* x, float* F_out,
                         void* stream) {
  g_err.clear();
  MM_TRY(level_check(h, level));
  if (!x || !F_out) {
    set_error("NULL buffer");
    return MM_ERR_INVALID_ARG;
  }
  if (h->p.approx_levels <= 0 || h->p.exact_repulsion) {
    set_error("mm_repulsion_h needs a hierarchy built with approx_levels > 0 "
              "(and exact_repulsion = 0)");
    return MM_ERR_INVALID_ARG;
  }
  DeviceGuard dg(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  const Level& L = h->levels[level];
  mm_status cst;
  const float2* xi = x_in_internal(h, level, x, 0, s, &cst);
  MM_TRY(cst);
  const bool mapped = level == 0 && h->ord.perm0;
  float2* Fi = mapped ? h->pbuf[1] : (float2*)F_out;
  XSel xs{xi, xi, h->zero};
  // the coarsest level maps to itself: Eq. 3 is then the exact sum
  if (!L.hmap)
    MM_TRY(exact_repulsion(xs, L.n, Fi, s));
  else
    MM_TRY(approx_repulsion(L, xs, h->xc, Fi, s));
  return x_out_user(h, level, Fi, F_out, s);
}

mm_status mm_layout(mm_hierarchy* h, const mm_params* p, const float* x_init, float* x_out,
                    mm_layout_stats* stats, void* stream) {
  g_err.clear();
  if (!h) {
    set_error("hierarchy is NULL");
    return MM_ERR_INVALID_ARG;
  }
  DeviceGuard dg(h->device);
  return layout(h, p, x_init, x_out, stats, (cudaStream_t)stream);
}

mm_status mm_sweep_profile(mm_hierarchy* h, int32_t level, const float* x, int32_t reps,
                           double* stage_ms, int64_t* work, void* stream) {
  g_err.clear();
  MM_TRY(level_check(h, level));
  if (!x || !stage_ms || reps < 1) {
    set_error("invalid arguments");
    return MM_ERR_INVALID_ARG;
  }
  DeviceGuard dg(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  const Level& L = h->levels[level];
  // the entropy sum the multilevel layout uses on this level
  const bool exact = level_exact(h, level, false);
  // level 0 in the hierarchy's own order (as the layout runs it)
  mm_status cst;
  const float2* xi = x_in_internal(h, level, x, 0, s, &cst);
  MM_TRY(cst);
  if (L.fused) {
    // fused level kernel: phases from clock64 stamps of one sweep (stage
    // order: stage x, bbox, sort, radix tree, prefix sums, records, walk or
    // exact sum, update + reductions; schedule step reported as controller)
    long long* prof = nullptr;
    float2* tmp = nullptr;
    MM_CK(cudaMalloc(&prof, 10 * sizeof(long long)));
    MM_CK(cudaMalloc(&tmp, sizeof(float2) * (size_t)std::max(L.n, 1)));
    SchedParams sp = sched_of(h->p, 1 << 30);
    sp.early_exit = 0;
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int khz = 0;
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, h->device);
    mm_status st = MM_OK;
    for (int r = 0; r <= reps && st == MM_OK; ++r) {
      set_state<<<1, 1, 0, s>>>(h->sstate, 0.3);
      MM_CK(cudaMemsetAsync(prof, 0, 10 * sizeof(long long), s));
      SmallArgs a = small_args(h, level, exact, h->sstate, sp, nullptr, 0, nullptr, 1);
      a.b0 = const_cast<float2*>(xi);
      a.b1 = tmp;
      a.prof = prof;
      st = small_level(a, s);
      long long hp[10];
      if (st == MM_OK) {
        cudaMemcpyAsync(hp, prof, sizeof(hp), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) st = MM_ERR_CUDA;
      }
      if (st != MM_OK || r == 0) continue;
      for (int i = 0; i < 9; ++i) {
        const long long d = (hp[i + 1] && hp[i]) ? hp[i + 1] - hp[i] : 0;
        acc[i] += khz > 0 ? (double)d / khz : 0.0;  // cycles / kHz = ms
      }
    }
    cudaFree(prof);
    cudaFree(tmp);
    MM_TRY(st);
    // 9 intervals mapped onto the 8 reported stages: [x staging + bbox],
    // morton+sort, radix tree, prefix sums, records, walk, update, schedule
    stage_ms[0] = (acc[0] + acc[1]) / reps;
    stage_ms[1] = 0.0;
    stage_ms[2] = acc[2] / reps;
    stage_ms[3] = (acc[3] + acc[4]) / reps;
    stage_ms[4] = acc[5] / reps;
    stage_ms[5] = acc[6] / reps;
    stage_ms[6] = acc[7] / reps;
    stage_ms[7] = acc[8] / reps;
    if (work) {
      work[0] = 0;
      work[1] = 0;
      work[2] = L.nnzS;
      work[3] = L.n;
    }
    return tree_error(h, s);
  }
  float2* tmp = nullptr;
  unsigned long long* cnt = nullptr;
  MM_CK(cudaMalloc(&tmp, sizeof(float2) * (size_t)std::max(L.n, 1)));
  MM_CK(cudaMalloc(&cnt, 2 * sizeof(unsigned long long)));
  MM_CK(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s));
  XSel xs{xi, tmp, h->zero};
  cudaEvent_t ev[9];
  for (auto& e : ev) MM_CK(cudaEventCreate(&e));
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  SchedParams sp = sched_of(h->p, 1 << 30);
  sp.early_exit = 0;
  mm_status st = MM_OK;
  for (int r = 0; r <= reps && st == MM_OK; ++r) {  // r = 0 warms up
    set_state<<<1, 1, 0, s>>>(h->sstate, 0.3);
    if (exact) {
      cudaEventRecord(ev[0], s);
      for (int i = 1; i <= 5; ++i) cudaEventRecord(ev[i], s);
      st = exact_repulsion(xs, L.n, h->F, s, h->xpart, h->xarrive);
    } else {
      st = bh_build(xs, L.n, h->p.theta, leaf_of(h->p), h->tree, s, ev, true, group_of(h->p));
      if (st == MM_OK)
        st = bh_traverse(L.n, h->tree, h->F, L.walk_warps > 0 ? L.walk_warps : h->p.traverse_warps,
                         nullptr, s, h->p.bh_group);
    }
    // gather stage: the fused update, or on split levels the sums over S
    // alone; controller stage: then also the update from those sums
    const bool split = !exact && L.split_gather;
    cudaEventRecord(ev[6], s);
    if (st == MM_OK)
      st = split ? gather_sum(L, xs, h->gacc, h->gacc_st, s)
                 : gather_update(L, xs, h->F, h->sstate, h->partials, s);
    cudaEventRecord(ev[7], s);
    if (st == MM_OK && split)
      st = update_from_sum(L, xs, h->F, h->gacc, h->gacc_st, h->sstate, h->partials, s);
    if (st == MM_OK)
      st = controller(gather_blocks(L), h->partials, h->sstate, sp, nullptr, 0, nullptr, 0, false, s);
    cudaEventRecord(ev[8], s);
    if (cudaEventSynchronize(ev[8]) != cudaSuccess) {
      st = cuda_status(cudaGetLastError(), "profile sweep", __FILE__, __LINE__);
      break;
    }
    if (r == 0) continue;
    for (int i = 0; i < 8; ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
      acc[i] += ms;
    }
  }
  if (st == MM_OK && !exact && work) {
    st = bh_build(xs, L.n, h->p.theta, leaf_of(h->p), h->tree, s, nullptr, true, group_of(h->p));
    if (st == MM_OK)
      st = bh_traverse(L.n, h->tree, h->F, L.walk_warps > 0 ? L.walk_warps : h->p.traverse_warps,
                       cnt, s, h->p.bh_group);
  }
  unsigned long long hc[2] = {0, 0};
  if (st == MM_OK) {
    cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "profile", __FILE__, __LINE__);
  }
  for (auto& e : ev) cudaEventDestroy(e);
  cudaFree(tmp);
  cudaFree(cnt);
  MM_TRY(st);
  for (int i = 0; i < 8; ++i) stage_ms[i] = acc[i] / reps;
  if (work) {
    work[0] = (int64_t)hc[0];
    work[1] = exact ? (int64_t)L.n * L.n : (int64_t)hc[1];
    work[2] = L.nnzS;
    work[3] = L.n;
  }
  return tree_error(h, s);
}

namespace mm {
namespace {

__global__ void rp_to_i32_k(int n, const int64_t* __restrict__ a, int32_t* b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= n) b[i] = (int32_t)a[i];
}

// ABI sample -> internal sample (int32 row pointers in stream-ordered temps).
struct SampleTmp {
  int32_t* rp = nullptr;
  int32_t* crp = nullptr;
  cudaStream_t s = nullptr;
  ~SampleTmp() {
    if (rp) cudaFreeAsync(rp, s);
    if (crp) cudaFreeAsync(crp, s);
  }
};

mm_status make_sample(mm_prolong_net* net, const mm_prolong_sample* a, NetSample& smp,
                      SampleTmp& tmp, cudaStream_t s) {
  if (!net || !a || a->n < 1 || a->n_coarse < 1 || !a->row_ptr || !a->map || !a->crow_ptr ||
      !a->c_coarse || !a->x_coarse) {
    set_error("invalid prolongation sample");
    return MM_ERR_INVALID_ARG;
  }
  tmp.s = s;
  MM_CK(cudaMallocAsync(&tmp.rp, sizeof(int32_t) * (size_t)(a->n + 1), s));
  MM_CK(cudaMallocAsync(&tmp.crp, sizeof(int32_t) * (size_t)(a->n_coarse + 1), s));
  rp_to_i32_k<<<ceil_div(a->n + 1, 256), 256, 0, s>>>(a->n, a->row_ptr, tmp.rp);
  rp_to_i32_k<<<ceil_div(a->n_coarse + 1, 256), 256, 0, s>>>(a->n_coarse, a->crow_ptr, tmp.crp);
  MM_CK(cudaGetLastError());
  smp.n = a->n;
  smp.rp = tmp.rp;
  smp.col = a->col;
  smp.map = a->map;
  smp.xc = XSel{(const float2*)a->x_coarse, (const float2*)a->x_coarse, net->zero};
  smp.crp = tmp.crp;
  smp.ccol = a->ccol;
  smp.cc = a->c_coarse;
  smp.nc = a->n_coarse;
  smp.seed = a->seed;
  smp.level = a->level;
  MM_TRY(net_alloc(net->net, a->n));
  return MM_OK;
}

mm_status read_loss(Net& net, int n, double* loss, cudaStream_t s) {
  const int parts = ceil_div(n, 256);
  std::vector<double> h((size_t)parts);
  MM_CK(cudaMemcpyAsync(h.data(), net.loss_part, sizeof(double) * parts, cudaMemcpyDeviceToHost,
                        s));
  int err = 0;
  MM_CK(cudaMemcpyAsync(&err, net.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  MM_CK(cudaStreamSynchronize(s));
  if (err) {
    cudaMemsetAsync(net.err, 0, sizeof(int), s);
    set_error("tensor-core wait gave up");
    return MM_ERR_TIMEOUT;
  }
  double t = 0;
  for (double v : h) t += v;
  if (loss) *loss = t;
  return MM_OK;
}

}  // namespace
}  // namespace mm



mm_status mm_net_create(const float* params, mm_prolong_net** out) {
  g_err.clear();
  if (!params || !out) {
    set_error("params and out are required");
    return MM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  mm_prolong_net* net = new mm_prolong_net();
  cudaGetDevice(&net->device);
  mm_status st = gemm_setup();
  if (st == MM_OK) st = net_alloc(net->net, 1);
  if (st == MM_OK && cudaMalloc(&net->zero, sizeof(int32_t)) != cudaSuccess)
    st = cuda_status(cudaErrorMemoryAllocation, "cudaMalloc", __FILE__, __LINE__);
  if (st == MM_OK) cudaMemset(net->zero, 0, sizeof(int32_t));
  if (st == MM_OK) st = mm_net_params(net, nullptr, params);
  if (st != MM_OK) {
    mm_net_free(net);
    return st;
  }
  *out = net;
  return MM_OK;
}

void mm_net_free(mm_prolong_net* net) {
  if (!net) return;
  DeviceGuard dg(net->device);
  cudaDeviceSynchronize();
  net_free(net->net);
  if (net->zero) cudaFree(net->zero);
  delete net;
}

mm_status mm_net_params(mm_prolong_net* net, float* get, const float* set) {
  if (!net) {
    set_error("net is NULL");
    return MM_ERR_INVALID_ARG;
  }
  DeviceGuard dg(net->device);
  if (get) MM_CK(cudaMemcpy(get, net->net.P, sizeof(float) * MM_NET_PARAMS, cudaMemcpyDeviceToHost));
  if (set) {
    MM_CK(cudaMemcpy(net->net.P, set, sizeof(float) * MM_NET_PARAMS, cudaMemcpyHostToDevice));
    MM_CK(cudaMemset(net->net.M1, 0, sizeof(float) * MM_NET_PARAMS));
    MM_CK(cudaMemset(net->net.M2, 0, sizeof(float) * MM_NET_PARAMS));
    net->net.step = 0;
    MM_TRY(net_sync_weights(net->net, 0));
    MM_CK(cudaDeviceSynchronize());
  }
  return MM_OK;
}

mm_status mm_net_forward(mm_prolong_net* net, const mm_prolong_sample* smp, float* x_fine,
                         double* loss, void* stream) {
  g_err.clear();
  if (!net) {
    set_error("net is NULL");
    return MM_ERR_INVALID_ARG;
  }
  DeviceGuard dg(net->device);
  cudaStream_t s = (cudaStream_t)stream;
  NetSample ns;
  SampleTmp tmp;
  MM_TRY(make_sample(net, smp, ns, tmp, s));
  MM_TRY(net_forward(net->net, ns, (float2*)x_fine, (const float2*)smp->x_target, s));
  return read_loss(net->net, ns.n, smp->x_target ? loss : nullptr, s);
}

mm_status mm_net_gradients(mm_prolong_net* net, const mm_prolong_sample* smp, float* grads,
                           double* loss, void* stream) {
  g_err.clear();
  if (!net || !smp || !smp->x_target) {
    set_error("gradients need a network and a sample with x_target");
    return MM_ERR_INVALID_ARG;
  }
  DeviceGuard dg(net->device);
  cudaStream_t s = (cudaStream_t)stream;
  NetSample ns;
  SampleTmp tmp;
  MM_TRY(make_sample(net, smp, ns, tmp, s));
  MM_TRY(net_forward(net->net, ns, nullptr, (const float2*)smp->x_target, s));
  MM_TRY(net_backward(net->net, ns, s));
  MM_TRY(read_loss(net->net, ns.n, loss, s));
  if (grads)
    MM_CK(cudaMemcpy(grads, net->net.G, sizeof(float) * MM_NET_PARAMS, cudaMemcpyDeviceToHost));
  return MM_OK;
}

mm_status mm_net_train_step(mm_prolong_net* net, const mm_prolong_sample* smp, float lr,
                            double* loss, void* stream) {
  g_err.clear();
  if (!net || !smp || !smp->x_target || !(lr > 0.f)) {
    set_error("a training step needs a network, a sample with x_target and lr > 0");
    return MM_ERR_INVALID_ARG;
  }
  DeviceGuard dg(net->device);
  cudaStream_t s = (cudaStream_t)stream;
  NetSample ns;
  SampleTmp tmp;
  MM_TRY(make_sample(net, smp, ns, tmp, s));
  MM_TRY(net_forward(net->net, ns, nullptr, (const float2*)smp->x_target, s));
  MM_TRY(net_backward(net->net, ns, s));
  MM_TRY(net_adam_step(net->net, lr, s));
  return read_loss(net->net, ns.n, loss, s);
}

mm_status mm_hierarchy_set_net(mm_hierarchy* h, mm_prolong_net* net) {
  g_err.clear();
  if (!h) {
    set_error("hierarchy is NULL");
    return MM_ERR_INVALID_ARG;
  }
  if (!h->subs.empty()) {
    set_error("the learned prolongation applies to single-graph hierarchies");
    return MM_ERR_UNSUPPORTED;
  }
  DeviceGuard dg(h->device);
  if (net) MM_TRY(net_alloc(net->net, h->levels[0].n));
  h->net = net;
  if (h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  return MM_OK;
}

mm_status mm_layout_levels(mm_hierarchy* h, const mm_params* p, float* const* level_x,
                           void* stream) {
  g_err.clear();
  if (!h || !level_x || !h->subs.empty()) {
    set_error("need a single-graph hierarchy and level outputs");
    return MM_ERR_INVALID_ARG;
  }
  DeviceGuard dg(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  mm_params q = p ? *p : h->p;
  MM_TRY(check_params(&q));
  MM_TRY(ensure_trace(h, q));
  if (h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  MM_TRY(build_graph(h, q, false, level_x));
  MM_CK(cudaMemsetAsync(h->lsw, 0, sizeof(int32_t) * 2 * MM_MAX_LEVELS, s));
  MM_CK(cudaGraphLaunch(h->gexec, s));
  MM_CK(cudaStreamSynchronize(s));
  // the recording graph is not kept: the next mm_layout builds its own
  cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
  return tree_error(h, s);
}

mm_status mm_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, const void* B,
                       const float* bias, int32_t relu, float* out_f32, void* out_bf16,
                       void* stream) {
  g_err.clear();
  cudaStream_t s = (cudaStream_t)stream;
  MM_TRY(gemm_setup());
  int* err = nullptr;
  MM_CK(cudaMallocAsync(&err, sizeof(int), s));
  MM_CK(cudaMemsetAsync(err, 0, sizeof(int), s));
  mm_status st = gemm_bf16(A, M, K, B, N, bias, relu, out_bf16, out_f32, err, s);
  int he = 0;
  cudaMemcpyAsync(&he, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(err, s);
  cudaError_t e = cudaStreamSynchronize(s);
  MM_TRY(st);
  MM_CK(e);
  if (he) {
    set_error("tensor-core wait gave up");
    return MM_ERR_TIMEOUT;
  }
  return MM_OK;
}

mm_status mm_gemm_bf16_tn(int32_t n, int32_t R, const void* A, const void* B, float* out,
                          void* stream) {
  g_err.clear();
  if (n < 0 || (R != 16 && R != 128) || !A || !B || !out) {
    set_error("mm_gemm_bf16_tn: need n >= 0, R in {16, 128}, device A, B, out");
    return MM_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    MM_CK(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)R * 64, s));
    MM_CK(cudaStreamSynchronize(s));
    return MM_OK;
  }
  MM_TRY(gemm_setup());
  int* err = nullptr;
  float* part = nullptr;
  MM_CK(cudaMallocAsync(&err, sizeof(int), s));
  MM_CK(cudaMallocAsync(&part, sizeof(float) * (size_t)gemm_tn_parts(n) * R * 64, s));
  MM_CK(cudaMemsetAsync(err, 0, sizeof(int), s));
  mm_status st = gemm_tn_bf16(A, n, R, B, out, part, err, s);
  int he = 0;
  cudaMemcpyAsync(&he, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(part, s);
  cudaFreeAsync(err, s);
  cudaError_t e = cudaStreamSynchronize(s);
  MM_TRY(st);
  MM_CK(e);
  if (he) {
    set_error("tensor-core wait gave up");
    return MM_ERR_TIMEOUT;
  }
  return MM_OK;
}

mm_status mm_net_gemm_profile(int32_t n, int32_t reps, double* ms, void* stream) {
  g_err.clear();
  if (n < 128 || reps < 1 || !ms) {
    set_error("mm_net_gemm_profile: need n >= 128, reps >= 1, ms");
    return MM_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  MM_TRY(gemm_setup());
  const size_t nA = (size_t)n * 128, nB = (size_t)n * 64;
  void *A = nullptr, *W = nullptr, *C = nullptr, *G = nullptr;
  float *out = nullptr, *part = nullptr;
  int* err = nullptr;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  mm_status st = MM_OK;
  auto ck = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == MM_OK) st = cuda_status(e, what, __FILE__, __LINE__);
  };
  ck(cudaMallocAsync(&A, 2 * nA, s), "alloc");
  ck(cudaMallocAsync(&W, 2 * 64 * 128, s), "alloc");
  ck(cudaMallocAsync(&C, 2 * nB, s), "alloc");
  ck(cudaMallocAsync(&G, 2 * nB, s), "alloc");
  ck(cudaMallocAsync(&out, sizeof(float) * 128 * 64, s), "alloc");
  ck(cudaMallocAsync(&part, sizeof(float) * (size_t)gemm_tn_parts(n) * 128 * 64, s), "alloc");
  ck(cudaMallocAsync(&err, sizeof(int), s), "alloc");
  // operand values do not change the work: a constant bit pattern (BF16 1/8)
  if (st == MM_OK) {
    ck(cudaMemsetAsync(A, 0x3e, 2 * nA, s), "memset");
    ck(cudaMemsetAsync(W, 0x3e, 2 * 64 * 128, s), "memset");
    ck(cudaMemsetAsync(G, 0x3e, 2 * nB, s), "memset");
    ck(cudaMemsetAsync(err, 0, sizeof(int), s), "memset");
  }
  for (auto& e : ev) ck(cudaEventCreate(&e), "event");
  float t0 = 0.f, t1 = 0.f;
  if (st == MM_OK) {
    // one warm-up of each, then reps launches of each between events
    st = gemm_bf16(A, n, 128, W, 64, nullptr, 0, C, nullptr, err, s);
    if (st == MM_OK) st = gemm_tn_partials(A, n, 128, G, part, gemm_tn_parts(n), err, s);
    ck(cudaEventRecord(ev[0], s), "record");
    for (int r = 0; r < reps && st == MM_OK; ++r)
      st = gemm_bf16(A, n, 128, W, 64, nullptr, 0, C, nullptr, err, s);
    ck(cudaEventRecord(ev[1], s), "record");
    for (int r = 0; r < reps && st == MM_OK; ++r)
      st = gemm_tn_partials(A, n, 128, G, part, gemm_tn_parts(n), err, s);
    ck(cudaEventRecord(ev[2], s), "record");
    ck(cudaEventSynchronize(ev[2]), "sync");
    ck(cudaEventElapsedTime(&t0, ev[0], ev[1]), "elapsed");
    ck(cudaEventElapsedTime(&t1, ev[1], ev[2]), "elapsed");
  }
  int he = 0;
  if (err) cudaMemcpy(&he, err, sizeof(int), cudaMemcpyDeviceToHost);
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  void* bufs[] = {A, W, C, G, out, part, err};
  for (void* b : bufs)
    if (b) cudaFreeAsync(b, s);
  cudaStreamSynchronize(s);
  MM_TRY(st);
  if (he) {
    set_error("tensor-core wait gave up");
    return MM_ERR_TIMEOUT;
  }
  ms[0] = t0 / reps;
  ms[1] = t1 / reps;
  return MM_OK;
}

mm_status mm_autotune(mm_hierarchy* h, const float* thetas, int32_t n_theta, double max_rel_drift,
                      mm_tune_result* out, void* stream) {
  g_err.clear();
  if (!h) {
    set_error("hierarchy is NULL");
    return MM_ERR_INVALID_ARG;
  }
  DeviceGuard dg(h->device);
  return autotune(h, thetas, n_theta, max_rel_drift, out, (cudaStream_t)stream);
}

mm_status mm_objective(mm_hierarchy* h, int32_t level, const float* x, double alpha,
                       double* stress, double* lnsum, double* M, void* stream) {
  g_err.clear();
  MM_TRY(level_check(h, level));
  if (!x) {
    set_error("x is NULL");
    return MM_ERR_INVALID_ARG;
  }
  DeviceGuard dg(h->device);
  double out[3];
  mm_status cst;
  const float2* xi = x_in_internal(h, level, x, 0, (cudaStream_t)stream, &cst);
  MM_TRY(cst);
  MM_TRY(objective_exact(h->levels[level], xi, alpha, out, (cudaStream_t)stream));
  if (stress) *stress = out[0];
  if (lnsum) *lnsum = out[1];
  if (M) *M = out[2];
  return MM_OK;
}

mm_status mm_objective_bh(mm_hierarchy* h, int32_t level, const float* x, double alpha,
                          float theta, double* stress, double* lnsum, double* M, void* stream) {
  g_err.clear();
  MM_TRY(level_check(h, level));
  if (!x || !(theta >= 0.f)) {
    set_error("x is NULL or theta < 0");
    return MM_ERR_INVALID_ARG;
  }
  DeviceGuard dg(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  mm_status cst;
  const float2* xi = x_in_internal(h, level, x, 0, s, &cst);
  MM_TRY(cst);
  const Level& L = h->levels[level];
  float* phi = nullptr;
  MM_CK(cudaMallocAsync(&phi, sizeof(float) * (size_t)std::max(L.n, 1), s));
  XSel xs{xi, xi, h->zero};
  // the group walk's decisions (leaf buckets, all 32 points of a task vote)
  mm_status st = bh_build(xs, L.n, theta, leaf_of(h->p), h->tree, s, nullptr, true, true);
  if (st == MM_OK) st = bh_potential(L.n, h->tree, h->F, phi, L.walk_warps, s);
  double out[3] = {0, 0, 0};
  if (st == MM_OK) st = objective_from_phi(L, xi, phi, alpha, out, s);
  cudaFreeAsync(phi, s);
  MM_TRY(st);
  MM_TRY(tree_error(h, s));
  if (stress) *stress = out[0];
  if (lnsum) *lnsum = out[1];
  if (M) *M = out[2];
  return MM_OK;
}

mm_status mm_khop(int32_t n, const int64_t* row_ptr, const int32_t* col, const float* edge_len,
                  const float* node_c, int32_t k, int64_t* s_ptr, int64_t* nnz_S, int32_t* s_col,
                  float* s_d, float* rho, void* stream) {
  g_err.clear();
  if (n < 1 || !row_ptr || !s_ptr || !nnz_S || (s_col && (!s_d || !rho))) {
    set_error("invalid arguments");
    return MM_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* rp = nullptr;
  int32_t* sp = nullptr;
  SEnt* S = nullptr;
  float* r = nullptr;
  int64_t nnz = 0;
  MM_CK(cudaMalloc(&rp, sizeof(int32_t) * (size_t)(n + 1)));
  rp_to_i32<<<ceil_div(n + 1, 256), 256, 0, s>>>(n, row_ptr, rp);
  mm_status st = build_khop(n, rp, col, edge_len, node_c, k, &sp, &S, &r, &nnz, s);
  if (st == MM_OK) {
    i32_to_i64<<<ceil_div(n + 1, 256), 256, 0, s>>>(n + 1, sp, s_ptr);
    *nnz_S = nnz;
    if (s_col) {
      if (nnz) split_sent<<<ceil_div(nnz, 256), 256, 0, s>>>(nnz, S, s_col, s_d);
      cudaMemcpyAsync(rho, r, sizeof(float) * n, cudaMemcpyDeviceToDevice, s);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "mm_khop", __FILE__, __LINE__);
  }
  cudaFree(rp);
  if (sp) cudaFree(sp);
  if (S) cudaFree(S);
  if (r) cudaFree(r);
  return st;
}

mm_status mm_cluster(int32_t n, const int64_t* row_ptr, const int32_t* col, const float* omega,
                     const float* node_c, float U, int32_t rounds, uint64_t seed, int32_t level,
                     int32_t* labels_out, void* stream) {
  g_err.clear();
  if (n < 1 || !row_ptr || !node_c || !labels_out || rounds < 0) {
    set_error("invalid arguments");
    return MM_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* rp = nullptr;
  MM_CK(cudaMalloc(&rp, sizeof(int32_t) * (size_t)(n + 1)));
  rp_to_i32<<<ceil_div(n + 1, 256), 256, 0, s>>>(n, row_ptr, rp);
  mm_status st = cluster_lp(n, rp, col, omega, node_c, U, rounds, seed, level, labels_out, s);
  cudaStreamSynchronize(s);
  cudaFree(rp);
  return st;
}

mm_status mm_contract(int32_t n, const int64_t* row_ptr, const int32_t* col, const float* omega,
                      const float* node_c, const int32_t* labels, int32_t* map, float* c_out,
                      int64_t* crow_ptr, int32_t* ccol, float* comega, int32_t* n_coarse,
                      int64_t* nnz_coarse, void* stream) {
  g_err.clear();
  if (n < 1 || !row_ptr || !node_c || !labels || !map || !c_out || !crow_ptr || !ccol ||
      !comega || !n_coarse || !nnz_coarse) {
    set_error("invalid arguments");
    return MM_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* rp = nullptr;
  MM_CK(cudaMalloc(&rp, sizeof(int32_t) * (size_t)(n + 1)));
  rp_to_i32<<<ceil_div(n + 1, 256), 256, 0, s>>>(n, row_ptr, rp);
  Level out;
  mm_status st = contract(n, rp, col, omega, node_c, labels, map, out, s);
  if (st == MM_OK) {
    *n_coarse = out.n;
    *nnz_coarse = out.nnzE;
    cudaMemcpyAsync(c_out, out.c, sizeof(float) * out.n, cudaMemcpyDeviceToDevice, s);
    i32_to_i64<<<ceil_div(out.n + 1, 256), 256, 0, s>>>(out.n + 1, out.rp, crow_ptr);
    if (out.nnzE) {
      cudaMemcpyAsync(ccol, out.col, sizeof(int32_t) * out.nnzE, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(comega, out.omega, sizeof(float) * out.nnzE, cudaMemcpyDeviceToDevice, s);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "mm_contract", __FILE__, __LINE__);
  }
  free_level(out);
  cudaFree(rp);
  return st;
}

mm_status mm_prolong(int32_t n_fine, const int32_t* map, const float* x_coarse,
                     const float* c_coarse, uint64_t seed, int32_t level, float* x_fine,
                     void* stream) {
  g_err.clear();
  if (n_fine < 0 || (n_fine > 0 && (!map || !x_coarse || !c_coarse || !x_fine))) {
    set_error("invalid arguments");
    return MM_ERR_INVALID_ARG;
  }
  int32_t* zero = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  MM_CK(cudaMalloc(&zero, sizeof(int32_t)));
  cudaMemsetAsync(zero, 0, sizeof(int32_t), s);
  XSel xc{(const float2*)x_coarse, (const float2*)x_coarse, zero};
  mm_status st = prolong(n_fine, map, xc, c_coarse, seed, level, (float2*)x_fine, s);
  cudaStreamSynchronize(s);
  cudaFree(zero);
  return st;
}

mm_status mm_layout_host(int32_t n, const int64_t* row_ptr, const int32_t* col,
                         const float* edge_len, const mm_params* p, float* x_out,
                         mm_layout_stats* stats, void* stream) {
  g_err.clear();
  if (n < 1 || !row_ptr || !x_out) {
    set_error("invalid arguments");
    return MM_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nnz = row_ptr[n];
  int64_t* drp = nullptr;
  int32_t* dcol = nullptr;
  float* dlen = nullptr;
  float* dx = nullptr;
  mm_hierarchy* h = nullptr;
  mm_status st = MM_OK;
  cudaError_t e = cudaMalloc(&drp, sizeof(int64_t) * (size_t)(n + 1));
  if (e == cudaSuccess) e = cudaMalloc(&dcol, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1));
  if (e == cudaSuccess && edge_len)
    e = cudaMalloc(&dlen, sizeof(float) * (size_t)std::max<int64_t>(nnz, 1));
  if (e == cudaSuccess) e = cudaMalloc(&dx, sizeof(float2) * (size_t)n);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(drp, row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nnz)
    e = cudaMemcpyAsync(dcol, col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && edge_len && nnz)
    e = cudaMemcpyAsync(dlen, edge_len, sizeof(float) * nnz, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) st = cuda_status(e, "mm_layout_host upload", __FILE__, __LINE__);
  if (st == MM_OK) {
    mm_graph g;
    memset(&g, 0, sizeof(g));
    g.n = n;
    g.nnz = nnz;
    g.row_ptr = drp;
    g.col = dcol;
    g.edge_len = dlen;
    g.num_graphs = 1;
    st = mm_build_hierarchy(&g, p, stream, &h);
  }
  if (st == MM_OK) st = mm_layout(h, p, nullptr, dx, stats, stream);
  if (st == MM_OK) {
    e = cudaMemcpyAsync(x_out, dx, sizeof(float2) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "mm_layout_host download", __FILE__, __LINE__);
  }
  std::string keep = g_err;
  mm_free_hierarchy(h);
  cudaFree(drp);
  cudaFree(dcol);
  if (dlen) cudaFree(dlen);
  cudaFree(dx);
  g_err = keep;
  return st;
}

}  // extern "C"
