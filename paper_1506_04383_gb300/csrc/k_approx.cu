// The hierarchy approximation of the entropy sum, Eq. 3 (Sec. 3.2, "Faster
// Local Improvement"; MulMent_h):
//
//   F_u = sum_{v != u, M(v) = M(u)} r(u,v)
//       + sum_{v' != M(u)} nu(v') (x_u - x'_{v'}) / |x_u - x'_{v'}|^2
//
// M maps the current level's vertices to the level h levels down (or the
// coarsest), nu(v') counts the current-level vertices mapped to v', and
// x'_{v'} is their midpoint, refreshed from the current positions before
// every sweep.  The sweep then subtracts the exact r-values over S, as for
// the other repulsion modes (the last term of Eq. 3).
//
// Per level, once (build): the composed map M and the members of every
// coarse vertex, sorted by vertex id (a stable radix sort of (M(v), v)),
// with segment offsets.  Per sweep: one warp per coarse vertex sums its
// members' positions (fixed order), then four threads per vertex (in member
// order) add the far sum over all coarse midpoints and the exact near sum
// over its own group, both staged through shared memory in tiles (FP32-pipe
// bound: n (n' - 1) far plus sum_c m_c (m_c - 1) near pair terms).
#include <cuda_runtime.h>

#include <algorithm>

#include "mm_internal.cuh"

namespace mm {

namespace {

constexpr int kApproxThreads = 256;

__global__ void compose_map_kernel(int n, int32_t* hmap, const int32_t* __restrict__ next) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) hmap[i] = next[hmap[i]];
}

__global__ void iota_keys_kernel(int n, const int32_t* __restrict__ hmap, uint32_t* keys,
                                 int32_t* vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    keys[i] = (uint32_t)hmap[i];
    vals[i] = i;
  }
}

// moff[c] = first position of coarse vertex c in the sorted keys (empty
// segments get the next segment's start); moff[nt] = n.
__global__ void segment_offsets_kernel(int n, const uint32_t* __restrict__ keys, int nt,
                                       int32_t* moff) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  const int prev = i > 0 ? (int)keys[i - 1] : -1;
  const int cur = i < n ? (int)keys[i] : nt;
  for (int c = prev + 1; c <= cur; ++c) moff[c] = i;
}

// One warp per coarse vertex: midpoint of its members (lane-strided sums
// added in a fixed shuffle tree) and its member count nu.
__global__ void midpoints_kernel(int nt, const int32_t* __restrict__ moff,
                                 const int32_t* __restrict__ members, XSel xs, float4* xc) {
  const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= nt) return;
  const float2* x = xs.cur();
  const int b = moff[warp], e = moff[warp + 1];
  float sx = 0.f, sy = 0.f;
  for (int j = b + lane; j < e; j += 32) {
    const float2 p = x[members[j]];
    sx += p.x;
    sy += p.y;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
  }
  if (lane == 0) {
    const float nu = (float)(e - b);
    xc[warp] = nu > 0.f ? make_float4(sx / nu, sy / nu, nu, 0.f)
                        : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Groups of consecutive members a block stages through shared memory for
// the near sums (more than this many distinct groups in one block -- small
// groups -- and each thread walks its own group directly).
constexpr int kStagedGroups = 8;
// Threads per vertex: the vertex's far and near terms are dealt round robin
// to kSplit lanes and added back with shuffles in a fixed order, so a level
// of n vertices runs kSplit * n threads (a single thread per vertex leaves
// most warp slots empty on levels of ~10^5 vertices).
constexpr int kSplit = 4;
constexpr int kVertsPerBlock = kApproxThreads / kSplit;

// kSplit threads per vertex, vertices taken in member order (u = members[i],
// so a block covers whole groups or runs of them).  Far sum: every other
// coarse midpoint, tiles of (x', nu) in shared memory, u's own representative
// skipped.  Near sum: the exact r-values over u's own group, staged in tiles
// of positions shared by the block's threads of that group (the point
// itself and coincident points have |x_u - x_v| = 0 and add nothing).
__global__ void __launch_bounds__(kApproxThreads) approx_force_kernel(
    int n, XSel xs, const int32_t* __restrict__ hmap, const int32_t* __restrict__ moff,
    const int32_t* __restrict__ members, int nt, const float4* __restrict__ xc,
    float2* __restrict__ F) {
  __shared__ float4 tile[kApproxThreads];
  __shared__ float2 near[kApproxThreads];
  const float2* x = xs.cur();
  const int sub = threadIdx.x % kSplit;
  const int i0 = blockIdx.x * kVertsPerBlock;
  const int i = i0 + threadIdx.x / kSplit;
  const bool live = i < n;
  const int u = live ? members[i] : 0;
  const float2 xu = live ? x[u] : make_float2(0.f, 0.f);
  const int cu = live ? hmap[u] : -1;
  float fx = 0.f, fy = 0.f;
  auto term = [&](float2 p, float wgt, bool on) {
    const float dx = xu.x - p.x, dy = xu.y - p.y;
    const float q = fmaf(dx, dx, dy * dy);
    const float s = (on && q > 0.f) ? __fdividef(wgt, q) : 0.f;
    fx = fmaf(s, dx, fx);
    fy = fmaf(s, dy, fy);
  };
  for (int t0 = 0; t0 < nt; t0 += kApproxThreads) {
    const int cnt = min(kApproxThreads, nt - t0);
    if (threadIdx.x < cnt) tile[threadIdx.x] = xc[t0 + threadIdx.x];
    __syncthreads();
#pragma unroll 4
    for (int k = sub; k < cnt; k += kSplit) {
      const float4 c = tile[k];
      // the own representative carries no far term; coincident: r = 0
      term(make_float2(c.x, c.y), c.z, t0 + k != cu);
    }
    __syncthreads();
  }
  // groups present in this block (members are sorted by group)
  const int c0 = hmap[members[i0]];
  const int c1 = hmap[members[min(n - 1, i0 + kVertsPerBlock - 1)]];
  if (c1 - c0 < kStagedGroups) {
    for (int c = c0; c <= c1; ++c) {
      const int b = moff[c], e = moff[c + 1];
      for (int t0 = b; t0 < e; t0 += kApproxThreads) {
        const int cnt = min(kApproxThreads, e - t0);
        if (threadIdx.x < cnt) near[threadIdx.x] = x[members[t0 + threadIdx.x]];
        __syncthreads();
        if (cu == c) {
#pragma unroll 4
          for (int k = sub; k < cnt; k += kSplit) term(near[k], 1.f, true);
        }
        __syncthreads();
      }
    }
  } else if (live) {
    for (int j = moff[cu] + sub; j < moff[cu + 1]; j += kSplit) term(x[members[j]], 1.f, true);
  }
  // the kSplit partial sums of a vertex sit in consecutive lanes
#pragma unroll
  for (int o = 1; o < kSplit; o <<= 1) {
    fx += __shfl_xor_sync(0xffffffffu, fx, o);
    fy += __shfl_xor_sync(0xffffffffu, fy, o);
  }
  if (live && sub == 0) F[u] = make_float2(fx, fy);
}

}  // namespace

mm_status approx_setup(Level& L, const std::vector<Level>& levels, int level, int h,
                       cudaStream_t s) {
  const int top = (int)levels.size() - 1;
  const int t = std::min(level + h, top);
  if (t <= level || L.n < 1) return MM_OK;
  L.nt = levels[t].n;
  MM_CK(cudaMallocAsync(&L.hmap, sizeof(int32_t) * (size_t)L.n, s));
  MM_CK(cudaMallocAsync(&L.members, sizeof(int32_t) * (size_t)L.n, s));
  MM_CK(cudaMallocAsync(&L.moff, sizeof(int32_t) * ((size_t)L.nt + 1), s));
  MM_CK(cudaMemcpyAsync(L.hmap, L.map, sizeof(int32_t) * (size_t)L.n, cudaMemcpyDeviceToDevice,
                        s));
  for (int j = level + 1; j < t; ++j)
    compose_map_kernel<<<ceil_div(L.n, 256), 256, 0, s>>>(L.n, L.hmap, levels[j].map);
  uint32_t *k0 = nullptr, *k1 = nullptr;
  int32_t* v1 = nullptr;
  MM_CK(cudaMallocAsync(&k0, sizeof(uint32_t) * (size_t)L.n, s));
  MM_CK(cudaMallocAsync(&k1, sizeof(uint32_t) * (size_t)L.n, s));
  MM_CK(cudaMallocAsync(&v1, sizeof(int32_t) * (size_t)L.n, s));
  iota_keys_kernel<<<ceil_div(L.n, 256), 256, 0, s>>>(L.n, L.hmap, k0, L.members);
  int bits = 1;
  while (bits < 32 && (1ll << bits) < (int64_t)L.nt) ++bits;
  SortWS ws;
  mm_status st = sort_ws_alloc(ws, L.n);
  uint32_t* keys = nullptr;
  int32_t* vals = nullptr;
  auto check = [&](cudaError_t e, const char* what) {
    if (st == MM_OK && e != cudaSuccess) st = cuda_status(e, what, __FILE__, __LINE__);
  };
  if (st == MM_OK)
    st = radix_sort_u32(k0, k1, L.members, v1, L.n, 0, bits, ws, s, &keys, &vals);
  if (st == MM_OK && vals != L.members)
    check(cudaMemcpyAsync(L.members, vals, sizeof(int32_t) * (size_t)L.n,
                          cudaMemcpyDeviceToDevice, s),
          "cudaMemcpyAsync(members)");
  if (st == MM_OK) {
    segment_offsets_kernel<<<ceil_div(L.n + 1, 256), 256, 0, s>>>(L.n, keys, L.nt, L.moff);
    check(cudaGetLastError(), "segment_offsets_kernel");
  }
  // the sort workspace is freed synchronously: finish the work that uses it
  check(cudaStreamSynchronize(s), "cudaStreamSynchronize(approx_setup)");
  sort_ws_free(ws);
  cudaFreeAsync(k0, s);
  cudaFreeAsync(k1, s);
  cudaFreeAsync(v1, s);
  return st;
}

mm_status approx_repulsion(const Level& L, XSel x, float4* xc, float2* F, cudaStream_t s) {
  if (L.n <= 0) return MM_OK;
  if (!L.hmap) {
    set_error("level has no approximation map (approx_levels = 0 or coarsest level)");
    return MM_ERR_INVALID_ARG;
  }
  midpoints_kernel<<<ceil_div((int64_t)L.nt * 32, 256), 256, 0, s>>>(L.nt, L.moff, L.members, x,
                                                                      xc);
  approx_force_kernel<<<ceil_div(L.n, kVertsPerBlock), kApproxThreads, 0, s>>>(
      L.n, x, L.hmap, L.moff, L.members, L.nt, xc, F);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

}  // namespace mm
