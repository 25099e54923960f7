// Barnes-Hut quadtree rebuilt on the device every sweep, and its traversal.
//
// The long-range entropy term of Eq. 2 needs F_u = sum_{v != u} r(u,v) for
// every vertex; Barnes and Hut (cited in Sec. 2.2 and Sec. 2.3) approximate
// it with a quadtree: a cell of side w whose centroid is at distance D from u
// (and which does not contain u) is accepted when w / D < theta and then
// contributes count * r(u, centroid); leaves are summed exactly.
//
// GB300 design:
//   * cells are Morton-prefix cells of 16-bit-per-axis keys over the bounding
//     square, so the tree is defined by one radix sort of 32-bit keys;
//   * the binary radix tree (Karras 2012) over the sorted keys is built in
//     one pass; a binary node is a quadtree cell when its common-prefix
//     length first reaches a new even bit count ("transparent" nodes that
//     only split a quadrant pair are skipped at record time), duplicate keys
//     form bucket leaves at depth 16;
//   * centroids come from one bottom-up pass with epoch-stamped visit flags
//     (no reset kernel), which also writes 32-byte node records
//     (centroid, (w/theta)^2, count | first child, escape, point range);
//   * the walk is warp-synchronous and stackless: the warp follows
//     first-child / escape links in pre-order, each lane keeps the escape
//     node of the last cell it accepted and is idle until the warp reaches
//     it.  Every lane applies exactly its own acceptance test, so the result
//     equals a per-vertex Barnes-Hut walk of the same quadtree, while node
//     loads are warp-uniform (one broadcast transaction per visited node).
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>

#include "mm_internal.cuh"

namespace mm {

namespace {

constexpr int kBBoxThreads = 256;
constexpr int kBBoxMaxBlocks = 2 * kSMs;
constexpr int kNone = -2;  // lane is active

__device__ __forceinline__ uint32_t spread16(uint32_t v) {
  v &= 0xffffu;
  v = (v | (v << 8)) & 0x00ff00ffu;
  v = (v | (v << 4)) & 0x0f0f0f0fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Bounding square of the layout.  The last block to finish reduces the
// per-block partials (fixed order) and writes root = (min x, min y, side,
// 2^16 / side); it also bumps the epoch (ticket[1]) used by the bottom-up
// pass.
__global__ void __launch_bounds__(kBBoxThreads) bbox_kernel(XSel xs, int n, float4* partials,
                                                            unsigned* ticket, float4* root) {
  const float2* x = xs.cur();
  float mnx = CUDART_INF_F, mny = CUDART_INF_F, mxx = -CUDART_INF_F, mxy = -CUDART_INF_F;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 p = x[i];
    mnx = fminf(mnx, p.x); mny = fminf(mny, p.y);
    mxx = fmaxf(mxx, p.x); mxy = fmaxf(mxy, p.y);
  }
  __shared__ float4 sh[kBBoxThreads / 32];
  __shared__ bool last;
  mnx = warp_min(mnx); mny = warp_min(mny); mxx = warp_max(mxx); mxy = warp_max(mxy);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = make_float4(mnx, mny, mxx, mxy);
  __syncthreads();
  if (threadIdx.x == 0) {
    float4 r = sh[0];
    for (int w = 1; w < kBBoxThreads / 32; ++w) {
      r.x = fminf(r.x, sh[w].x); r.y = fminf(r.y, sh[w].y);
      r.z = fmaxf(r.z, sh[w].z); r.w = fmaxf(r.w, sh[w].w);
    }
    partials[blockIdx.x] = r;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  if (threadIdx.x == 0) {
    float4 r = __ldcg(&partials[0]);
    for (int b = 1; b < (int)gridDim.x; ++b) {
      const float4 q = __ldcg(&partials[b]);
      r.x = fminf(r.x, q.x); r.y = fminf(r.y, q.y);
      r.z = fmaxf(r.z, q.z); r.w = fmaxf(r.w, q.w);
    }
    const float side = fmaxf(r.z - r.x, r.w - r.y);
    const float scale = side > 0.f ? 65536.0f / side : 0.f;
    *root = make_float4(r.x, r.y, side, scale);
    ticket[0] = 0u;
    ticket[1] += 1u;
  }
}

__global__ void morton_kernel(XSel xs, int n, const float4* __restrict__ root,
                              uint32_t* __restrict__ keys, int32_t* __restrict__ vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 p = xs.cur()[i];
  const float4 r = *root;
  const float fx = (p.x - r.x) * r.w, fy = (p.y - r.y) * r.w;
  // clamp in float first: the conversion of out-of-range values is undefined
  const uint32_t ix = (uint32_t)fminf(fmaxf(fx, 0.f), 65535.f);
  const uint32_t iy = (uint32_t)fminf(fmaxf(fy, 0.f), 65535.f);
  keys[i] = (spread16(ix) << 1) | spread16(iy);
  vals[i] = i;
}

// Common prefix length of sorted keys i and j; equal keys are told apart by
// their index (values > 32), out-of-range j gives -1.
__device__ __forceinline__ int prefix_len(const uint32_t* __restrict__ k, int n, int i,
                                          int64_t j) {
  if (j < 0 || j >= n) return -1;
  const uint32_t a = k[i], b = k[(int)j];
  if (a != b) return __clz(a ^ b);
  return 32 + __clz((uint32_t)i ^ (uint32_t)j);
}

// Karras (2012) binary radix tree: internal node i covers [lo, hi]; its split
// g separates [lo, g] and [g+1, hi].  Node ids: internal 0..n-2 (root 0),
// leaf j -> n-1+j.
__global__ void karras_kernel(const uint32_t* __restrict__ k, int n, int32_t* lo, int32_t* hi,
                              int32_t* left, int32_t* right, int32_t* delta, int32_t* owner,
                              int32_t* parent) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  const int dr = prefix_len(k, n, i, (int64_t)i + 1);
  const int dl = prefix_len(k, n, i, (int64_t)i - 1);
  const int d = dr > dl ? 1 : -1;
  const int dmin = d > 0 ? dl : dr;
  int64_t lmax = 2;
  while (prefix_len(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int64_t l = 0;
  for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
    if (prefix_len(k, n, i, i + (l + t) * d) > dmin) l += t;
  const int j = (int)(i + l * d);
  const int dnode = prefix_len(k, n, i, j);
  int64_t s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (prefix_len(k, n, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  const int g = (int)(i + s * d + (d < 0 ? -1 : 0));
  const int a = min(i, j), b = max(i, j);
  const int L = (a == g) ? (n - 1 + g) : g;
  const int R = (b == g + 1) ? (n - 1 + g + 1) : g + 1;
  lo[i] = a; hi[i] = b; left[i] = L; right[i] = R; delta[i] = dnode; owner[g] = i;
  parent[L] = i; parent[R] = i;
  if (i == 0) parent[0] = -1;
}

struct TreeView {
  int n;
  const int32_t* lo; const int32_t* hi; const int32_t* left; const int32_t* right;
  const int32_t* delta; const int32_t* owner; const int32_t* parent;
};

// A transparent internal node (same quadtree depth as its parent) is
// replaced by its left child, which is always a visible node.
__device__ __forceinline__ int resolve(const TreeView& t, int x) {
  if (x >= t.n - 1 || x == 0) return x;
  const int dx = t.delta[x];
  if (dx >= 32) return x;
  const int dp = t.delta[t.parent[x]];
  return (dp >> 1) == (dx >> 1) ? t.left[x] : x;
}

// Next node in pre-order after the subtree whose last point is h.
__device__ __forceinline__ int escape_of(const TreeView& t, int h) {
  if (h >= t.n - 1) return -1;
  return resolve(t, t.right[t.owner[h]]);
}

__device__ void write_record(const TreeView& t, int id, double2 sum, float side, float theta,
                             float4* nodeA, int4* nodeB) {
  const int n = t.n;
  if (id >= n - 1) {  // leaf j
    const int j = id - (n - 1);
    if (n > 1 && t.delta[t.parent[id]] >= 32) return;  // inside a bucket
    nodeA[id] = make_float4((float)sum.x, (float)sum.y, 0.f, 1.f);
    nodeB[id] = make_int4(-1, escape_of(t, j), j, j + 1);
    return;
  }
  const int dd = t.delta[id];
  const int dp = id == 0 ? -1 : t.delta[t.parent[id]];
  int depth, first;
  if (dd >= 32) {  // duplicate keys: bucket leaf at the deepest level
    if (dp >= 32) return;
    depth = kKeyBits;
    first = -1;
  } else {
    if (dp >= 0 && (dp >> 1) == (dd >> 1)) return;  // transparent
    depth = dd >> 1;
    first = resolve(t, t.left[id]);
  }
  const int a = t.lo[id], b = t.hi[id];
  const double cnt = (double)(b - a + 1);
  const float w = ldexpf(side, -depth);
  const float rc = theta > 0.f ? (w / theta) * (w / theta) : CUDART_INF_F;
  nodeA[id] = make_float4((float)(sum.x / cnt), (float)(sum.y / cnt), rc, (float)cnt);
  nodeB[id] = make_int4(first, escape_of(t, b), a, b + 1);
}

// One thread per leaf: writes the sorted positions and leaf records, then
// climbs; the second thread to reach an internal node sums its children and
// writes its record (the first one stops).
__global__ void bottomup_kernel(XSel xs, const int32_t* __restrict__ vals, TreeView t,
                                uint32_t* visit, double2* sums, float4* nodeA, int4* nodeB,
                                float2* xsorted, const float4* __restrict__ root, float theta,
                                const unsigned* ticket) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = t.n;
  if (j >= n) return;
  const float2 p = xs.cur()[vals[j]];
  xsorted[j] = p;
  const float side = root->z;
  const uint32_t epoch = ticket[1];
  int cur = n - 1 + j;
  double2 s = make_double2(p.x, p.y);
  sums[cur] = s;
  write_record(t, cur, s, side, theta, nodeA, nodeB);
  if (n == 1) return;
  while (true) {
    const int par = t.parent[cur];
    if (par < 0) break;
    __threadfence();
    if (atomicExch(&visit[par], epoch) != epoch) break;  // first arrival
    const int L = t.left[par], R = t.right[par];
    const double2 a = __ldcg(&sums[L]);
    const double2 b = __ldcg(&sums[R]);
    s = make_double2(a.x + b.x, a.y + b.y);
    sums[par] = s;
    write_record(t, par, s, side, theta, nodeA, nodeB);
    cur = par;
  }
}

// Guards: node ids must stay in [0, 2n-1) and a walk visits each node at
// most once, so more than 2n visits or an out-of-range id means a broken
// tree; the warp then stops and raises err[0] instead of faulting or
// looping.
template <bool kCount>
__global__ void traverse_kernel(int n, const float2* __restrict__ xs,
                                const int32_t* __restrict__ vals,
                                const float4* __restrict__ nodeA,
                                const int4* __restrict__ nodeB, float2* __restrict__ F,
                                unsigned long long* counters, int* err) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (wid * 32 >= n) return;
  const int pos = (int)(wid * 32 + lane);
  const bool valid = pos < n;
  const float2 xu = valid ? xs[pos] : make_float2(0.f, 0.f);
  int wait = valid ? kNone : -1;
  int cur = n > 1 ? 0 : -1;
  float fx = 0.f, fy = 0.f;
  unsigned visits = 0, inter = 0;
  const int nodes = 2 * n - 1;
  int budget = 2 * n + 2;
  while (cur >= 0) {
    if (cur >= nodes || --budget < 0) {
      if (lane == 0) atomicOr(err, 1);
      break;
    }
    const float4 A = __ldg(&nodeA[cur]);
    const int4 B = __ldg(&nodeB[cur]);
    if (wait == cur) wait = kNone;
    bool desc = false;
    if (wait == kNone) {
      const float dx = xu.x - A.x, dy = xu.y - A.y;
      const float q = fmaf(dx, dx, dy * dy);
      const bool inside = pos >= B.z && pos < B.w;
      if (!inside && q > A.z) {
        const float sc = __fdividef(A.w, q);
        fx = fmaf(sc, dx, fx);
        fy = fmaf(sc, dy, fy);
        wait = B.y;
        if (kCount) ++inter;
      } else if (B.x < 0) {
        const int pb = max(B.z, 0), pe = min(B.w, n);
        for (int p = pb; p < pe; ++p) {
          if (p == pos) continue;
          const float2 xv = xs[p];
          const float ex = xu.x - xv.x, ey = xu.y - xv.y;
          const float eq = fmaf(ex, ex, ey * ey);
          if (eq > 0.f) {
            const float inv = __fdividef(1.f, eq);
            fx = fmaf(inv, ex, fx);
            fy = fmaf(inv, ey, fy);
          }
          if (kCount) ++inter;
        }
        wait = B.y;
      } else {
        desc = true;
      }
    }
    if (kCount) ++visits;
    cur = __any_sync(0xffffffffu, desc) ? B.x : B.y;
  }
  if (valid) F[vals[pos]] = make_float2(fx, fy);
  if (kCount) {
    // counters[0] = warp node visits, counters[1] = lane interactions
    unsigned tot = inter;
#pragma unroll
    for (int o = 16; o; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0) {
      atomicAdd(&counters[0], (unsigned long long)visits);
      atomicAdd(&counters[1], (unsigned long long)tot);
    }
  }
}

constexpr int kExactThreads = 256;

__global__ void __launch_bounds__(kExactThreads) exact_kernel(XSel xs, int n, float2* F) {
  __shared__ float2 tile[kExactThreads];
  const float2* x = xs.cur();
  const int u = blockIdx.x * kExactThreads + threadIdx.x;
  const float2 xu = u < n ? x[u] : make_float2(0.f, 0.f);
  float fx = 0.f, fy = 0.f;
  for (int t0 = 0; t0 < n; t0 += kExactThreads) {
    const int cnt = min(kExactThreads, n - t0);
    if (threadIdx.x < cnt) tile[threadIdx.x] = x[t0 + threadIdx.x];
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < cnt; ++k) {
      const float dx = xu.x - tile[k].x, dy = xu.y - tile[k].y;
      const float q = fmaf(dx, dx, dy * dy);
      const float inv = q > 0.f ? __fdividef(1.f, q) : 0.f;
      fx = fmaf(inv, dx, fx);
      fy = fmaf(inv, dy, fy);
    }
    __syncthreads();
  }
  if (u < n) F[u] = make_float2(fx, fy);
}

}  // namespace

mm_status tree_ws_alloc(TreeWS& ws, int64_t n) {
  const size_t N = (size_t)(n > 1 ? n : 2);
  ws.cap = n;
  MM_CK(cudaMalloc(&ws.keys[0], sizeof(uint32_t) * N));
  MM_CK(cudaMalloc(&ws.keys[1], sizeof(uint32_t) * N));
  MM_CK(cudaMalloc(&ws.vals[0], sizeof(int32_t) * N));
  MM_CK(cudaMalloc(&ws.vals[1], sizeof(int32_t) * N));
  MM_CK(cudaMalloc(&ws.xs, sizeof(float2) * N));
  MM_CK(cudaMalloc(&ws.lo, sizeof(int32_t) * N));
  MM_CK(cudaMalloc(&ws.hi, sizeof(int32_t) * N));
  MM_CK(cudaMalloc(&ws.left, sizeof(int32_t) * N));
  MM_CK(cudaMalloc(&ws.right, sizeof(int32_t) * N));
  MM_CK(cudaMalloc(&ws.delta, sizeof(int32_t) * N));
  MM_CK(cudaMalloc(&ws.owner, sizeof(int32_t) * N));
  MM_CK(cudaMalloc(&ws.parent, sizeof(int32_t) * 2 * N));
  MM_CK(cudaMalloc(&ws.visit, sizeof(uint32_t) * N));
  MM_CK(cudaMemset(ws.visit, 0, sizeof(uint32_t) * N));
  MM_CK(cudaMalloc(&ws.sums, sizeof(double2) * 2 * N));
  MM_CK(cudaMalloc(&ws.nodeA, sizeof(float4) * 2 * N));
  MM_CK(cudaMalloc(&ws.nodeB, sizeof(int4) * 2 * N));
  MM_CK(cudaMalloc(&ws.partials, sizeof(float4) * kBBoxMaxBlocks));
  MM_CK(cudaMalloc(&ws.root, sizeof(float4)));
  MM_CK(cudaMalloc(&ws.ticket, 2 * sizeof(unsigned)));
  MM_CK(cudaMemset(ws.ticket, 0, 2 * sizeof(unsigned)));
  MM_CK(cudaMalloc(&ws.err, sizeof(int)));
  MM_CK(cudaMemset(ws.err, 0, sizeof(int)));
  // unwritten records read as leaves whose escape ends the walk
  MM_CK(cudaMemset(ws.nodeB, 0xff, sizeof(int4) * 2 * N));
  MM_TRY(sort_ws_alloc(ws.sort, N));
  return MM_OK;
}

void tree_ws_free(TreeWS& ws) {
  void* ptrs[] = {ws.keys[0], ws.keys[1], ws.vals[0], ws.vals[1], ws.xs, ws.lo, ws.hi,
                  ws.left, ws.right, ws.delta, ws.owner, ws.parent, ws.visit, ws.sums,
                  ws.nodeA, ws.nodeB, ws.partials, ws.root, ws.ticket, ws.err};
  for (void* p : ptrs) cudaFree(p);
  sort_ws_free(ws.sort);
  ws = TreeWS();
}

mm_status bh_build(XSel x, int n, float theta, TreeWS& ws, cudaStream_t s, cudaEvent_t* ev) {
  if (n <= 0) return MM_OK;
  if (n > ws.cap) {
    set_error("tree workspace holds %lld vertices, level has %d", (long long)ws.cap, n);
    return MM_ERR_INVALID_ARG;
  }
  const int bb = std::min(kBBoxMaxBlocks, ceil_div(n, kBBoxThreads));
  auto mark = [&](int i) {
    if (ev) cudaEventRecord(ev[i], s);
  };
  mark(0);
  bbox_kernel<<<bb, kBBoxThreads, 0, s>>>(x, n, ws.partials, ws.ticket, ws.root);
  mark(1);
  morton_kernel<<<ceil_div(n, 256), 256, 0, s>>>(x, n, ws.root, ws.keys[0], ws.vals[0]);
  mark(2);
  uint32_t* keys;
  int32_t* vals;
  MM_TRY(radix_sort_u32(ws.keys[0], ws.keys[1], ws.vals[0], ws.vals[1], n, 0, 32, ws.sort, s,
                        &keys, &vals));
  mark(3);
  // 4 passes: the result is back in buffer 0
  if (n > 1) karras_kernel<<<ceil_div(n - 1, 256), 256, 0, s>>>(keys, n, ws.lo, ws.hi, ws.left,
                                                                 ws.right, ws.delta, ws.owner,
                                                                 ws.parent);
  mark(4);
  TreeView tv{n, ws.lo, ws.hi, ws.left, ws.right, ws.delta, ws.owner, ws.parent};
  bottomup_kernel<<<ceil_div(n, 256), 256, 0, s>>>(x, vals, tv, ws.visit, ws.sums, ws.nodeA,
                                                   ws.nodeB, ws.xs, ws.root, theta, ws.ticket);
  mark(5);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

mm_status bh_traverse(int n, const TreeWS& ws, float2* F, int warps_per_block,
                      unsigned long long* counters, cudaStream_t s) {
  if (n <= 0) return MM_OK;
  const int wpb = warps_per_block > 0 ? warps_per_block : 4;
  const int warps = ceil_div(n, 32);
  const int blocks = ceil_div(warps, wpb);
  if (counters)
    traverse_kernel<true><<<blocks, wpb * 32, 0, s>>>(n, ws.xs, ws.vals[0], ws.nodeA, ws.nodeB,
                                                       F, counters, ws.err);
  else
    traverse_kernel<false><<<blocks, wpb * 32, 0, s>>>(n, ws.xs, ws.vals[0], ws.nodeA,
                                                        ws.nodeB, F, nullptr, ws.err);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

mm_status exact_repulsion(XSel x, int n, float2* F, cudaStream_t s) {
  if (n <= 0) return MM_OK;
  exact_kernel<<<ceil_div(n, kExactThreads), kExactThreads, 0, s>>>(x, n, F);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

}  // namespace mm
