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
constexpr int kBBoxMaxBlocks = 2 * kMaxSMs;  // buffer bound; grids: 2 x num_sms()
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
// per-block partials and writes root = (min x, min y, side, 2^16 / side);
// it also bumps the build epoch (ticket[1]) that tags the sort's look-back
// status words, and zeroes the sort histograms and tile counters.
__global__ void __launch_bounds__(kBBoxThreads) bbox_kernel(XSel xs, int n, float4* partials,
                                                            unsigned* ticket, float4* root,
                                                            uint32_t* hist, uint32_t* counters) {
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
  // last block: reduce the partials in parallel, reset the sort state
  float4 r = make_float4(CUDART_INF_F, CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F);
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const float4 q = __ldcg(&partials[b]);
    r.x = fminf(r.x, q.x); r.y = fminf(r.y, q.y);
    r.z = fmaxf(r.z, q.z); r.w = fmaxf(r.w, q.w);
  }
  r.x = warp_min(r.x); r.y = warp_min(r.y); r.z = warp_max(r.z); r.w = warp_max(r.w);
  __syncthreads();
  if (lane == 0) sh[warp] = r;
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) hist[i] = 0u;
  if (threadIdx.x < 4) counters[threadIdx.x] = 0u;
  __syncthreads();
  if (threadIdx.x == 0) {
    r = sh[0];
    for (int w = 1; w < kBBoxThreads / 32; ++w) {
      r.x = fminf(r.x, sh[w].x); r.y = fminf(r.y, sh[w].y);
      r.z = fmaxf(r.z, sh[w].z); r.w = fmaxf(r.w, sh[w].w);
    }
    const float side = fmaxf(r.z - r.x, r.w - r.y);
    const float scale = side > 0.f ? 65536.0f / side : 0.f;
    *root = make_float4(r.x, r.y, side, scale);
    ticket[0] = 0u;
    ticket[1] += 1u;
  }
}

// Morton keys (16 bits per axis) and the four 8-bit digit histograms of the
// radix sort, in one pass over the positions.
__global__ void __launch_bounds__(kSortThreads) morton_hist_kernel(
    XSel xs, int n, int tile, const float4* __restrict__ root, uint32_t* __restrict__ keys,
    int32_t* __restrict__ vals, uint32_t* hist, uint32_t mask) {
  __shared__ uint32_t h[4][256];
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) (&h[0][0])[i] = 0u;
  __syncthreads();
  const float2* x = xs.cur();
  const float4 r = *root;
  const int base = blockIdx.x * tile;
  for (int j = threadIdx.x; j < tile; j += kSortThreads) {
    const int i = base + j;
    if (i >= n) break;
    const float2 p = x[i];
    const float fx = (p.x - r.x) * r.w, fy = (p.y - r.y) * r.w;
    // clamp in float first: the conversion of out-of-range values is undefined
    const uint32_t ix = (uint32_t)fminf(fmaxf(fx, 0.f), 65535.f);
    const uint32_t iy = (uint32_t)fminf(fmaxf(fy, 0.f), 65535.f);
    const uint32_t k = ((spread16(ix) << 1) | spread16(iy)) & mask;
    keys[i] = k;
    vals[i] = i;
#pragma unroll
    for (int d = 0; d < 4; ++d) atomicAdd(&h[d][(k >> (8 * d)) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) {
    const uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(&hist[i], c);
  }
}

// One stable counting pass of the sort (8-bit digit at `shift`) with
// decoupled look-back: a block takes the next tile in order, publishes its
// per-digit counts, accumulates the counts of the preceding tiles from their
// status words (epoch | flag | value; flag 1 = tile count, 2 = inclusive
// prefix) and scatters.  Waits are bounded: after spin_limit polls (the
// library passes kSpinLimit, about 0.1-1 s of polling) the block raises
// err[0] |= 2 and treats the missing tile as empty, so the kernel always
// finishes; every scatter stays inside [0, n) either way.
constexpr int kSpinLimit = 1 << 22;
constexpr int kLookback = 8;  // status words read per look-back step

template <int IPT>
__global__ void __launch_bounds__(kSortThreads) onesweep_pass(
    const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    int32_t* __restrict__ vout, int n, int pass, const uint32_t* __restrict__ hist,
    uint32_t* counters, unsigned long long* status, const unsigned* ticket, int* err,
    int spin_limit) {
  constexpr int kWarps = kSortThreads / 32;
  __shared__ uint32_t whist[kWarps][256];
  __shared__ uint32_t dbase[256];
  __shared__ int tile_sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int shift = 8 * pass;
  constexpr int kTile = kSortThreads * IPT;
  const int tiles = (n + kTile - 1) / kTile;
  if (threadIdx.x == 0) tile_sh = (int)atomicAdd(&counters[pass], 1u);
  for (int i = threadIdx.x; i < kWarps * 256; i += blockDim.x) (&whist[0][0])[i] = 0u;
  if (threadIdx.x < 32) {
    // exclusive scan of the 256 global digit counts of this pass
    uint32_t v[8], sum = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      v[j] = hist[pass * 256 + lane * 8 + j];
      sum += v[j];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    uint32_t run = inc - sum;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      dbase[lane * 8 + j] = run;
      run += v[j];
    }
  }
  __syncthreads();
  const int tile = tile_sh;
  const int64_t base = (int64_t)tile * kTile + warp * (32 * IPT);
  uint32_t key[IPT];
  int32_t val[IPT];
  uint32_t dig[IPT];
  unsigned peers[IPT];
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const int64_t idx = base + j * 32 + lane;
    const unsigned valid = __ballot_sync(0xffffffffu, idx < n);
    peers[j] = 0;
    if (idx < n) {
      key[j] = kin[idx];
      val[j] = vin[idx];
      dig[j] = (key[j] >> shift) & 255u;
      peers[j] = __match_any_sync(valid, dig[j]);
      if (lane == __ffs(peers[j]) - 1) whist[warp][dig[j]] += __popc(peers[j]);
    }
    __syncwarp();
  }
  __syncthreads();
  {
    const int d = threadIdx.x;  // one thread per digit (256 threads)
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) cnt += whist[w][d];
    const unsigned long long ep = (unsigned long long)ticket[1] << 32;
    unsigned long long* st = status + ((size_t)pass * tiles) * 256;
    volatile unsigned long long* vst = st;
    if (tile == 0) {
      vst[d] = ep | (2ull << 30) | cnt;
    } else {
      vst[(size_t)tile * 256 + d] = ep | (1ull << 30) | cnt;
    }
    uint32_t excl = 0;
    if (tile > 0) {
      // the status words of the kLookback nearest preceding tiles are read
      // together (independent loads), then added from the nearest back to
      // the first inclusive prefix; a word not yet published stops the
      // window and is polled again.  Walking back one tile per load would
      // make the last tile wait about (tiles x load latency).
      int t = tile - 1;
      int spins = 0;
      bool done = false;
      while (!done) {
        unsigned long long w[kLookback];
#pragma unroll
        for (int k = 0; k < kLookback; ++k)
          w[k] = t - k >= 0 ? vst[(size_t)(t - k) * 256 + d] : 0ull;
        int used = 0;
        bool stop = false;
#pragma unroll
        for (int k = 0; k < kLookback; ++k) {
          if (stop) continue;
          const uint32_t flag = (uint32_t)(w[k] >> 30) & 3u;
          if (t - k < 0 || (w[k] & 0xffffffff00000000ull) != ep || flag == 0) {
            stop = true;
            continue;
          }
          excl += (uint32_t)(w[k] & 0x3fffffffull);
          used = k + 1;
          if (flag == 2) done = stop = true;
        }
        if (done) break;
        t -= used;
        if (used == 0) {
          if (++spins > spin_limit) {
            atomicOr(err, 2);
            break;
          }
          __nanosleep(32);
        }
      }
      __threadfence();
      vst[(size_t)tile * 256 + d] = ep | (2ull << 30) | (excl + cnt);
    }
    uint32_t run = dbase[d] + excl;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = whist[w][d];
      whist[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    uint32_t pos = 0;
    const bool valid = peers[j] != 0;
    if (valid) pos = whist[warp][dig[j]] + __popc(peers[j] & lt);
    __syncwarp();
    if (valid && lane == __ffs(peers[j]) - 1) whist[warp][dig[j]] += __popc(peers[j]);
    __syncwarp();
    if (valid && pos < (uint32_t)n) {
      kout[pos] = key[j];
      vout[pos] = val[j];
    }
  }
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
__device__ __forceinline__ void karras_node(const uint32_t* __restrict__ k, int n, int i,
                                            int32_t* lo, int32_t* hi, int32_t* left,
                                            int32_t* right, int32_t* delta, int32_t* owner,
                                            int32_t* parent) {
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

// One radix-tree node per thread: the binary searches are chains of
// dependent loads, so they need all the parallelism there is.
__global__ void karras_kernel(const uint32_t* __restrict__ k, int n, int32_t* lo, int32_t* hi,
                              int32_t* left, int32_t* right, int32_t* delta, int32_t* owner,
                              int32_t* parent) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n - 1) karras_node(k, n, i, lo, hi, left, right, delta, owner, parent);
}

// Position sums in fixed point: a coordinate becomes (v - v0) * 2^32 / side
// (v0, side: the root square), an integer below 2^32 that keeps every bit of
// the FP32 difference; up to 2^31 of them add up exactly in 64 bits, in any
// order, at full integer rate (FP64 runs at a small fraction of the FP32
// rate on this GPU).  A cell's centroid is the difference of two prefix sums
// over its sorted range, divided by its count.
__device__ __forceinline__ unsigned long long fixq(float v, float v0, float scale) {
  const float f = fminf(fmaxf((v - v0) * scale, 0.f), 4294967040.f);  // largest float < 2^32
  return (unsigned long long)(uint32_t)f;
}

// Per tile of kSortThreads * IPT sorted positions: the inclusive fixed-point
// prefix sums within the tile (the tile total goes to tile_sum).
template <int IPT>
__global__ void __launch_bounds__(kSortThreads) scan_xs_kernel(
    XSel xs, const int32_t* __restrict__ vals, int n, const float4* __restrict__ root,
    float2* __restrict__ xsorted, ulonglong2* __restrict__ incl,
    ulonglong2* __restrict__ tile_sum) {
  const int base = blockIdx.x * (kSortThreads * IPT) + threadIdx.x * IPT;
  const float2* x = xs.cur();
  const float4 r = *root;
  const float scale = r.w * 65536.f;  // 2^32 / side
  unsigned long long qx[IPT], qy[IPT];
  unsigned long long sx = 0, sy = 0;
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const int i = base + j;
    qx[j] = qy[j] = 0;
    if (i < n) {
      const float2 v = x[vals[i]];
      xsorted[i] = v;
      qx[j] = fixq(v.x, r.x, scale);
      qy[j] = fixq(v.y, r.y, scale);
    }
    sx += qx[j];
    sy += qy[j];
  }
  // block exclusive scan of the per-thread sums
  __shared__ unsigned long long shx[kSortThreads / 32], shy[kSortThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long ix = sx, iy = sy;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long tx = __shfl_up_sync(0xffffffffu, ix, o);
    const unsigned long long ty = __shfl_up_sync(0xffffffffu, iy, o);
    if (lane >= o) { ix += tx; iy += ty; }
  }
  if (lane == 31) { shx[warp] = ix; shy[warp] = iy; }
  __syncthreads();
  unsigned long long rx = ix - sx, ry = iy - sy;
  for (int w = 0; w < warp; ++w) { rx += shx[w]; ry += shy[w]; }
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    rx += qx[j];
    ry += qy[j];
    if (base + j < n) incl[base + j] = make_ulonglong2(rx, ry);
  }
  if (threadIdx.x == kSortThreads - 1) tile_sum[blockIdx.x] = make_ulonglong2(rx, ry);
}

// Exclusive scan of the tile totals (one block).
__global__ void __launch_bounds__(1024) tile_scan_kernel(ulonglong2* tile_sum, int tiles) {
  __shared__ unsigned long long shx[32], shy[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int per = (tiles + blockDim.x - 1) / blockDim.x;
  const int beg = threadIdx.x * per, end = min(beg + per, tiles);
  unsigned long long sx = 0, sy = 0;
  for (int i = beg; i < end; ++i) { sx += tile_sum[i].x; sy += tile_sum[i].y; }
  unsigned long long ix = sx, iy = sy;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long tx = __shfl_up_sync(0xffffffffu, ix, o);
    const unsigned long long ty = __shfl_up_sync(0xffffffffu, iy, o);
    if (lane >= o) { ix += tx; iy += ty; }
  }
  if (lane == 31) { shx[warp] = ix; shy[warp] = iy; }
  __syncthreads();
  unsigned long long run_x = ix - sx, run_y = iy - sy;
  for (int w = 0; w < warp; ++w) { run_x += shx[w]; run_y += shy[w]; }
  __syncthreads();
  for (int i = beg; i < end; ++i) {
    const ulonglong2 c = tile_sum[i];
    tile_sum[i] = make_ulonglong2(run_x, run_y);
    run_x += c.x;
    run_y += c.y;
  }
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

__device__ void write_record(const TreeView& t, int id, float2 c, float side, float theta,
                             int leaf, int maxdepth, NodeRec* node) {
  const int n = t.n;
  if (id >= n - 1) {  // leaf j
    const int j = id - (n - 1);
    if (n > 1 && t.delta[t.parent[id]] >= 32) return;  // inside a bucket
    node[id].a = make_float4(c.x, c.y, 0.f, 1.f);
    node[id].b = make_int4(-1, escape_of(t, j), j, 1);
    return;
  }
  const int dd = t.delta[id];
  const int dp = id == 0 ? -1 : t.delta[t.parent[id]];
  int depth, first;
  if (dd >= 32) {  // duplicate keys: bucket leaf at the deepest level
    if (dp >= 32) return;
    depth = maxdepth;
    first = -1;
  } else {
    if (dp >= 0 && (dp >> 1) == (dd >> 1)) return;  // transparent
    depth = dd >> 1;
    first = resolve(t, t.left[id]);
  }
  const int a = t.lo[id], b = t.hi[id];
  // a cell of at most `leaf` points is a leaf: opened, it is summed exactly
  if (b - a + 1 <= leaf) first = -1;
  const float cnt = (float)(b - a + 1);
  const float w = ldexpf(side, -depth);
  const float rc = theta > 0.f ? (w / theta) * (w / theta) : CUDART_INF_F;
  node[id].a = make_float4(c.x, c.y, rc, cnt);
  node[id].b = make_int4(first, escape_of(t, b), a, b - a + 1);
}

// Fixed-point sum of the sorted positions [0, k): tile offset + inclusive
// sum in the tile.
__device__ __forceinline__ ulonglong2 prefix_at(const ulonglong2* __restrict__ incl,
                                                const ulonglong2* __restrict__ tile_off,
                                                int tile, int k) {
  if (k == 0) return make_ulonglong2(0, 0);
  const ulonglong2 a = tile_off[(k - 1) / tile];
  const ulonglong2 b = incl[k - 1];
  return make_ulonglong2(a.x + b.x, a.y + b.y);
}

// Node-parallel records: a cell's position sum is the difference of two
// prefix sums over its sorted range (exact integers); the centroid is that
// sum over the count, mapped back from fixed point in FP32.
// kFold: tile_off holds the raw tile totals (no tile scan ran) and every
// block scans them itself (few tiles: cheaper than one more launch): lane l
// of warp 0 adds a run of kFoldTiles / 32 consecutive tiles, a warp scan
// offsets the runs.
constexpr int kFoldTiles = 256;

template <bool kFold>
__global__ void records_kernel(TreeView t, const float2* __restrict__ xsorted,
                               const ulonglong2* __restrict__ incl,
                               const ulonglong2* __restrict__ tile_off, int tile,
                               const float4* __restrict__ root, float theta, int leaf,
                               int maxdepth, NodeRec* node, unsigned* walk_next) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = t.n;
  if (id == 0) *walk_next = 0u;  // the walk that follows deals its tasks from 0
  if (kFold) {
    constexpr int kPer = kFoldTiles / 32;
    __shared__ ulonglong2 off[kFoldTiles];
    const int tiles = (n + tile - 1) / tile;
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x, b0 = lane * kPer;
      unsigned long long sx = 0, sy = 0;
#pragma unroll
      for (int q = 0; q < kPer; ++q)
        if (b0 + q < tiles) { sx += tile_off[b0 + q].x; sy += tile_off[b0 + q].y; }
      unsigned long long ix = sx, iy = sy;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long tx = __shfl_up_sync(0xffffffffu, ix, o);
        const unsigned long long ty = __shfl_up_sync(0xffffffffu, iy, o);
        if (lane >= o) { ix += tx; iy += ty; }
      }
      unsigned long long rx = ix - sx, ry = iy - sy;
#pragma unroll
      for (int q = 0; q < kPer; ++q)
        if (b0 + q < tiles) {
          off[b0 + q] = make_ulonglong2(rx, ry);
          rx += tile_off[b0 + q].x;
          ry += tile_off[b0 + q].y;
        }
    }
    __syncthreads();
    tile_off = off;
  }
  if (id >= 2 * n - 1) return;
  const float4 r = *root;
  float2 c;
  if (id >= n - 1) {
    c = xsorted[id - (n - 1)];
  } else {
    const int lo = t.lo[id], hi = t.hi[id];
    const ulonglong2 a = prefix_at(incl, tile_off, tile, lo);
    const ulonglong2 b = prefix_at(incl, tile_off, tile, hi + 1);
    const float cnt = (float)(hi - lo + 1);
    const float scale = r.w * 65536.f;
    c = make_float2(r.x, r.y);  // all points coincide (side 0): the corner is each
    if (scale > 0.f) {
      c.x = r.x + ((float)(b.x - a.x) / cnt) / scale;
      c.y = r.y + ((float)(b.y - a.y) / cnt) / scale;
    }
  }
  write_record(t, id, c, r.z, theta, leaf, maxdepth, node);
}

// A cell record in one 256-bit load through the read-only path (the
// records are written by an earlier launch and only read by the walks).
__device__ __forceinline__ void ld_node(const NodeRec* __restrict__ p, float4& A, int4& B) {
  unsigned a0, a1, a2, a3;
  asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(a0), "=r"(a1), "=r"(a2), "=r"(a3), "=r"(B.x), "=r"(B.y), "=r"(B.z), "=r"(B.w)
      : "l"(p));
  A = make_float4(__uint_as_float(a0), __uint_as_float(a1), __uint_as_float(a2),
                  __uint_as_float(a3));
}

// Guards: node ids must stay in [0, 2n-1) and a walk visits each node at
// most once, so more than 2n visits or an out-of-range id means a broken
// tree; the warp then stops and raises err[0] instead of faulting or
// looping.
template <bool kCount>
__global__ void traverse_kernel(int n, const float2* __restrict__ xs,
                                const int32_t* __restrict__ vals,
                                const NodeRec* __restrict__ node, float2* __restrict__ F,
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
    float4 A;
    int4 B;
    ld_node(node + cur, A, B);
    if (wait == cur) wait = kNone;
    bool desc = false;
    if (wait == kNone) {
      const float dx = xu.x - A.x, dy = xu.y - A.y;
      const float q = fmaf(dx, dx, dy * dy);
      const bool inside = (unsigned)(pos - B.z) < (unsigned)B.w;
      if (!inside && q > A.z) {
        const float sc = __fdividef(A.w, q);
        fx = fmaf(sc, dx, fx);
        fy = fmaf(sc, dy, fy);
        wait = B.y;
        if (kCount) ++inter;
      } else if (B.x < 0) {
        const int pb = max(B.z, 0), pe = min(B.z + B.w, n);
        for (int p = pb; p < pe; ++p) {
          if (p == pos) continue;
          const float2 xv = xs[p];
          const float ex = xu.x - xv.x, ey = xu.y - xv.y;
          const float eq = fmaf(ex, ex, ey * ey);
          // the point itself (and any coincident one) has eq == 0: r = 0
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

constexpr int kSeedPoints = 256;  // a seed subtree holds at most this many points

constexpr int kSeedMax = 128;
constexpr int kGroupMaxWarps = 16;  // warps per block

struct GroupShared {
  int seeds[kGroupMaxWarps][kSeedMax];  // per task slot
  int nseeds[kGroupMaxWarps];
  float2 part[kGroupMaxWarps][32];      // per warp
};

// Packed FP32 pairs (fma.rn.f32x2 and friends, native on sm_100 and later:
// one instruction for both lanes of a float2).  Positions, offsets and the
// force accumulator are (x, y) pairs, so one packed operation does the work
// of two scalar ones.
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// Approximate reciprocal (the PTX rcp.approx instruction: one special-
// function-unit operation, relative error below 2^-22); q > 0 here.
__device__ __forceinline__ float rcp_approx(float q) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(q));
  return r;
}

// Group acceptance: the 32 Morton-consecutive points of a task walk the
// tree together (pre-order over first-child / escape links) and accept a
// cell only when every one of them passes the per-point test (w / |x_u - c|
// < theta, u not inside); a per-point accepted cell is then accepted too or
// opened into children, so each point's sum refines its per-point
// Barnes-Hut sum.  The walk is uniform across the warp: one vote per cell.
// W warps may share a task (small levels): the first warp records opened
// cells of at most `seed` points as seeds (up to kSeedMax) instead of
// entering them, the task's W warps then walk the seed subtrees (seed j by
// warp j mod W), and the W partial sums are added in warp order, so results
// are reproducible.
//
// Per visit the bookkeeping is kept small: the walk is a plain loop (a
// separate instance for the seeding walk); the acceptance test of a lane
// without a point always passes (its position is +inf and its index -1)
// instead of being tested; the point-in-cell test is one unsigned
// comparison; the accepted-cell term is computed on every visit and masked
// (no branch), the next cell is a select, and only the exact leaf sum is a
// (warp-uniform) branch; the leaf sum has no branch (a coincident point has
// a zero offset, and 1e-30 added to its squared distance keeps its term at
// zero); the record is one 256-bit load;
// and the position / offset / accumulator arithmetic is done on packed
// (x, y) pairs.
//
// kPhi: the walk also sums the log potential phi_u = sum_{v != u} ln|x_u - x_v|
// (the entropy term of Eq. 1) with the same decisions: an accepted cell
// adds count * ln|x_u - centroid|, a leaf its points exactly, a coincident
// point 0.
template <bool kCount, bool kSeeding, bool kPhi = false>
__device__ __forceinline__ void vote_walk(int cur, int stop, int n, int seed, int pos,
                                          unsigned long long xu, const float2* __restrict__ xs,
                                          const NodeRec* __restrict__ node,
                                          unsigned long long& acc,
                                          int& budget, bool& broken, int* seeds, int& nseeds,
                                          unsigned& visits, unsigned& inter, float& phi) {
  const unsigned nodes = 2u * (unsigned)n - 1u;
  const int lane = threadIdx.x & 31;
  const unsigned long long* xp = reinterpret_cast<const unsigned long long*>(xs);
  while (cur != stop) {
    if ((unsigned)cur >= nodes || --budget < 0) {
      broken = true;
      return;
    }
    float4 A;
    int4 B;
    ld_node(node + cur, A, B);
    if (kCount) ++visits;
    const unsigned long long d = sub2(xu, pk2(A.x, A.y));
    const float2 df = upk2(d);
    const float q = fmaf(df.x, df.x, df.y * df.y);
    const bool far = (unsigned)(pos - B.z) >= (unsigned)B.w && q > A.z;
    const bool take = __all_sync(0xffffffffu, far);
    // count / distance^2 of the accepted cell, 0 when the cell is not taken
    const float s = take ? A.w * rcp_approx(q) : 0.f;
    acc = fma2(pk2(s, s), d, acc);
    if (kPhi && take) phi = fmaf(0.5f * A.w, __logf(q), phi);
    if (kCount && take) ++inter;
    const bool leaf = !take && B.x < 0;
    if (leaf) {  // uniform: every lane read the same record
      const int pb = max(B.z, 0), pe = min(B.z + B.w, n);
#pragma unroll 4
      for (int p = pb; p < pe; ++p) {
        const unsigned long long e = sub2(xu, __ldg(&xp[p]));
        const float2 ef = upk2(e);
        // |e|^2 + 1e-30: the same float as |e|^2 for any two points that are
        // not (nearly) coincident, and a coincident point's zero offset keeps
        // its term at zero
        const float eq = fmaf(ef.x, ef.x, fmaf(ef.y, ef.y, 1e-30f));
        const float r = rcp_approx(eq);
        acc = fma2(pk2(r, r), e, acc);
        if (kPhi) {
          const float e2 = fmaf(ef.x, ef.x, ef.y * ef.y);
          phi += e2 > 0.f ? 0.5f * __logf(e2) : 0.f;
        }
      }
      if (kCount) inter += (unsigned)max(pe - pb, 0);
    }
    if (kSeeding && !take && !leaf && B.w <= seed && nseeds < kSeedMax) {
      if (lane == 0) seeds[nseeds] = cur;
      __syncwarp();
      if (lane == 0) ++nseeds;
      __syncwarp();
      cur = B.y;
    } else {
      cur = (take || leaf) ? B.y : B.x;
    }
  }
}

template <bool kCount, bool kPhi = false>
__global__ void __launch_bounds__(512, 3) traverse_vote_kernel(
    int n, int W, int seed, const float2* __restrict__ xs, const int32_t* __restrict__ vals,
    const NodeRec* __restrict__ node, float2* __restrict__ F, unsigned long long* counters,
    int* err, float* __restrict__ Phi = nullptr) {
  __shared__ GroupShared sh;
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  const int slot = wb / W, w = wb % W;
  const int tpb = (blockDim.x >> 5) / W;
  const int64_t task = (int64_t)blockIdx.x * tpb + slot;
  const bool live = task * 32 < n;
  const int p0 = (int)(task * 32) + lane;
  const bool valid = live && p0 < n;
  // a lane without a point: position +inf and index -1, so its acceptance
  // test always passes and it never vetoes a cell
  const int pos = valid ? p0 : -1;
  const float2 x0 = valid ? xs[p0] : make_float2(CUDART_INF_F, CUDART_INF_F);
  const unsigned long long xu = pk2(x0.x, x0.y);
  unsigned long long acc = pk2(0.f, 0.f);
  int* seeds = sh.seeds[slot];
  int& nseeds = sh.nseeds[slot];
  unsigned visits = 0, inter = 0;
  float phi = 0.f;
  int budget = 2 * n + 2;
  bool broken = false;
  if (w == 0 && live) {
    if (lane == 0) nseeds = 0;
    __syncwarp();
    if (W > 1 && seed > 0)
      vote_walk<kCount, true, kPhi>(n > 1 ? 0 : -1, -1, n, seed, pos, xu, xs, node, acc, budget,
                                    broken, seeds, nseeds, visits, inter, phi);
    else
      vote_walk<kCount, false, kPhi>(n > 1 ? 0 : -1, -1, n, seed, pos, xu, xs, node, acc, budget,
                                     broken, seeds, nseeds, visits, inter, phi);
  }
  float2 f = upk2(acc);
  if (W > 1) {
    __syncthreads();
    const int ns = live ? nseeds : 0;
    for (int j = w; j < ns && !broken; j += W) {
      const int c = seeds[j];
      vote_walk<kCount, false, kPhi>(c, __ldg(&node[c].b.y), n, seed, pos, xu, xs, node, acc,
                                     budget, broken, seeds, nseeds, visits, inter, phi);
    }
    f = upk2(acc);
    sh.part[wb][lane] = f;
    __syncthreads();
    if (w == 0) {
      float sx = 0.f, sy = 0.f;
      for (int k = 0; k < W; ++k) {
        sx += sh.part[slot * W + k][lane].x;
        sy += sh.part[slot * W + k][lane].y;
      }
      f = make_float2(sx, sy);
    }
    if (kPhi) {
      __syncthreads();
      sh.part[wb][lane].x = phi;
      __syncthreads();
      if (w == 0) {
        float sp = 0.f;
        for (int k = 0; k < W; ++k) sp += sh.part[slot * W + k][lane].x;
        phi = sp;
      }
    }
  }
  if (broken && lane == 0) atomicOr(err, 1);
  if (w == 0 && valid) {
    F[vals[p0]] = f;
    if (kPhi) Phi[vals[p0]] = phi;
  }
  if (kCount) {
    unsigned tot = valid ? inter : 0u;
#pragma unroll
    for (int o = 16; o; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0 && live) {
      atomicAdd(&counters[0], (unsigned long long)visits);
      atomicAdd(&counters[1], (unsigned long long)tot);
    }
  }
}

// The group walk with one warp per task (W = 1, the large levels) as a
// persistent grid: every warp takes the next 32-point task from a counter
// (zeroed by the record kernel of the same build) until none is left, so
// no SM idles in a last, partly filled wave while others still walk.  Each
// task writes only its own points: the result does not depend on which
// warp took it.
template <bool kCount>
__global__ void __launch_bounds__(256, 6) traverse_dyn_kernel(
    int n, const float2* __restrict__ xs, const int32_t* __restrict__ vals,
    const NodeRec* __restrict__ node, float2* __restrict__ F, unsigned* walk_next,
    unsigned long long* counters, int* err) {
  const int lane = threadIdx.x & 31;
  const int tasks = (n + 31) / 32;
  unsigned visits = 0, inter = 0;
  int no_seed = 0;
  for (;;) {
    int task = 0;
    if (lane == 0) task = (int)atomicAdd(walk_next, 1u);
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task >= tasks) break;
    const int p0 = task * 32 + lane;
    const bool valid = p0 < n;
    const int pos = valid ? p0 : -1;
    const float2 x0 = valid ? xs[p0] : make_float2(CUDART_INF_F, CUDART_INF_F);
    unsigned long long acc = pk2(0.f, 0.f);
    unsigned v = 0, it = 0;
    float phi = 0.f;
    int budget = 2 * n + 2;
    bool broken = false;
    vote_walk<kCount, false, false>(n > 1 ? 0 : -1, -1, n, 0, pos, pk2(x0.x, x0.y), xs, node,
                                    acc, budget, broken, nullptr, no_seed, v, it, phi);
    if (broken && lane == 0) atomicOr(err, 1);
    if (valid) F[vals[p0]] = upk2(acc);
    if (kCount) {
      visits += v;
      inter += valid ? it : 0u;
    }
  }
  if (kCount) {
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
  const unsigned long long xu2 = pk2(xu.x, xu.y);
  const unsigned long long* tp = reinterpret_cast<const unsigned long long*>(tile);
  unsigned long long acc = pk2(0.f, 0.f);
  for (int t0 = 0; t0 < n; t0 += kExactThreads) {
    const int cnt = min(kExactThreads, n - t0);
    if (threadIdx.x < cnt) tile[threadIdx.x] = x[t0 + threadIdx.x];
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < cnt; ++k) {
      // packed (x, y) offset and accumulator; a coincident point (its own
      // included) has a zero offset, and the 1e-30 added to the squared
      // distance (lost in rounding for any other pair) keeps its term at zero
      const unsigned long long d = sub2(xu2, tp[k]);
      const float2 df = upk2(d);
      const float q = fmaf(df.x, df.x, fmaf(df.y, df.y, 1e-30f));
      const float r = rcp_approx(q);
      acc = fma2(pk2(r, r), d, acc);
    }
    __syncthreads();
  }
  if (u < n) F[u] = upk2(acc);
}

// The same sum for levels too small to fill the GPU one vertex per thread:
// block (vb, c) sums the sources of chunk c for vertices 128 vb ..; each
// block stores its partial, and the last block of a vertex block to arrive
// adds the chunk partials in chunk order (reproducible) and resets the
// arrival counter for the next sweep.
constexpr int kExactSplitThreads = 128;

__global__ void __launch_bounds__(kExactSplitThreads) exact_split_kernel(
    XSel xs, int n, int chunk, int chunks, float2* __restrict__ part, unsigned* arrive,
    float2* __restrict__ F) {
  __shared__ float2 tile[kExactSplitThreads];
  __shared__ bool last;
  const float2* x = xs.cur();
  const int vb = blockIdx.x, c = blockIdx.y;
  const int u = vb * kExactSplitThreads + threadIdx.x;
  const float2 xu = u < n ? x[u] : make_float2(0.f, 0.f);
  const unsigned long long xu2 = pk2(xu.x, xu.y);
  const unsigned long long* tp = reinterpret_cast<const unsigned long long*>(tile);
  unsigned long long acc = pk2(0.f, 0.f);
  const int j0 = c * chunk, j1 = min(n, j0 + chunk);
  for (int t0 = j0; t0 < j1; t0 += kExactSplitThreads) {
    const int cnt = min(kExactSplitThreads, j1 - t0);
    if (threadIdx.x < cnt) tile[threadIdx.x] = x[t0 + threadIdx.x];
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < cnt; ++k) {
      // packed (x, y) offset and accumulator; a coincident point (its own
      // included) has a zero offset, and the 1e-30 added to the squared
      // distance (lost in rounding for any other pair) keeps its term at zero
      const unsigned long long d = sub2(xu2, tp[k]);
      const float2 df = upk2(d);
      const float q = fmaf(df.x, df.x, fmaf(df.y, df.y, 1e-30f));
      const float r = rcp_approx(q);
      acc = fma2(pk2(r, r), d, acc);
    }
    __syncthreads();
  }
  if (u < n) part[(size_t)c * n + u] = upk2(acc);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&arrive[vb], 1u) == (unsigned)(chunks - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (u < n) {
    float sx = 0.f, sy = 0.f;
    for (int q = 0; q < chunks; ++q) {
      const float2 pq = __ldcg(&part[(size_t)q * n + u]);
      sx += pq.x;
      sy += pq.y;
    }
    F[u] = make_float2(sx, sy);
  }
  if (threadIdx.x == 0) arrive[vb] = 0u;
}

}  // namespace

bool tree_tile_scan(int64_t n) {
  return ceil_div(n, (int64_t)kSortThreads * sort_ipt(n)) > kFoldTiles;
}

size_t tree_status_words(int64_t n) {
  return (size_t)4 * ceil_div(n > 1 ? n : 2, kSortMinTile) * 256;
}

mm_status walk_setup(TreeWS& ws) {
  int per_sm = 0;
  MM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, traverse_dyn_kernel<false>, 256,
                                                      0));
  ws.walk_resident = std::max(1, per_sm) * num_sms();
  return MM_OK;
}

mm_status tree_ws_alloc(TreeWS& ws, int64_t n, cudaStream_t s) {
  const size_t N = (size_t)(n > 1 ? n : 2);
  const size_t tiles = (size_t)ceil_div((int64_t)N, kSortMinTile);
  ws.cap = n;
  MM_CK(cudaMallocAsync(&ws.keys[0], sizeof(uint32_t) * N, s));
  MM_CK(cudaMallocAsync(&ws.keys[1], sizeof(uint32_t) * N, s));
  MM_CK(cudaMallocAsync(&ws.vals[0], sizeof(int32_t) * N, s));
  MM_CK(cudaMallocAsync(&ws.vals[1], sizeof(int32_t) * N, s));
  MM_CK(cudaMallocAsync(&ws.xs, sizeof(float2) * N, s));
  MM_CK(cudaMallocAsync(&ws.lo, sizeof(int32_t) * N, s));
  MM_CK(cudaMallocAsync(&ws.hi, sizeof(int32_t) * N, s));
  MM_CK(cudaMallocAsync(&ws.left, sizeof(int32_t) * N, s));
  MM_CK(cudaMallocAsync(&ws.right, sizeof(int32_t) * N, s));
  MM_CK(cudaMallocAsync(&ws.delta, sizeof(int32_t) * N, s));
  MM_CK(cudaMallocAsync(&ws.owner, sizeof(int32_t) * N, s));
  MM_CK(cudaMallocAsync(&ws.parent, sizeof(int32_t) * 2 * N, s));
  MM_CK(cudaMallocAsync(&ws.incl, sizeof(ulonglong2) * N, s));
  MM_CK(cudaMallocAsync(&ws.tile_sum, sizeof(ulonglong2) * tiles, s));
  MM_CK(cudaMallocAsync(&ws.status, sizeof(unsigned long long) * tree_status_words(N), s));
  MM_CK(cudaMemsetAsync(ws.status, 0, sizeof(unsigned long long) * tree_status_words(N), s));
  MM_CK(cudaMallocAsync(&ws.hist, sizeof(uint32_t) * 4 * 256, s));
  MM_CK(cudaMallocAsync(&ws.counters, sizeof(uint32_t) * 4, s));
  MM_CK(cudaMallocAsync(&ws.walk_next, sizeof(unsigned), s));
  MM_CK(cudaMemsetAsync(ws.walk_next, 0, sizeof(unsigned), s));
  MM_CK(cudaMallocAsync(&ws.node, sizeof(NodeRec) * 2 * N, s));
  MM_CK(cudaMallocAsync(&ws.partials, sizeof(float4) * kBBoxMaxBlocks, s));
  MM_CK(cudaMallocAsync(&ws.root, sizeof(float4), s));
  MM_CK(cudaMallocAsync(&ws.ticket, 2 * sizeof(unsigned), s));
  MM_CK(cudaMemsetAsync(ws.ticket, 0, 2 * sizeof(unsigned), s));
  MM_CK(cudaMallocAsync(&ws.err, sizeof(int), s));
  MM_CK(cudaMemsetAsync(ws.err, 0, sizeof(int), s));
  // unwritten records read as leaves whose escape ends the walk
  MM_CK(cudaMemsetAsync(ws.node, 0xff, sizeof(NodeRec) * 2 * N, s));
  MM_TRY(walk_setup(ws));
  MM_CK(cudaStreamCreateWithFlags(&ws.aux, cudaStreamNonBlocking));
  MM_CK(cudaEventCreateWithFlags(&ws.fork, cudaEventDisableTiming));
  MM_CK(cudaEventCreateWithFlags(&ws.join, cudaEventDisableTiming));
  return MM_OK;
}

void tree_ws_free(TreeWS& ws) {
  void* ptrs[] = {ws.keys[0], ws.keys[1], ws.vals[0], ws.vals[1], ws.xs, ws.lo, ws.hi,
                  ws.left, ws.right, ws.delta, ws.owner, ws.parent, ws.incl, ws.tile_sum,
                  ws.status, ws.hist, ws.counters, ws.walk_next, ws.node, ws.partials, ws.root,
                  ws.ticket, ws.err};
  for (void* p : ptrs) cudaFree(p);
  if (ws.fork) cudaEventDestroy(ws.fork);
  if (ws.join) cudaEventDestroy(ws.join);
  if (ws.aux) cudaStreamDestroy(ws.aux);
  ws = TreeWS();
}

mm_status bh_bbox(XSel x, int n, TreeWS& ws, cudaStream_t s) {
  if (n <= 0) return MM_OK;
  const int bb = std::min(2 * num_sms(), ceil_div(n, kBBoxThreads));
  bbox_kernel<<<bb, kBBoxThreads, 0, s>>>(x, n, ws.partials, ws.ticket, ws.root, ws.hist,
                                          ws.counters);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

mm_status bh_build(XSel x, int n, float theta, int leaf, TreeWS& ws, cudaStream_t s,
                   cudaEvent_t* ev, bool with_bbox, bool coarse_keys) {
  if (n <= 0) return MM_OK;
  if (n > ws.cap) {
    set_error("tree workspace holds %lld vertices, level has %d", (long long)ws.cap, n);
    return MM_ERR_INVALID_ARG;
  }
  auto mark = [&](int i) {
    if (ev) cudaEventRecord(ev[i], s);
  };
  const int ipt = sort_ipt(n);
  const int tile = kSortThreads * ipt;
  const int tiles = ceil_div(n, tile);
  mark(0);
  if (with_bbox) MM_TRY(bh_bbox(x, n, ws, s));
  mark(1);
  // 32-bit keys: four stable 8-bit passes from buffer 0; coarse keys (the
  // low 8 bits cleared: cells down to depth 12) need only the passes over
  // the upper three digits, from buffer 1.  Either way the result ends in
  // buffer 0.
  const int first = coarse_keys ? 1 : 0;
  morton_hist_kernel<<<tiles, kSortThreads, 0, s>>>(x, n, tile, ws.root, ws.keys[first],
                                                   ws.vals[first], ws.hist,
                                                   coarse_keys ? 0xffffff00u : 0xffffffffu);
  mark(2);
  for (int pass = first; pass < 4; ++pass) {
    const int a = pass & 1;
    auto pass_kernel = ipt == 8   ? onesweep_pass<8>
                       : ipt == 4 ? onesweep_pass<4>
                       : ipt == 2 ? onesweep_pass<2>
                                  : onesweep_pass<1>;
    pass_kernel<<<tiles, kSortThreads, 0, s>>>(ws.keys[a], ws.vals[a], ws.keys[a ^ 1],
                                               ws.vals[a ^ 1], n, pass, ws.hist, ws.counters,
                                               ws.status, ws.ticket, ws.err, kSpinLimit);
  }
  mark(3);
  // the radix tree and the position prefix sums both need only the sorted
  // keys: the tree is built on a second stream (a parallel graph branch
  // under capture) while the sums run here
  cudaStream_t ts = ws.aux ? ws.aux : s;
  if (ws.aux) {
    MM_CK(cudaEventRecord(ws.fork, s));
    MM_CK(cudaStreamWaitEvent(ws.aux, ws.fork, 0));
  }
  if (n > 1)
    karras_kernel<<<ceil_div(n - 1, 256), 256, 0, ts>>>(ws.keys[0], n, ws.lo, ws.hi, ws.left,
                                                        ws.right, ws.delta, ws.owner, ws.parent);
  auto scan_kernel = ipt == 8   ? scan_xs_kernel<8>
                     : ipt == 4 ? scan_xs_kernel<4>
                     : ipt == 2 ? scan_xs_kernel<2>
                                : scan_xs_kernel<1>;
  scan_kernel<<<tiles, kSortThreads, 0, s>>>(x, ws.vals[0], n, ws.root, ws.xs, ws.incl,
                                             ws.tile_sum);
  const bool fold = tiles <= kFoldTiles;
  if (!fold) tile_scan_kernel<<<1, 1024, 0, s>>>(ws.tile_sum, tiles);
  if (ws.aux) {
    MM_CK(cudaEventRecord(ws.join, ws.aux));
    MM_CK(cudaStreamWaitEvent(s, ws.join, 0));
  }
  mark(4);
  TreeView tv{n, ws.lo, ws.hi, ws.left, ws.right, ws.delta, ws.owner, ws.parent};
  if (fold)
    records_kernel<true><<<ceil_div(2 * n - 1, 256), 256, 0, s>>>(
        tv, ws.xs, ws.incl, ws.tile_sum, tile, ws.root, theta, leaf,
        coarse_keys ? 12 : kKeyBits, ws.node, ws.walk_next);
  else
    records_kernel<false><<<ceil_div(2 * n - 1, 256), 256, 0, s>>>(
        tv, ws.xs, ws.incl, ws.tile_sum, tile, ws.root, theta, leaf,
        coarse_keys ? 12 : kKeyBits, ws.node, ws.walk_next);
  mark(5);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

mm_status bh_traverse(int n, const TreeWS& ws, float2* F, int warps_per_block,
                      unsigned long long* counters, cudaStream_t s, int mode) {
  if (n <= 0) return MM_OK;
  const int wpb = warps_per_block > 0 ? warps_per_block : 4;
  const int warps = ceil_div(n, 32);
  const int blocks = ceil_div(warps, wpb);
  if (mode != 0) {
    // W warps share a task of 32 points; blocks of at least 8 warps
    const int tasks = ceil_div(n, 32);
    const int W = std::max(1, std::min(kGroupMaxWarps, wpb));
    const int tpb = std::max(1, 8 / W);
    const int seed = W > 1 ? kSeedPoints : 0;
    if (W == 1) {
      // persistent: as many 256-thread blocks as fit (walk_setup), tasks
      // dealt by a counter
      const int grid = std::max(1, std::min(std::max(ws.walk_resident, 1), ceil_div(tasks, 8)));
      auto kern = counters ? traverse_dyn_kernel<true> : traverse_dyn_kernel<false>;
      kern<<<grid, 256, 0, s>>>(n, ws.xs, ws.vals[0], ws.node, F, ws.walk_next, counters,
                                ws.err);
      MM_CK(cudaGetLastError());
      return MM_OK;
    }
    auto kern = counters ? traverse_vote_kernel<true> : traverse_vote_kernel<false>;
    kern<<<ceil_div(tasks, tpb), tpb * W * 32, 0, s>>>(n, W, seed, ws.xs, ws.vals[0], ws.node, F,
                                                      counters, ws.err, nullptr);
  } else if (counters) {
    traverse_kernel<true><<<blocks, wpb * 32, 0, s>>>(n, ws.xs, ws.vals[0], ws.node, F,
                                                       counters, ws.err);
  } else {
    traverse_kernel<false><<<blocks, wpb * 32, 0, s>>>(n, ws.xs, ws.vals[0], ws.node, F,
                                                        nullptr, ws.err);
  }
  MM_CK(cudaGetLastError());
  return MM_OK;
}

mm_status bh_potential(int n, const TreeWS& ws, float2* F, float* Phi, int warps_per_block,
                       cudaStream_t s) {
  if (n <= 0) return MM_OK;
  const int wpb = warps_per_block > 0 ? warps_per_block : 4;
  const int tasks = ceil_div(n, 32);
  const int W = std::max(1, std::min(kGroupMaxWarps, wpb));
  const int tpb = std::max(1, 8 / W);
  const int seed = W > 1 ? kSeedPoints : 0;
  traverse_vote_kernel<false, true><<<ceil_div(tasks, tpb), tpb * W * 32, 0, s>>>(
      n, W, seed, ws.xs, ws.vals[0], ws.node, F, nullptr, ws.err, Phi);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

int exact_chunks(int n) {
  // split the sources until about sixteen 4-warp blocks per SM are busy
  // (the loop is latency-bound at fewer), within the partial-sum buffer
  // (kExactPartCap float2)
  const int vblocks = ceil_div(std::max(n, 1), kExactSplitThreads);
  const int want = ceil_div(16 * num_sms(), vblocks);
  return std::max(1, std::min(want, kExactPartCap / std::max(n, 1)));
}

mm_status exact_repulsion(XSel x, int n, float2* F, cudaStream_t s, float2* part,
                          unsigned* arrive) {
  if (n <= 0) return MM_OK;
  const int chunks = part && arrive ? exact_chunks(n) : 1;
  if (chunks <= 1) {
    exact_kernel<<<ceil_div(n, kExactThreads), kExactThreads, 0, s>>>(x, n, F);
  } else {
    const int chunk = ceil_div(ceil_div(n, chunks), 32) * 32;
    const int c = ceil_div(n, chunk);
    exact_split_kernel<<<dim3(ceil_div(n, kExactSplitThreads), c), kExactSplitThreads, 0, s>>>(
        x, n, chunk, c, part, arrive, F);
  }
  MM_CK(cudaGetLastError());
  return MM_OK;
}

// Self-test of the bounded look-back wait (a measurement and deployment aid,
// no paper counterpart).  One block of the sort pass is launched on a key
// set of two tiles with the tile counter preset to 1, so it takes tile 1 and
// waits for tile 0, which never runs: nothing ever publishes the status word
// it polls.  The wait must give up after spin_limit polls, raise error bit 2
// and let the kernel finish (all its reads and writes stay inside the
// buffers allocated here).  *timed_out = 1 if it did.
mm_status lookback_selftest(int spin_limit, int* timed_out, cudaStream_t s) {
  constexpr int kTile = kSortThreads;  // one key per thread
  constexpr int n = 2 * kTile;
  struct Bufs {
    uint32_t kin[n], kout[n], hist[4 * 256], counters[4];
    int32_t vin[n], vout[n];
    unsigned long long status[4 * 2 * 256];
    unsigned ticket[2];
    int err;
  };
  Bufs* d = nullptr;
  MM_CK(cudaMallocAsync((void**)&d, sizeof(Bufs), s));
  mm_status st = MM_OK;
  int err = 0;
  const uint32_t one = 1u;
  // zero everything; tile counter 1 (the block takes tile 1); epoch 1 (the
  // zeroed status words carry epoch 0, so none is ever valid)
  if (cudaMemsetAsync(d, 0, sizeof(Bufs), s) != cudaSuccess ||
      cudaMemcpyAsync(&d->counters[0], &one, 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(&d->ticket[1], &one, 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    st = cuda_status(cudaGetLastError(), "look-back self-test set-up", __FILE__, __LINE__);
  } else {
    onesweep_pass<1><<<1, kSortThreads, 0, s>>>(d->kin, d->vin, d->kout, d->vout, n, 0, d->hist,
                                                d->counters, d->status, d->ticket, &d->err,
                                                spin_limit);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&err, &d->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "look-back self-test", __FILE__, __LINE__);
  }
  cudaFreeAsync(d, s);
  *timed_out = (err & 2) ? 1 : 0;
  return st;
}

}  // namespace mm
