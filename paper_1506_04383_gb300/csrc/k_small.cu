// Fused level kernel for small levels: one CTA of 1024 threads runs a whole
// level schedule (Sec. 3.2) -- every Eq. 2 iteration and every alpha round --
// without leaving the kernel.
//
// On the coarse levels of a hierarchy (a few dozen to a few thousand
// vertices) a sweep is a chain of tiny dependent steps; issued as separate
// launches each costs a launch and an L2 round trip per node visit.  Here
// every per-sweep structure lives in shared memory:
//   bounding square -> Morton keys (16 bits per axis, the same cells as the
//   multi-kernel path) -> bitonic sort of (key, index) -> Karras radix tree
//   -> centroids from float-float prefix sums of the sorted positions ->
//   32-byte node records -> warp-synchronous stackless walk (per-lane
//   acceptance, as in the multi-kernel walk) -> Eq. 2 update over S (rows
//   read from global memory) -> block reductions (FP32 within a warp,
//   float-float across warps) -> the schedule step.
// With exact repulsion (the coarsest level) the walk is replaced by the
// all-pairs sum over the staged positions.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>

#include "mm_internal.cuh"

namespace mm {

namespace {

constexpr int kT = kSmallThreads;
constexpr int kN = kSmallMaxN;
constexpr int kNodes = 2 * kN - 1;
constexpr int kNone = -2;

struct __align__(16) SmallSmem {
  // about 216 KB: fits the 227 KB a CTA may opt into
  float4 nodeA[kNodes];       // (cx, cy, (w/theta)^2, count)
  short4 nodeB[kNodes];       // (first child, escape, lo, hi+1)
  union {                         // three phases, three uses:
    unsigned long long keys[kN];  //   sort keys (sort, radix tree)
    float4 P[kN + 1];             //   float-float prefix sums (x_hi, y_hi, x_lo, y_lo)
    float2 F[kN];                 //   long-range sums by vertex id (walk, update)
  };
  float2 xs[kN];              // sorted positions (tree build, walk)
  float2 xv[kN];              // positions by vertex id, staged once per sweep
  int32_t sp[kN + 1];         // S row pointers of the level (staged once)
  float rho[kN];              // rho of the level (staged once)
  int16_t lo[kN], hi[kN], left[kN], right[kN], owner[kN];
  int16_t parent[kNodes + 1];
  int16_t vals[kN];
  int8_t delta[kN];
};

__device__ __forceinline__ uint32_t spread16(uint32_t v) {
  v &= 0xffffu;
  v = (v | (v << 8)) & 0x00ff00ffu;
  v = (v | (v << 4)) & 0x0f0f0f0fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

__device__ __forceinline__ int plen(const SmallSmem& s, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  const uint32_t a = (uint32_t)(s.keys[i] >> 32), b = (uint32_t)(s.keys[j] >> 32);
  if (a != b) return __clz(a ^ b);
  return 32 + __clz((uint32_t)i ^ (uint32_t)j);
}

__device__ __forceinline__ int s_resolve(const SmallSmem& s, int n, int x) {
  if (x >= n - 1 || x == 0) return x;
  const int dx = s.delta[x];
  if (dx >= 32) return x;
  const int dp = s.delta[s.parent[x]];
  return (dp >> 1) == (dx >> 1) ? s.left[x] : x;
}

__device__ __forceinline__ int s_escape(const SmallSmem& s, int n, int h) {
  if (h >= n - 1) return -1;
  return s_resolve(s, n, s.right[s.owner[h]]);
}

// Block-wide sums of three per-thread partials: warp shuffles in FP32, the 32
// warp totals in float-float by warp 0.  Result valid in thread 0.
__device__ __forceinline__ void bsum3(float a, float b, float c, double* red, double out[3]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  float* fr = reinterpret_cast<float*>(red);
  __syncthreads();
  if (lane == 0) { fr[warp] = a; fr[32 + warp] = b; fr[64 + warp] = c; }
  __syncthreads();
  if (warp == 0) {
    float2 p = make_float2(lane < kT / 32 ? fr[lane] : 0.f, 0.f);
    float2 q = make_float2(lane < kT / 32 ? fr[32 + lane] : 0.f, 0.f);
    float2 r = make_float2(lane < kT / 32 ? fr[64 + lane] : 0.f, 0.f);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      p = ff_add(p, ff_shfl_xor(p, o));
      q = ff_add(q, ff_shfl_xor(q, o));
      r = ff_add(r, ff_shfl_xor(r, o));
    }
    if (lane == 0) {
      out[0] = (double)p.x + (double)p.y;
      out[1] = (double)q.x + (double)q.y;
      out[2] = (double)r.x + (double)r.y;
    }
  }
}

#define MM_STAMP(i)                                          \
  do {                                                       \
    if (prof && threadIdx.x == 0) prof[i] = clock64();       \
  } while (0)

// Bitonic sort of np keys (np a power of two <= 2048) in shared memory.
// Every stage whose compare distance j is below 64 pairs elements of the
// same 64-element block, so a warp does those stages in registers: lane l
// holds block elements l and l + 32, distance 32 is a swap inside the lane,
// shorter distances a shuffle.  Only distances >= 64 go through shared
// memory with a block barrier each (15 of the 66 stages at np = 2048).
__device__ __forceinline__ unsigned long long bitonic_cx(unsigned long long v, int i, int j,
                                                         int k) {
  const unsigned long long p = __shfl_xor_sync(0xffffffffu, v, j);
  const bool asc = (i & k) == 0, lower = (i & j) == 0;
  const unsigned long long mn = v < p ? v : p, mx = v < p ? p : v;
  return lower == asc ? mn : mx;
}

__device__ __forceinline__ void bitonic_regs(unsigned long long& v0, unsigned long long& v1,
                                             int i0, int k, int jmax) {
  for (int j = jmax; j > 0; j >>= 1) {
    if (j == 32) {
      // partner of i0 is i0 + 32 = the element in v1
      const bool asc = (i0 & k) == 0;
      const unsigned long long mn = v0 < v1 ? v0 : v1, mx = v0 < v1 ? v1 : v0;
      v0 = asc ? mn : mx;
      v1 = asc ? mx : mn;
    } else {
      v0 = bitonic_cx(v0, i0, j, k);
      v1 = bitonic_cx(v1, i0 + 32, j, k);
    }
  }
}

__device__ void sort_keys(unsigned long long* keys, int np) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = warp * 64 + lane, i1 = i0 + 32;
  // fewer than 64 keys: warp 0 sorts them padded with the largest key
  const bool live = warp * 64 < np;
  unsigned long long v0 = ~0ull, v1 = ~0ull;
  if (live) {
    if (i0 < np) v0 = keys[i0];
    if (i1 < np) v1 = keys[i1];
    for (int k = 2; k <= 64; k <<= 1) bitonic_regs(v0, v1, i0, k, k >> 1);
    if (i0 < np) keys[i0] = v0;
    if (i1 < np) keys[i1] = v1;
  }
  __syncthreads();
  for (int k = 128; k <= np; k <<= 1) {
    for (int j = k >> 1; j >= 64; j >>= 1) {
      for (int i = threadIdx.x; i < np; i += kT) {
        const int ij = i ^ j;
        if (ij > i) {
          const unsigned long long a = keys[i], b = keys[ij];
          const bool up = (i & k) == 0;
          if ((a > b) == up) { keys[i] = b; keys[ij] = a; }
        }
      }
      __syncthreads();
    }
    if (live) {
      v0 = keys[i0];
      v1 = keys[i1];
      bitonic_regs(v0, v1, i0, k, 32);
      keys[i0] = v0;
      keys[i1] = v1;
    }
    __syncthreads();
  }
}

__device__ void build_tree(SmallSmem& s, int n, float theta, int leaf, float4* root_sh,
                           double* red, long long* prof) {
  const float2* x = s.xv;
  const int tid = threadIdx.x;
  // bounding square
  float mnx = CUDART_INF_F, mny = CUDART_INF_F, mxx = -CUDART_INF_F, mxy = -CUDART_INF_F;
  for (int i = tid; i < n; i += kT) {
    const float2 p = x[i];
    mnx = fminf(mnx, p.x); mny = fminf(mny, p.y);
    mxx = fmaxf(mxx, p.x); mxy = fmaxf(mxy, p.y);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    mnx = fminf(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
    mny = fminf(mny, __shfl_xor_sync(0xffffffffu, mny, o));
    mxx = fmaxf(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
    mxy = fmaxf(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
  }
  float* fr = reinterpret_cast<float*>(red);
  const int lane = tid & 31, warp = tid >> 5;
  __syncthreads();
  if (lane == 0) {
    fr[4 * warp] = mnx; fr[4 * warp + 1] = mny; fr[4 * warp + 2] = mxx; fr[4 * warp + 3] = mxy;
  }
  __syncthreads();
  if (tid == 0) {
    float4 r = make_float4(fr[0], fr[1], fr[2], fr[3]);
    for (int w = 1; w < kT / 32; ++w) {
      r.x = fminf(r.x, fr[4 * w]); r.y = fminf(r.y, fr[4 * w + 1]);
      r.z = fmaxf(r.z, fr[4 * w + 2]); r.w = fmaxf(r.w, fr[4 * w + 3]);
    }
    const float side = fmaxf(r.z - r.x, r.w - r.y);
    *root_sh = make_float4(r.x, r.y, side, side > 0.f ? 65536.0f / side : 0.f);
  }
  __syncthreads();
  MM_STAMP(2);
  const float4 root = *root_sh;
  // Morton keys with the index in the low word: a total order that equals
  // the stable order of the multi-kernel radix sort
  int np = 2;
  while (np < n) np <<= 1;
  for (int i = tid; i < np; i += kT) {
    unsigned long long k = ~0ull;
    if (i < n) {
      const float2 p = x[i];
      const float fx = (p.x - root.x) * root.w, fy = (p.y - root.y) * root.w;
      const uint32_t ix = (uint32_t)fminf(fmaxf(fx, 0.f), 65535.f);
      const uint32_t iy = (uint32_t)fminf(fmaxf(fy, 0.f), 65535.f);
      k = ((unsigned long long)((spread16(ix) << 1) | spread16(iy)) << 32) | (uint32_t)i;
    }
    s.keys[i] = k;
  }
  __syncthreads();
  sort_keys(s.keys, np);
  MM_STAMP(3);
  for (int i = tid; i < n; i += kT) {
    const int v = (int)(uint32_t)s.keys[i];
    s.vals[i] = (int16_t)v;
    s.xs[i] = x[v];
  }
  __syncthreads();
  // Karras radix tree over the sorted keys
  for (int i = tid; i < n - 1; i += kT) {
    const int dr = plen(s, n, i, i + 1), dl = plen(s, n, i, i - 1);
    const int d = dr > dl ? 1 : -1;
    const int dmin = d > 0 ? dl : dr;
    int lmax = 2;
    while (plen(s, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
      if (plen(s, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = plen(s, n, i, j);
    int sp = 0, t = l;
    do {
      t = (t + 1) >> 1;
      if (plen(s, n, i, i + (sp + t) * d) > dnode) sp += t;
    } while (t > 1);
    const int g = i + sp * d + (d < 0 ? -1 : 0);
    const int a = min(i, j), b = max(i, j);
    const int L = (a == g) ? (n - 1 + g) : g;
    const int R = (b == g + 1) ? (n - 1 + g + 1) : g + 1;
    s.lo[i] = (int16_t)a; s.hi[i] = (int16_t)b; s.left[i] = (int16_t)L;
    s.right[i] = (int16_t)R; s.delta[i] = (int8_t)dnode; s.owner[g] = (int16_t)i;
    s.parent[L] = (int16_t)i; s.parent[R] = (int16_t)i;
  }
  if (tid == 0) s.parent[0] = -1;
  __syncthreads();
  MM_STAMP(4);
  // float-float prefix sums of the sorted positions: P[i] = sum_{j < i} xs[j]
  {
    const int i0 = 2 * tid;
    const float2 a = i0 < n ? s.xs[i0] : make_float2(0.f, 0.f);
    const float2 b2 = i0 + 1 < n ? s.xs[i0 + 1] : make_float2(0.f, 0.f);
    // pair sums (hi, lo) per coordinate
    float2 px = ff_add(make_float2(a.x, 0.f), make_float2(b2.x, 0.f));
    float2 py = ff_add(make_float2(a.y, 0.f), make_float2(b2.y, 0.f));
    float2 ix = px, iy = py;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float2 tx = make_float2(__shfl_up_sync(0xffffffffu, ix.x, o),
                                    __shfl_up_sync(0xffffffffu, ix.y, o));
      const float2 ty = make_float2(__shfl_up_sync(0xffffffffu, iy.x, o),
                                    __shfl_up_sync(0xffffffffu, iy.y, o));
      if (lane >= o) { ix = ff_add(ix, tx); iy = ff_add(iy, ty); }
    }
    float4* wsum = reinterpret_cast<float4*>(red);  // 32 warp totals (red holds 96 doubles)
    __syncthreads();
    if (lane == 31) wsum[warp] = make_float4(ix.x, ix.y, iy.x, iy.y);
    __syncthreads();
    float2 wx = make_float2(0.f, 0.f), wy = make_float2(0.f, 0.f);
    for (int w = 0; w < warp; ++w) {
      const float4 t = wsum[w];
      wx = ff_add(wx, make_float2(t.x, t.y));
      wy = ff_add(wy, make_float2(t.z, t.w));
    }
    // exclusive prefix of this pair = warp offset + inclusive - own pair
    const float2 ex = ff_add(wx, ff_add(ix, make_float2(-px.x, -px.y)));
    const float2 ey = ff_add(wy, ff_add(iy, make_float2(-py.x, -py.y)));
    const float2 ax = ff_add(ex, make_float2(a.x, 0.f)), ay = ff_add(ey, make_float2(a.y, 0.f));
    if (i0 < n) s.P[i0] = make_float4(ex.x, ey.x, ex.y, ey.y);
    if (i0 + 1 < n) s.P[i0 + 1] = make_float4(ax.x, ay.x, ax.y, ay.y);
    // the owner of the last element writes the total
    if (i0 == n - 1) s.P[n] = make_float4(ax.x, ay.x, ax.y, ay.y);
    if (i0 + 1 == n - 1) {
      const float2 tx = ff_add(ex, px), ty = ff_add(ey, py);
      s.P[n] = make_float4(tx.x, ty.x, tx.y, ty.y);
    }
  }
  __syncthreads();
  MM_STAMP(5);
  // node records
  for (int id = tid; id < 2 * n - 1; id += kT) {
    if (id >= n - 1) {
      const int j = id - (n - 1);
      if (n > 1 && s.delta[s.parent[id]] >= 32) continue;  // inside a bucket
      const float2 p = s.xs[j];
      s.nodeA[id] = make_float4(p.x, p.y, 0.f, 1.f);
      s.nodeB[id] = make_short4(-1, (short)s_escape(s, n, j), (short)j, (short)(j + 1));
      continue;
    }
    const int dd = s.delta[id];
    const int dp = id == 0 ? -1 : s.delta[s.parent[id]];
    int depth, first;
    if (dd >= 32) {
      if (dp >= 32) continue;
      depth = kKeyBits;
      first = -1;
    } else {
      if (dp >= 0 && (dp >> 1) == (dd >> 1)) continue;
      depth = dd >> 1;
      first = s_resolve(s, n, s.left[id]);
    }
    const int a = s.lo[id], b = s.hi[id];
    // a cell of at most `leaf` points is a leaf: opened, it is summed exactly
    if (b - a + 1 <= leaf) first = -1;
    const float cnt = (float)(b - a + 1);
    const float4 pa = s.P[a], pb = s.P[b + 1];
    const float2 dx = ff_add(make_float2(pb.x, pb.z), make_float2(-pa.x, -pa.z));
    const float2 dy = ff_add(make_float2(pb.y, pb.w), make_float2(-pa.y, -pa.w));
    const float w = ldexpf(root.z, -depth);
    const float rc = theta > 0.f ? (w / theta) * (w / theta) : CUDART_INF_F;
    s.nodeA[id] = make_float4((dx.x + dx.y) / cnt, (dy.x + dy.y) / cnt, rc, cnt);
    s.nodeB[id] = make_short4((short)first, (short)s_escape(s, n, b), (short)a, (short)(b + 1));
  }
  __syncthreads();
}

// Group acceptance over the shared-memory records: the task's 32 points
// accept a cell only when all of them pass the per-point test (the same rule
// as the multi-kernel group walk); the walk is uniform across the warp.
//
// A CTA has few tasks (about 4) and 32 warps, so W warps share a task: the
// task's first warp walks the tree, recording opened cells of at most
// kSmallSeedPts points as seeds instead of entering them; the W warps then
// walk the seed subtrees (seed j by warp j mod W) and their partial sums are
// added in warp order.  Every cell gets the decision of a single walk.  The
// seeds and partial sums live in the radix-tree arrays, which are dead
// between the record build and the next sweep.
constexpr int kSmallSeedMax = 64;
constexpr int kSmallSeedPts = 64;

__device__ __forceinline__ void walk_cells(const SmallSmem& s, int n, int cur, int stop,
                                           float2 xu, int pos, bool valid, float& fx, float& fy,
                                           int& budget, int* err, int* seeds, int* nseeds) {
  const int lane = threadIdx.x & 31;
  while (cur != stop && cur >= 0) {
    if (cur >= 2 * n - 1 || --budget < 0) {
      if (lane == 0) atomicOr(err, 1);
      return;
    }
    const float4 A = s.nodeA[cur];
    const short4 B = s.nodeB[cur];
    const float dx = xu.x - A.x, dy = xu.y - A.y;
    const float q = fmaf(dx, dx, dy * dy);
    const bool far = !valid || ((pos < B.z || pos >= B.w) && q > A.z);
    if (__all_sync(0xffffffffu, far)) {
      const float sc = __fdividef(A.w, q);
      fx = fmaf(sc, dx, fx);
      fy = fmaf(sc, dy, fy);
      cur = B.y;
    } else if (B.x < 0) {
      const int pb = max((int)B.z, 0), pe = min((int)B.w, n);
      for (int p = pb; p < pe; ++p) {
        const float2 xv = s.xs[p];
        const float ex = xu.x - xv.x, ey = xu.y - xv.y;
        const float eq = fmaf(ex, ex, ey * ey);
        if (p != pos && eq > 0.f) {
          const float inv = __fdividef(1.f, eq);
          fx = fmaf(inv, ex, fx);
          fy = fmaf(inv, ey, fy);
        }
      }
      cur = B.y;
    } else if (seeds && (int)B.w - (int)B.z <= kSmallSeedPts && *nseeds < kSmallSeedMax) {
      if (lane == 0) seeds[*nseeds] = cur;
      __syncwarp();
      if (lane == 0) *nseeds += 1;
      __syncwarp();
      cur = B.y;
    } else {
      cur = B.x;
    }
  }
}

// The seeds are dealt to kSmallVirt seed groups (seed j to group j mod 8);
// each group's walks are added in seed order and the groups in a fixed
// binary tree, ((g0 + g1) + (g2 + g3)) + ((g4 + g5) + (g6 + g7)), plus the
// first warp's own partial sum.  A warp of a W-warp task takes 8 / W
// consecutive groups and adds its complete subtree; the task's first warp
// adds the W subtotals with the rest of the tree.  The forces are therefore
// the same bits for every W: in a cluster launch (few tasks per CTA, W up
// to 8) and in the one-CTA batched launch (many tasks, W = 1).
constexpr int kSmallVirt = 8;

__device__ __forceinline__ float2 f2add(float2 a, float2 b) {
  return make_float2(a.x + b.x, a.y + b.y);
}

// In place: acc[0] = the complete pairwise tree over acc[0 .. width).
__device__ __forceinline__ void tree_sum(float2 (&acc)[kSmallVirt], int width) {
#pragma unroll
  for (int w = kSmallVirt; w > 1; w >>= 1) {
    if (w <= width) {
#pragma unroll
      for (int q = 0; q < kSmallVirt / 2; ++q)
        if (2 * q + 1 < w) acc[q] = f2add(acc[2 * q], acc[2 * q + 1]);
    }
  }
}

__device__ void walk_group(SmallSmem& s, int n, float2* F, int* err, int crank, int csize) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kWarps = kT / 32;
  const int nt = (n + 31) / 32;
  const int mine = crank < nt ? (nt - 1 - crank) / csize + 1 : 0;  // my tasks
  int W = 1;
  while (W < kSmallVirt && 2 * W * mine <= kWarps) W <<= 1;
  const int slots = kWarps / W, slot = warp / W, sub = warp % W;
  const int vper = kSmallVirt / W;  // seed groups per warp
  // scratch in the (dead) radix-tree arrays, 16-byte aligned
  unsigned char* scr = reinterpret_cast<unsigned char*>(
      ((uintptr_t)reinterpret_cast<unsigned char*>(s.lo) + 15) & ~(uintptr_t)15);
  float2(*part)[32] = reinterpret_cast<float2(*)[32]>(scr);            // [32 warps][32]
  int* seeds = reinterpret_cast<int*>(scr + sizeof(float2) * kWarps * 32) + slot * kSmallSeedMax;
  int* nseeds = reinterpret_cast<int*>(scr + sizeof(float2) * kWarps * 32) +
                kWarps * kSmallSeedMax + slot;
  for (int t0 = 0; t0 < mine; t0 += slots) {  // rounds: the same count in every warp
    const bool live = t0 + slot < mine;
    const int task = crank + csize * (t0 + slot);
    const int pos = task * 32 + lane;
    const bool valid = live && pos < n;
    const float2 xu = valid ? s.xs[pos] : make_float2(0.f, 0.f);
    float2 top = make_float2(0.f, 0.f);
    int budget = 2 * n + 2;
    if (sub == 0 && live) {
      if (lane == 0) *nseeds = 0;
      __syncwarp();
      walk_cells(s, n, n > 1 ? 0 : -1, -1, xu, pos, valid, top.x, top.y, budget, err, seeds,
                 nseeds);
    }
    __syncthreads();
    const int ns = live ? *nseeds : 0;
    float2 acc[kSmallVirt];
#pragma unroll
    for (int q = 0; q < kSmallVirt; ++q) acc[q] = make_float2(0.f, 0.f);
    for (int j = 0; j < ns; ++j) {
      const int v = j % kSmallVirt;
      if (v / vper != sub) continue;
      const int c = seeds[j];
      float2 t = make_float2(0.f, 0.f);
      walk_cells(s, n, c, s.nodeB[c].y, xu, pos, valid, t.x, t.y, budget, err, nullptr, nullptr);
      const int q = v - sub * vper;
#pragma unroll
      for (int qq = 0; qq < kSmallVirt; ++qq)
        if (qq == q) acc[qq] = f2add(acc[qq], t);
    }
    tree_sum(acc, vper);
    float2 total = acc[0];
    if (W > 1) {
      part[warp][lane] = total;
      __syncthreads();
      if (sub == 0) {
        float2 w8[kSmallVirt];
#pragma unroll
        for (int q = 0; q < kSmallVirt; ++q)
          w8[q] = q < W ? part[slot * W + q][lane] : make_float2(0.f, 0.f);
        tree_sum(w8, W);
        total = w8[0];
      }
    }
    if (sub == 0 && valid) F[s.vals[pos]] = f2add(top, total);
    __syncthreads();  // seeds and partial sums are reused next round
  }
}

// The per-point walk over the shared-memory records.  Task t = the 32 sorted
// positions [32t, 32t + 32); CTA `crank` of a cluster of `csize` takes the
// tasks t = crank (mod csize), its warps take those round robin.
__device__ void walk(const SmallSmem& s, int n, float2* F, int* err, int crank, int csize) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int task = crank + csize * warp; task * 32 < n; task += csize * (kT / 32)) {
    const int pos = task * 32 + lane;
    const bool valid = pos < n;
    const float2 xu = valid ? s.xs[pos] : make_float2(0.f, 0.f);
    int wait = valid ? kNone : -1;
    int cur = n > 1 ? 0 : -1;
    int budget = 2 * n + 2;
    float fx = 0.f, fy = 0.f;
    while (cur >= 0) {
      if (cur >= 2 * n - 1 || --budget < 0) {
        if (lane == 0) atomicOr(err, 1);
        break;
      }
      const float4 A = s.nodeA[cur];
      const short4 B = s.nodeB[cur];
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
        } else if (B.x < 0) {
          const int pb = max((int)B.z, 0), pe = min((int)B.w, n);
          for (int p = pb; p < pe; ++p) {
            if (p == pos) continue;
            const float2 xv = s.xs[p];
            const float ex = xu.x - xv.x, ey = xu.y - xv.y;
            const float eq = fmaf(ex, ex, ey * ey);
            if (eq > 0.f) {
              const float inv = __fdividef(1.f, eq);
              fx = fmaf(inv, ex, fx);
              fy = fmaf(inv, ey, fy);
            }
          }
          wait = B.y;
        } else {
          desc = true;
        }
      }
      cur = __any_sync(0xffffffffu, desc) ? B.x : B.y;
    }
    if (valid) F[s.vals[pos]] = make_float2(fx, fy);
  }
}

// Barrier over the CTAs of the cluster (a CTA barrier for a cluster of one)
// with release/acquire semantics: global and shared memory written before it
// by any thread of the cluster is visible to every thread after it.
__device__ __forceinline__ void cluster_sync(int csize) {
  if (csize == 1) {
    __syncthreads();
    return;
  }
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// One level's schedule on the `csize` CTAs of a cluster (csize = 1: one
// CTA).  Every CTA stages all positions and builds the same tree; CTA crank
// walks and updates the vertices of its tasks, writing their new positions
// and per-vertex partial sums to global memory; CTA 0 reduces the partials
// in vertex order (the same order for every cluster size, so the schedule's
// decisions do not depend on it) and takes the schedule step.
__device__ __forceinline__ void run_level(const SmallArgs& a, int crank, int csize) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmallSmem& s = *reinterpret_cast<SmallSmem*>(smem_raw);
  __shared__ double red[96];
  __shared__ float4 root;
  __shared__ int sh_done;
  // every CTA keeps its own copy of the schedule state and takes the same
  // (deterministic) steps on it; CTA 0 writes it back at the end
  __shared__ SweepState lst;
  const int n = a.n, tid = threadIdx.x;
  if (tid == 0) lst = *a.st;
  float2* F = s.F;
  for (int i = tid; i <= n; i += kT) s.sp[i] = a.sp[i];
  for (int i = tid; i < n; i += kT) s.rho[i] = a.rho[i];
  const int nt = (n + 31) / 32;                                // tasks
  const int mine = crank < nt ? ((nt - 1 - crank) / csize + 1) * 32 : 0;  // my positions
  for (int sweep = 0;; ++sweep) {
    if (tid == 0 && sweep == 0 && a.prof && crank == 0) a.prof[0] = clock64();
    __syncthreads();
    const float2* xg = lst.parity ? a.b1 : a.b0;
    float2* xo = lst.parity ? a.b0 : a.b1;
    const float alpha = (float)lst.alpha;
    // per-vertex partial sums alternate between two buffers: a CTA that
    // runs ahead into the next sweep cannot overwrite sums still being read
    float4* part = a.part + (sweep & 1) * kSmallMaxN;
    for (int i = tid; i < n; i += kT) s.xv[i] = __ldcg(&xg[i]);
    __syncthreads();
    const float2* x = s.xv;
    long long* prof = (sweep == 0 && crank == 0) ? a.prof : nullptr;
    MM_STAMP(1);
    if (a.exact) {
      // no tree: the build stamps coincide, the sum is the "walk" interval
      MM_STAMP(2);
      MM_STAMP(3);
      MM_STAMP(4);
      MM_STAMP(5);
      MM_STAMP(6);
      const int lane = tid & 31, warp = tid >> 5;
      for (int task = crank + csize * warp; task * 32 < n; task += csize * (kT / 32)) {
        const int u = task * 32 + lane;
        if (u >= n) continue;
        const float2 xu = x[u];
        float fx = 0.f, fy = 0.f;
        for (int k = 0; k < n; ++k) {
          const float dx = xu.x - x[k].x, dy = xu.y - x[k].y;
          const float q = fmaf(dx, dx, dy * dy);
          const float inv = q > 0.f ? __fdividef(1.f, q) : 0.f;
          fx = fmaf(inv, dx, fx);
          fy = fmaf(inv, dy, fy);
        }
        F[u] = make_float2(fx, fy);
      }
    } else {
      build_tree(s, n, a.theta, a.leaf, &root, red, prof);
      MM_STAMP(6);
      if (a.group)
        walk_group(s, n, F, a.err, crank, csize);
      else
        walk(s, n, F, a.err, crank, csize);
    }
    __syncthreads();
    MM_STAMP(7);
    // Eq. 2 over S for my positions: G lanes per row (G = a.lanes, a power
    // of two <= 32), positions, row pointers and rho from shared memory
    {
      const int G = a.lanes;
      const int lg = tid & (G - 1);
      for (int base = 0; base < mine; base += kT / G) {
        const int j = base + tid / G;
        const int pos = (crank + csize * (j >> 5)) * 32 + (j & 31);
        const bool ok = j < mine && pos < n;
        const int u = ok ? (a.exact ? pos : (int)s.vals[pos]) : 0;
        float gx = 0.f, gy = 0.f, rx = 0.f, ry = 0.f, st = 0.f;
        float2 xu = make_float2(0.f, 0.f);
        if (ok) {
          xu = x[u];
          const int e1 = s.sp[u + 1];
#pragma unroll 4
          for (int e = s.sp[u] + lg; e < e1; e += G) {
            const SEnt en = a.S[e];
            const float2 xw = x[en.col];
            const float dx = xu.x - xw.x, dy = xu.y - xw.y;
            const float q = fmaf(dx, dx, dy * dy);
            const float inv = q > 0.f ? rsqrtf(q) : 0.f;
            const float dist = q * inv;
            const float w = __fdividef(1.f, en.d * en.d);
            const float du = en.d * inv;
            gx = fmaf(w, fmaf(du, dx, xw.x), gx);
            gy = fmaf(w, fmaf(du, dy, xw.y), gy);
            const float inv2 = inv * inv;
            rx = fmaf(dx, inv2, rx);
            ry = fmaf(dy, inv2, ry);
            const float t = dist - en.d;
            st = fmaf(w * t, t, st);
          }
        }
        for (int o = G >> 1; o; o >>= 1) {
          gx += __shfl_xor_sync(0xffffffffu, gx, o);
          gy += __shfl_xor_sync(0xffffffffu, gy, o);
          rx += __shfl_xor_sync(0xffffffffu, rx, o);
          ry += __shfl_xor_sync(0xffffffffu, ry, o);
          st += __shfl_xor_sync(0xffffffffu, st, o);
        }
        if (ok && lg == 0) {
          const float2 f = F[u];
          const float r = s.rho[u];
          const float nx = (gx + alpha * (f.x - rx)) / r;
          const float ny = (gy + alpha * (f.y - ry)) / r;
          xo[u] = make_float2(nx, ny);
          const float ddx = nx - xu.x, ddy = ny - xu.y;
          part[u] = make_float4(fmaf(ddx, ddx, ddy * ddy), fmaf(xu.x, xu.x, xu.y * xu.y),
                                0.5f * st, 0.f);
        }
      }
    }
    cluster_sync(csize);  // every new position and partial is written
    MM_STAMP(8);
    {
      // the same reduction, in vertex order, in every CTA
      float psdx = 0.f, psx = 0.f, psst = 0.f;
      for (int u = tid; u < n; u += kT) {
        const float4 q = __ldcg(&part[u]);
        psdx += q.x;
        psx += q.y;
        psst += q.z;
      }
      double tot[3];
      bsum3(psdx, psx, psst, red, tot);
      if (tid == 0) {
        const bool done = schedule_step(&lst, a.sched, tot[0], tot[1], tot[2],
                                        crank == 0 ? a.trace : nullptr, a.trace_cap,
                                        crank == 0 ? a.lsw : nullptr);
        sh_done = (done || sweep + 1 >= a.max_sweeps) ? 1 : 0;
      }
    }
    __syncthreads();
    MM_STAMP(9);
    if (sh_done) break;
  }
  if (crank == 0 && tid == 0) *a.st = lst;
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

// One level on one cluster (the grid is one cluster; a plain launch is a
// cluster of one CTA).
__global__ void __launch_bounds__(kT, 1) small_level_kernel(SmallArgs a) {
  run_level(a, (int)cluster_rank(), (int)cluster_size());
}

// Batched form: CTA b runs the level described by args[b] (one graph each).
__global__ void __launch_bounds__(kT, 1) small_level_batch_kernel(const SmallArgs* args) {
  const SmallArgs a = args[blockIdx.x];
  run_level(a, 0, 1);
}

int g_max_cluster = 0;  // largest cluster the fused kernel can be launched with

}  // namespace

static_assert(sizeof(SmallSmem) + 1024 <= 227 * 1024, "fused level kernel exceeds shared memory");
// the walk's scratch (partial sums of 32 warps, seeds of up to 32 task slots
// and their counts, 16-byte alignment slack) fits the radix-tree arrays
static_assert(15 + sizeof(float2) * 32 * 32 + sizeof(int) * (32 * kSmallSeedMax + 32) <=
                  5 * sizeof(int16_t) * kN,
              "walk scratch exceeds the radix-tree arrays");

size_t small_level_smem() { return sizeof(SmallSmem); }

int small_level_max_cluster() { return g_max_cluster > 0 ? g_max_cluster : 1; }

mm_status small_level_setup() {
  MM_CK(cudaFuncSetAttribute(small_level_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SmallSmem)));
  MM_CK(cudaFuncSetAttribute(small_level_batch_kernel,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SmallSmem)));
  if (g_max_cluster == 0) {
    // 16 CTAs (one per SM: the shared memory allows one) if a GPC can hold
    // such a cluster, else the portable 8
    int best = 1;
    if (cudaFuncSetAttribute(small_level_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed,
                             1) == cudaSuccess) {
      for (int c : {16, 8, 4, 2}) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = c;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(kT);
        cfg.dynamicSmemBytes = sizeof(SmallSmem);
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, small_level_kernel, &cfg) == cudaSuccess &&
            clusters > 0) {
          best = c;
          break;
        }
      }
    }
    cudaGetLastError();  // a refused query leaves no error behind
    g_max_cluster = best;
  }
  return MM_OK;
}

mm_status small_level_batch(const SmallArgs* dev_args, int count, cudaStream_t s) {
  if (count <= 0) return MM_OK;
  small_level_batch_kernel<<<count, kT, sizeof(SmallSmem), s>>>(dev_args);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

mm_status small_level(const SmallArgs& a, cudaStream_t s) {
  if (a.n < 1 || a.n > kSmallMaxN) {
    set_error("fused level kernel takes 1..%d vertices, got %d", kSmallMaxN, a.n);
    return MM_ERR_INVALID_ARG;
  }
  const int c = std::max(1, std::min(a.cluster, small_level_max_cluster()));
  if (c == 1) {
    small_level_kernel<<<1, kT, sizeof(SmallSmem), s>>>(a);
  } else {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = c;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kT);
    cfg.dynamicSmemBytes = sizeof(SmallSmem);
    cfg.stream = s;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    MM_CK(cudaLaunchKernelEx(&cfg, small_level_kernel, a));
  }
  MM_CK(cudaGetLastError());
  return MM_OK;
}

}  // namespace mm
