// One Jacobi iteration of Eq. 2 over the pair set S, fused with the
// reductions the alpha schedule needs, plus the device-side schedule
// controller, prolongation and the initial layout.
//
//   x'_u = ( sum_{v in S_u} w_uv (x_v + d_uv (x_u - x_v)/|x_u - x_v|)
//          + alpha (F_u - sum_{v in S_u} r(u,v)) ) / rho_u
//
// with F_u the Barnes-Hut (or exact) sum of r(u,v) over all v != u, so that
// F_u - sum_S r is the entropy sum over the pairs outside S (Eq. 2; the
// subtraction is the one of Eq. 3).  The kernel streams the CSR of S once:
// G lanes cooperate on one row (G chosen from the mean row length so a row
// is read as consecutive 8-byte entries), rows longer than a threshold are
// handled by a whole block each, and per-block FP32 partials of
// sum|x'-x|^2, sum|x|^2 and the stress, added in float-float, feed the
// controller.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>

#include "mm_internal.cuh"

namespace mm {

namespace {

struct RowAcc {
  float gx, gy, sx, sy, st;
};

__device__ __forceinline__ void accumulate_v(RowAcc& a, float2 xu, SEnt en, float2 xv) {
  const float dx = xu.x - xv.x, dy = xu.y - xv.y;
  const float q = fmaf(dx, dx, dy * dy);
  const float inv = q > 0.f ? rsqrtf(q) : 0.f;   // 1/|x_u - x_v|, 0 if coincident
  const float dist = q * inv;
  const float w = __fdividef(1.f, en.d * en.d);
  const float du = en.d * inv;                    // d / |x_u - x_v|
  a.gx = fmaf(w, fmaf(du, dx, xv.x), a.gx);
  a.gy = fmaf(w, fmaf(du, dy, xv.y), a.gy);
  const float inv2 = inv * inv;
  a.sx = fmaf(dx, inv2, a.sx);
  a.sy = fmaf(dy, inv2, a.sy);
  const float t = dist - en.d;
  a.st = fmaf(w * t, t, a.st);
}

__device__ __forceinline__ void accumulate(RowAcc& a, float2 xu, SEnt en, const float2* x) {
  accumulate_v(a, xu, en, __ldg(&x[en.col]));
}

// Entries b + lg, b + lg + G, ... < e of one S row, four at a time: the four
// entry loads, then the four position loads, are issued back to back (the
// row -> entry -> position chain is three dependent loads; batching them
// keeps four of each in flight per lane).  Same order of additions as one
// entry at a time.
template <int G>
__device__ __forceinline__ void accumulate_row(RowAcc& a, float2 xu, const SEnt* __restrict__ S,
                                               int b, int e, int lg, const float2* x) {
  constexpr int kU = 4;
  for (int k0 = b + lg; k0 < e; k0 += kU * G) {
    SEnt en[kU];
    float2 xv[kU];
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      const int k = k0 + j * G;
      en[j] = k < e ? S[k] : SEnt{0, 1.f};
    }
#pragma unroll
    for (int j = 0; j < kU; ++j)
      xv[j] = k0 + j * G < e ? __ldg(&x[en[j].col]) : make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < kU; ++j)
      if (k0 + j * G < e) accumulate_v(a, xu, en[j], xv[j]);
  }
}

// Bounding box accumulator (starts empty: min = +huge, max = -huge).
struct Box {
  float x0, y0, x1, y1;
  __device__ Box() : x0(3.0e38f), y0(3.0e38f), x1(-3.0e38f), y1(-3.0e38f) {}
  __device__ void add(float x, float y) {
    x0 = fminf(x0, x); y0 = fminf(y0, y); x1 = fmaxf(x1, x); y1 = fmaxf(y1, y);
  }
};

__device__ __forceinline__ void finish_vertex(int u, const RowAcc& a, float2 xu, float alpha,
                                              const float* rho, const float2* F, float2* xo,
                                              float& s_dx, float& s_x, float& s_st, Box& box) {
  const float2 f = F[u];
  const float r = rho[u];
  const float nx = (a.gx + alpha * (f.x - a.sx)) / r;
  const float ny = (a.gy + alpha * (f.y - a.sy)) / r;
  xo[u] = make_float2(nx, ny);
  box.add(nx, ny);
  const float ddx = nx - xu.x, ddy = ny - xu.y;
  s_dx = fmaf(ddx, ddx, fmaf(ddy, ddy, s_dx));
  s_x = fmaf(xu.x, xu.x, fmaf(xu.y, xu.y, s_x));
  s_st = fmaf(0.5f, a.st, s_st);
}

// Per-thread FP32 partials -> block totals in FP32 (warp shuffles, then the
// warp totals in warp 0); a block adds a few thousand terms at most, the
// blocks' totals are added in float-float by the last block.  Result in
// thread 0.
template <int kT>
__device__ __forceinline__ float4 block_sum3(float a, float b, float c) {
  __shared__ float sh[3][kT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if (lane == 0) { sh[0][warp] = a; sh[1][warp] = b; sh[2][warp] = c; }
  __syncthreads();
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
  if (warp == 0) {
    a = lane < kT / 32 ? sh[0][lane] : 0.f;
    b = lane < kT / 32 ? sh[1][lane] : 0.f;
    c = lane < kT / 32 ? sh[2][lane] : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    r = make_float4(a, b, c, 0.f);
  }
  return r;
}

// Float-float sums of per-block totals parts[0 .. nparts), each thread
// taking every kT-th block, then the block tree.  Result in thread 0.
template <int kT>
__device__ __forceinline__ void sum_parts(const float4* parts, int nparts, double out[3]) {
  float2 a = make_float2(0.f, 0.f), b = a, c = a;
  for (int i = threadIdx.x; i < nparts; i += kT) {
    const float4 q = __ldcg(&parts[i]);
    a = ff_add(a, make_float2(q.x, 0.f));
    b = ff_add(b, make_float2(q.y, 0.f));
    c = ff_add(c, make_float2(q.z, 0.f));
  }
  block_ffsum3<kT>(a, b, c, out);
}

template <int kT>
__device__ __forceinline__ float4 block_box(Box b) {
  __shared__ float4 sh[kT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    b.x0 = fminf(b.x0, __shfl_xor_sync(0xffffffffu, b.x0, o));
    b.y0 = fminf(b.y0, __shfl_xor_sync(0xffffffffu, b.y0, o));
    b.x1 = fmaxf(b.x1, __shfl_xor_sync(0xffffffffu, b.x1, o));
    b.y1 = fmaxf(b.y1, __shfl_xor_sync(0xffffffffu, b.y1, o));
  }
  __syncthreads();
  if (lane == 0) sh[warp] = make_float4(b.x0, b.y0, b.x1, b.y1);
  __syncthreads();
  float4 r = sh[0];
  for (int w = 1; w < kT / 32; ++w) {
    r.x = fminf(r.x, sh[w].x); r.y = fminf(r.y, sh[w].y);
    r.z = fmaxf(r.z, sh[w].z); r.w = fmaxf(r.w, sh[w].w);
  }
  return r;
}

// End of an update launch: the block publishes its partial sums (and the
// bounding box of the positions it wrote); with `epi` set, the last block to
// arrive reduces all nparts partials in block order and takes the schedule
// step (Sec. 3.2), and -- with a box buffer -- writes the next sweep's root
// square, zeroes the sort state and starts a new look-back epoch, so the
// next sweep needs no separate controller or bounding-box launch.
template <int kT>
__device__ void update_tail(float s_dx, float s_x, float s_st, const Box& box, float4* parts,
                            int part_off, int nparts, int epi, const SweepEpilogue& ep) {
  __shared__ bool last;
  const float4 tot = block_sum3<kT>(s_dx, s_x, s_st);
  float4 bb = make_float4(0.f, 0.f, 0.f, 0.f);
  if (ep.box) bb = block_box<kT>(box);
  if (threadIdx.x == 0) {
    parts[part_off + blockIdx.x] = tot;
    if (ep.box) ep.box[part_off + blockIdx.x] = bb;
    if (epi) {
      __threadfence();
      last = atomicAdd(ep.arrive, 1u) == gridDim.x - 1;
    }
  }
  if (!epi) return;
  __syncthreads();
  if (!last) return;
  __threadfence();
  float4 r = make_float4(CUDART_INF_F, CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F);
  if (ep.box) {
    for (int i = threadIdx.x; i < nparts; i += kT) {
      const float4 q = __ldcg(&ep.box[i]);
      r.x = fminf(r.x, q.x); r.y = fminf(r.y, q.y);
      r.z = fmaxf(r.z, q.z); r.w = fmaxf(r.w, q.w);
    }
  }
  double out[3];
  sum_parts<kT>(parts, nparts, out);
  if (ep.box) {
    Box q;
    q.x0 = r.x; q.y0 = r.y; q.x1 = r.z; q.y1 = r.w;
    const float4 w = block_box<kT>(q);
    for (int i = threadIdx.x; i < 4 * 256; i += kT) ep.hist[i] = 0u;
    if (threadIdx.x < 4) ep.counters[threadIdx.x] = 0u;
    if (threadIdx.x == 0) {
      const float side = fmaxf(w.z - w.x, w.w - w.y);
      *ep.root = make_float4(w.x, w.y, side, side > 0.f ? 65536.0f / side : 0.f);
      ep.tree_ticket[0] = 0u;
      ep.tree_ticket[1] += 1u;
    }
  }
  if (threadIdx.x == 0) {
    const bool done = schedule_step(ep.st, ep.sp, out[0], out[1], out[2], ep.trace,
                                    ep.trace_cap, ep.lsw);
    if (ep.use_h) cudaGraphSetConditional(ep.h, done ? 0u : 1u);
    *ep.arrive = 0u;
  }
}

// G lanes per vertex; rows with more than `heavy` entries are skipped here.
// kMode 0: the whole update (sum over S_u, new position, reductions).
// kMode 1: only the sum over S_u, stored per vertex in acc/acc_st (it needs
//   nothing but x, so it can run beside the tree build and the walk).
// kMode 2: the rest of the update from acc/acc_st.  Grid, vertex-to-thread
//   assignment and arithmetic are those of kMode 0, so modes 1 + 2 give
//   bit-identical positions, partial sums and schedule steps.
template <int G, int kMode>
__global__ void __launch_bounds__(kGatherThreads) gather_light(
    int n, const int32_t* __restrict__ sp, const SEnt* __restrict__ S,
    const float* __restrict__ rho, XSel xs, const float2* __restrict__ F,
    const SweepState* st, int heavy, float4* partials, int nparts, int epi, SweepEpilogue ep,
    float4* __restrict__ acc, float* __restrict__ acc_st) {
  const float2* x = xs.cur();
  float2* xo = xs.next();
  const float alpha = kMode == 1 ? 0.f : (float)st->alpha;
  constexpr int kGroups = kGatherThreads / G;
  const int g = threadIdx.x / G, lg = threadIdx.x % G;
  float s_dx = 0.f, s_x = 0.f, s_st = 0.f;
  Box box;
  for (int base = blockIdx.x * kGroups; base < n; base += gridDim.x * kGroups) {
    const int u = base + g;
    RowAcc a = {0.f, 0.f, 0.f, 0.f, 0.f};
    bool mine = false;
    float2 xu = make_float2(0.f, 0.f);
    if (u < n) {
      const int b = sp[u], e = sp[u + 1];
      if (e - b <= heavy) {
        mine = true;
        xu = x[u];
        if (kMode != 2) accumulate_row<G>(a, xu, S, b, e, lg, x);
      }
    }
    if (kMode != 2 && G > 1) {
#pragma unroll
      for (int o = G / 2; o; o >>= 1) {
        a.gx += __shfl_xor_sync(0xffffffffu, a.gx, o);
        a.gy += __shfl_xor_sync(0xffffffffu, a.gy, o);
        a.sx += __shfl_xor_sync(0xffffffffu, a.sx, o);
        a.sy += __shfl_xor_sync(0xffffffffu, a.sy, o);
        a.st += __shfl_xor_sync(0xffffffffu, a.st, o);
      }
    }
    if (mine && lg == 0) {
      if (kMode == 1) {
        acc[u] = make_float4(a.gx, a.gy, a.sx, a.sy);
        acc_st[u] = a.st;
      } else {
        if (kMode == 2) {
          const float4 q = acc[u];
          a = RowAcc{q.x, q.y, q.z, q.w, acc_st[u]};
        }
        finish_vertex(u, a, xu, alpha, rho, F, xo, s_dx, s_x, s_st, box);
      }
    }
  }
  if (kMode != 1) update_tail<kGatherThreads>(s_dx, s_x, s_st, box, partials, 0, nparts, epi, ep);
}

// One block per heavy row (power-law hubs); kMode as for gather_light.
template <int kMode>
__global__ void __launch_bounds__(kGatherThreads) gather_heavy(
    const int32_t* __restrict__ heavy_list, int n_heavy, const int32_t* __restrict__ sp,
    const SEnt* __restrict__ S, const float* __restrict__ rho, XSel xs,
    const float2* __restrict__ F, const SweepState* st, float4* partials, int part_off,
    int nparts, int epi, SweepEpilogue ep, float4* __restrict__ acc, float* __restrict__ acc_st) {
  const float2* x = xs.cur();
  float2* xo = xs.next();
  const float alpha = kMode == 1 ? 0.f : (float)st->alpha;
  __shared__ float red[5][kGatherThreads / 32];
  float s_dx = 0.f, s_x = 0.f, s_st = 0.f;
  Box box;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int h = blockIdx.x; h < n_heavy; h += gridDim.x) {
    const int u = heavy_list[h];
    const float2 xu = x[u];
    if (kMode == 2) {
      if (threadIdx.x == 0) {
        const float4 q = acc[u];
        const RowAcc t = {q.x, q.y, q.z, q.w, acc_st[u]};
        finish_vertex(u, t, xu, alpha, rho, F, xo, s_dx, s_x, s_st, box);
      }
      continue;
    }
    RowAcc a = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = sp[u] + threadIdx.x; k < sp[u + 1]; k += blockDim.x) accumulate(a, xu, S[k], x);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      a.gx += __shfl_xor_sync(0xffffffffu, a.gx, o);
      a.gy += __shfl_xor_sync(0xffffffffu, a.gy, o);
      a.sx += __shfl_xor_sync(0xffffffffu, a.sx, o);
      a.sy += __shfl_xor_sync(0xffffffffu, a.sy, o);
      a.st += __shfl_xor_sync(0xffffffffu, a.st, o);
    }
    if (lane == 0) {
      red[0][warp] = a.gx; red[1][warp] = a.gy; red[2][warp] = a.sx;
      red[3][warp] = a.sy; red[4][warp] = a.st;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      RowAcc t = {0.f, 0.f, 0.f, 0.f, 0.f};
      for (int w = 0; w < kGatherThreads / 32; ++w) {
        t.gx += red[0][w]; t.gy += red[1][w]; t.sx += red[2][w];
        t.sy += red[3][w]; t.st += red[4][w];
      }
      if (kMode == 1) {
        acc[u] = make_float4(t.gx, t.gy, t.sx, t.sy);
        acc_st[u] = t.st;
      } else {
        finish_vertex(u, t, xu, alpha, rho, F, xo, s_dx, s_x, s_st, box);
      }
    }
    __syncthreads();
  }
  if (kMode != 1)
    update_tail<kGatherThreads>(s_dx, s_x, s_st, box, partials, part_off, nparts, epi, ep);
}

constexpr int kCtlThreads = 256;

// Reduces the per-block partials in a fixed order and advances the alpha
// schedule of Sec. 3.2: at most iters_per_alpha iterations per alpha (fewer
// if the relative change |x'-x|/|x| drops below eps), alpha := max(factor *
// alpha, alpha_min); at alpha_min iterate until the change is below
// eps_final or max_iters_at_min iterations.
__global__ void __launch_bounds__(kCtlThreads) controller_kernel(
    int nparts, const float4* __restrict__ partials, SweepState* st, SchedParams sp,
    float* trace, int trace_cap, int* level_sweeps_out, cudaGraphConditionalHandle h,
    int use_h) {
  double out[3];
  sum_parts<kCtlThreads>(partials, nparts, out);
  if (threadIdx.x != 0) return;
  const bool done = schedule_step(st, sp, out[0], out[1], out[2], trace, trace_cap,
                                  level_sweeps_out);
  if (use_h) cudaGraphSetConditional(h, done ? 0u : 1u);
}

__device__ __forceinline__ float u01(uint32_t z) { return (float)(z >> 8) * (1.0f / 16777216.0f); }

// Random polar placement around the coarse representative (Sec. 3.2).
__global__ void prolong_kernel(int nf, const int32_t* __restrict__ map, XSel xc,
                               const float* __restrict__ cc, uint32_t k0, uint32_t k1,
                               uint32_t level, float2* xf_direct) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nf) return;
  uint32_t z[4];
  philox4x32_10((uint32_t)v, level, 0u, 0u, k0, k1, z);
  const int p = map[v];
  const float2 P = xc.cur()[p];
  const float phi = 6.28318530717958647692f * u01(z[0]);
  const float rad = sqrtf(cc[p]) * u01(z[1]);
  float sn, cs;
  sincosf(phi, &sn, &cs);
  float2* out = xf_direct ? xf_direct : xc.next();
  out[v] = make_float2(fmaf(rad, cs, P.x), fmaf(rad, sn, P.y));
}

// Resets the schedule for a new level; flip = 1 moves to the buffer the
// prolongation just wrote.
__global__ void level_start_kernel(SweepState* st, double alpha0, int flip) {
  st->alpha = alpha0;
  st->it_in_round = 0;
  st->level_sweeps = 0;
  st->done = 0;
  if (flip) st->parity ^= 1;
}

// Initial layout of the coarsest level (Sec. 3.1): one vertex at the origin;
// two vertices at their target distance d (first S entry of vertex 0);
// more than two placed around the origin at radius R = sqrt(sum c).
__global__ void init_coarsest_kernel(int n, const float* __restrict__ c, const SEnt* s0,
                                     uint32_t k0, uint32_t k1, uint32_t level, float R,
                                     float2* x0, SweepState* st, double alpha0) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v == 0) {
    st->parity = 0;
    st->alpha = alpha0;
    st->it_in_round = 0;
    st->level_sweeps = 0;
    st->done = 0;
  }
  if (v >= n) return;
  if (n == 1) {
    x0[0] = make_float2(0.f, 0.f);
  } else if (n == 2) {
    const float D = s0[0].d;
    x0[v] = make_float2(v == 0 ? -0.5f * D : 0.5f * D, 0.f);
  } else {
    uint32_t z[4];
    philox4x32_10((uint32_t)v, level, 1u, 0u, k0, k1, z);
    const float phi = 6.28318530717958647692f * u01(z[0]);
    const float rad = R * u01(z[1]);
    float sn, cs;
    sincosf(phi, &sn, &cs);
    x0[v] = make_float2(rad * cs, rad * sn);
  }
}

__global__ void copy_current_kernel(XSel xs, int n, const int32_t* __restrict__ perm,
                                    float2* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = xs.cur()[perm ? perm[i] : i];
}

template <int G, int kMode>
void launch_light(const Level& L, XSel x, const float2* F, const SweepState* st, float4* partials,
                  int blocks, int nparts, int epi, const SweepEpilogue& ep, float4* acc,
                  float* acc_st, cudaStream_t s) {
  gather_light<G, kMode><<<blocks, kGatherThreads, 0, s>>>(L.n, L.sp, L.s, L.rho, x, F, st,
                                                           L.heavy_degree, partials, nparts, epi,
                                                           ep, acc, acc_st);
}

template <int kMode>
mm_status launch_gather(const Level& L, XSel x, const float2* F, const SweepState* st,
                        float4* partials, const SweepEpilogue* epi, float4* acc, float* acc_st,
                        cudaStream_t s) {
  const int lb = gather_light_blocks(L);
  const int hb = gather_heavy_blocks(L);
  const int nparts = lb + hb;
  SweepEpilogue ep{};
  if (epi) ep = *epi;
  // the epilogue runs in the last launch of the update
  const int epi_light = epi && hb == 0 ? 1 : 0;
  switch (L.lanes) {
    case 1: launch_light<1, kMode>(L, x, F, st, partials, lb, nparts, epi_light, ep, acc, acc_st, s); break;
    case 2: launch_light<2, kMode>(L, x, F, st, partials, lb, nparts, epi_light, ep, acc, acc_st, s); break;
    case 4: launch_light<4, kMode>(L, x, F, st, partials, lb, nparts, epi_light, ep, acc, acc_st, s); break;
    case 8: launch_light<8, kMode>(L, x, F, st, partials, lb, nparts, epi_light, ep, acc, acc_st, s); break;
    case 16: launch_light<16, kMode>(L, x, F, st, partials, lb, nparts, epi_light, ep, acc, acc_st, s); break;
    case 32: launch_light<32, kMode>(L, x, F, st, partials, lb, nparts, epi_light, ep, acc, acc_st, s); break;
    default:
      set_error("unsupported lanes per vertex %d", L.lanes);
      return MM_ERR_INVALID_ARG;
  }
  if (hb > 0)
    gather_heavy<kMode><<<hb, kGatherThreads, 0, s>>>(L.heavy, L.n_heavy, L.sp, L.s, L.rho, x, F,
                                                      st, partials, lb, nparts, epi ? 1 : 0, ep,
                                                      acc, acc_st);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

}  // namespace

int gather_light_blocks(const Level& L) {
  const int groups = kGatherThreads / std::max(1, L.lanes);
  return std::max(1, std::min(ceil_div(L.n, groups), 16 * num_sms()));
}

int gather_heavy_blocks(const Level& L) {
  return L.n_heavy > 0 ? std::min(L.n_heavy, 8 * num_sms()) : 0;
}

int gather_blocks(const Level& L) { return gather_light_blocks(L) + gather_heavy_blocks(L); }

mm_status gather_update(const Level& L, XSel x, const float2* F, const SweepState* st,
                        float4* partials, cudaStream_t s, const SweepEpilogue* epi) {
  if (L.n <= 0) return MM_OK;
  return launch_gather<0>(L, x, F, st, partials, epi, nullptr, nullptr, s);
}

mm_status gather_sum(const Level& L, XSel x, float4* acc, float* acc_st, cudaStream_t s) {
  if (L.n <= 0) return MM_OK;
  return launch_gather<1>(L, x, nullptr, nullptr, nullptr, nullptr, acc, acc_st, s);
}

mm_status update_from_sum(const Level& L, XSel x, const float2* F, const float4* acc,
                          const float* acc_st, const SweepState* st, float4* partials,
                          cudaStream_t s, const SweepEpilogue* epi) {
  if (L.n <= 0) return MM_OK;
  return launch_gather<2>(L, x, F, st, partials, epi, const_cast<float4*>(acc),
                          const_cast<float*>(acc_st), s);
}

mm_status controller(int nblocks, const float4* partials, SweepState* st, SchedParams sp,
                     float* trace, int trace_cap, int* level_sweeps_out,
                     cudaGraphConditionalHandle handle, bool use_handle, cudaStream_t s) {
  controller_kernel<<<1, kCtlThreads, 0, s>>>(nblocks, partials, st, sp, trace, trace_cap,
                                              level_sweeps_out, handle, use_handle ? 1 : 0);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

mm_status prolong(int n_fine, const int32_t* map, XSel xc, const float* cc, uint64_t seed,
                  int level, float2* xf_direct, cudaStream_t s) {
  if (n_fine <= 0) return MM_OK;
  prolong_kernel<<<ceil_div(n_fine, 256), 256, 0, s>>>(
      n_fine, map, xc, cc, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32),
      (uint32_t)level, xf_direct);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

mm_status level_start(SweepState* st, double alpha0, int flip, cudaStream_t s) {
  level_start_kernel<<<1, 1, 0, s>>>(st, alpha0, flip);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

mm_status init_coarsest(int n, const float* c, const SEnt* s0, uint64_t seed, int level,
                        float R, float2* x0, SweepState* st, double alpha0, cudaStream_t s) {
  init_coarsest_kernel<<<ceil_div(std::max(n, 1), 256), 256, 0, s>>>(
      n, c, s0, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), (uint32_t)level, R, x0,
      st, alpha0);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

mm_status copy_current(XSel x, int n, float2* out, cudaStream_t s, const int32_t* perm) {
  if (n <= 0) return MM_OK;
  copy_current_kernel<<<ceil_div(n, 256), 256, 0, s>>>(x, n, perm, out);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

}  // namespace mm
