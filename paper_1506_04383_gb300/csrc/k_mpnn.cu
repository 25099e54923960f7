// Learned prolongation: a 3-layer message-passing network (hidden 64) that
// adds a drift to the paper's random polar prolongation (Sec. 3.2,
// "Uncoarsening"):   x_v = x'_p + r_v + o_v,   p = M(v),
//   o_v = beta_0 a_v + beta_1 b_v + beta_2 r_v,
//   beta = head(H_3),  H_l = ReLU([H_{l-1} | mean_N H_{l-1}] W_l + b_l),
// with a_v the mean direction from x'_p to the coarse positions of v's
// neighbours in other clusters, b_v the mean direction from x'_p to p's
// coarse neighbours, r_v the polar offset itself and g_v = x'_p - m (m the
// mean of the coarse layout; beta_3 g is a growth about the centre); the 8
// input scalars are rotation/translation/scale invariant, so o is
// equivariant.
//
// Forward and backward run on the device: the dense layers are tcgen05 BF16
// GEMMs with FP32 accumulation (k_gemm.cu), aggregation / head / loss / ReLU
// masks / weight-gradient reductions / Adam are CUDA-core kernels with FP32
// accumulation.  Parameters are FP32 masters; BF16 copies feed the tensor
// cores (W^T for the forward GEMM, W for the backward one).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "mm_internal.cuh"

namespace mm {

namespace {

constexpr int kH = kNetHidden;   // 64
constexpr int kF = kNetFeatures; // 8
constexpr int kO = kNetOut;      // 4
constexpr int kStatThreads = 1024;

// Mean m and RMS radius S of the coarse layout (one block): FP32 sums per
// thread, FP64 across the block.  stat = (m.x, m.y, S).
__global__ void __launch_bounds__(kStatThreads) net_stat(int nc, XSel xc, float* stat) {
  __shared__ double red[2][kStatThreads / 32];
  __shared__ double mean[2];
  const float2* X = xc.cur();
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  float sx = 0.f, sy = 0.f;
  for (int i = tid; i < nc; i += kStatThreads) {
    const float2 p = X[i];
    sx += p.x;
    sy += p.y;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
  }
  if (lane == 0) {
    red[0][w] = sx;
    red[1][w] = sy;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0, b = 0;
    for (int i = 0; i < kStatThreads / 32; ++i) {
      a += red[0][i];
      b += red[1][i];
    }
    mean[0] = a / nc;
    mean[1] = b / nc;
  }
  __syncthreads();
  const float mx = (float)mean[0], my = (float)mean[1];
  float ss = 0.f;
  for (int i = tid; i < nc; i += kStatThreads) {
    const float2 p = X[i];
    const float dx = p.x - mx, dy = p.y - my;
    ss = fmaf(dx, dx, fmaf(dy, dy, ss));
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  __syncthreads();
  if (lane == 0) red[0][w] = ss;
  __syncthreads();
  if (tid == 0) {
    double a = 0;
    for (int i = 0; i < kStatThreads / 32; ++i) a += red[0][i];
    stat[0] = mx;
    stat[1] = my;
    stat[2] = (float)sqrt(a / nc);
  }
}

// ---------------------------------------------------------------- features
__device__ __forceinline__ float u01f(uint32_t z) { return (float)(z >> 8) * (1.0f / 16777216.0f); }

__global__ void net_features(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const int32_t* __restrict__ map, XSel xc,
                             const int32_t* __restrict__ crp, const int32_t* __restrict__ ccol,
                             const float* __restrict__ cc, const float* __restrict__ stat,
                             uint32_t k0, uint32_t k1, uint32_t level,
                             __nv_bfloat16* __restrict__ f, float2* __restrict__ basis) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const float2* X = xc.cur();
  const int p = map[v];
  const float2 xp = X[p];
  float ax = 0.f, ay = 0.f;
  int cnt = 0;
  const int deg = rp[v + 1] - rp[v];
  for (int e = rp[v]; e < rp[v + 1]; ++e) {
    const int q = map[col[e]];
    if (q == p) continue;
    const float2 xq = X[q];
    ax += xq.x - xp.x;
    ay += xq.y - xp.y;
    ++cnt;
  }
  if (cnt) { ax /= cnt; ay /= cnt; }
  float bx = 0.f, by = 0.f;
  const int cd = crp[p + 1] - crp[p];
  for (int e = crp[p]; e < crp[p + 1]; ++e) {
    const float2 xq = X[ccol[e]];
    bx += xq.x - xp.x;
    by += xq.y - xp.y;
  }
  if (cd) { bx /= cd; by /= cd; }
  uint32_t z[4];
  philox4x32_10((uint32_t)v, level, 0u, 0u, k0, k1, z);
  const float phi = 6.28318530717958647692f * u01f(z[0]);
  const float R = sqrtf(cc[p]);
  const float rad = R * u01f(z[1]);
  float sn, cs;
  sincosf(phi, &sn, &cs);
  const float rx = rad * cs, ry = rad * sn;
  const float na = sqrtf(ax * ax + ay * ay), nb = sqrtf(bx * bx + by * by);
  const float gx = xp.x - stat[0], gy = xp.y - stat[1];
  float g[kF];
  g[0] = sqrtf(gx * gx + gy * gy) / fmaxf(stat[2], 1e-30f);
  g[1] = logf(cc[p]);
  g[2] = log1pf((float)deg);
  g[3] = (float)cnt / (float)max(deg, 1);
  g[4] = na / R;
  g[5] = nb / R;
  g[6] = (ax * bx + ay * by) / (na * nb + 1e-12f);
  g[7] = (ax * rx + ay * ry) / (na * R + 1e-12f);
#pragma unroll
  for (int j = 0; j < kF; ++j) f[(size_t)v * kF + j] = __float2bfloat16_rn(g[j]);
  basis[kO * (size_t)v] = make_float2(ax, ay);
  basis[kO * (size_t)v + 1] = make_float2(bx, by);
  basis[kO * (size_t)v + 2] = make_float2(rx, ry);
  basis[kO * (size_t)v + 3] = make_float2(gx, gy);
}

// Hcat[v] = [H[v] | mean over neighbours of H] (BF16, width 2D), one warp
// per vertex, FP32 accumulation.
template <int D>
__global__ void net_aggregate(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                              const __nv_bfloat16* __restrict__ H, __nv_bfloat16* __restrict__ Hc) {
  const int lane = threadIdx.x & 31;
  const int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (v >= n) return;
  constexpr int P = (D + 31) / 32;  // features per lane
  float acc[P];
#pragma unroll
  for (int j = 0; j < P; ++j) acc[j] = 0.f;
  const int b = rp[v], e = rp[v + 1];
  for (int k = b; k < e; ++k) {
    const int w = col[k];
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const int d = lane + 32 * j;
      if (d < D) acc[j] += __bfloat162float(H[(size_t)w * D + d]);
    }
  }
  const float inv = e > b ? 1.f / (float)(e - b) : 0.f;
#pragma unroll
  for (int j = 0; j < P; ++j) {
    const int d = lane + 32 * j;
    if (d < D) {
      Hc[(size_t)v * 2 * D + d] = H[(size_t)v * D + d];
      Hc[(size_t)v * 2 * D + D + d] = __float2bfloat16_rn(acc[j] * inv);
    }
  }
}

// Head: beta = H3 Wo + bo, o = beta0 a + beta1 b + beta2 r + beta3 g.
// Inference writes x_v = x'_p + r_v + o_v; training also forms the loss
// terms and dbeta = d loss / d beta.
__global__ void net_head(int n, const __nv_bfloat16* __restrict__ H3, const float* __restrict__ Wo,
                         const float* __restrict__ bo, const float2* __restrict__ basis,
                         const int32_t* __restrict__ map, XSel xc, const float* __restrict__ cc,
                         float2* xout, const float2* __restrict__ target, float* dbeta,
                         double* loss_part) {
  __shared__ float w[kH * kO + kO];
  for (int i = threadIdx.x; i < kH * kO + kO; i += blockDim.x)
    w[i] = i < kH * kO ? Wo[i] : bo[i - kH * kO];
  __syncthreads();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (v < n) {
    float beta[kO];
#pragma unroll
    for (int j = 0; j < kO; ++j) beta[j] = w[kH * kO + j];
    for (int d = 0; d < kH; ++d) {
      const float h = __bfloat162float(H3[(size_t)v * kH + d]);
#pragma unroll
      for (int j = 0; j < kO; ++j) beta[j] = fmaf(h, w[d * kO + j], beta[j]);
    }
    float2 e[kO];
#pragma unroll
    for (int j = 0; j < kO; ++j) e[j] = basis[kO * (size_t)v + j];
    float ox = 0.f, oy = 0.f;
#pragma unroll
    for (int j = 0; j < kO; ++j) {
      ox = fmaf(beta[j], e[j].x, ox);
      oy = fmaf(beta[j], e[j].y, oy);
    }
    const float2 r = e[2];
    const int p = map[v];
    // prolongation: into xout, or (no output, no target) into xc.next()
    float2* dst = xout ? xout : (target ? nullptr : xc.next());
    if (dst) {
      const float2 xp = xc.cur()[p];
      dst[v] = make_float2(xp.x + r.x + ox, xp.y + r.y + oy);
    }
    if (target) {
      const float2 xp = xc.cur()[p];
      const float2 t = target[v];
      const float tx = t.x - xp.x - r.x, ty = t.y - xp.y - r.y;
      const float dx = ox - tx, dy = oy - ty;
      const float cp = cc[p];
      l = (dx * dx + dy * dy) / cp;
      const float g = 2.f / ((float)n * cp);
#pragma unroll
      for (int j = 0; j < kO; ++j) dbeta[kO * (size_t)v + j] = g * (dx * e[j].x + dy * e[j].y);
    }
  }
  if (loss_part) {
    // block sum of the loss terms (FP32 per thread, FP64 per block)
    __shared__ float red[32];
    float s = l;
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
      loss_part[blockIdx.x] = t / n;
    }
  }
}

// dH3 = dbeta Wo^T (FP32 [n x 64]).
__global__ void net_head_back(int n, const float* __restrict__ dbeta, const float* __restrict__ Wo,
                              float* __restrict__ dH) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * kH) return;
  const int v = i / kH, d = i % kH;
  const float* g = dbeta + kO * (size_t)v;
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kO; ++j) s = fmaf(g[j], Wo[d * kO + j], s);
  dH[i] = s;
}

// dZ = dH * (H > 0) in BF16 (the backward GEMM's A operand) and FP32 (the
// weight-gradient reduction).
__global__ void net_relu_back(int m, const float* __restrict__ dH,
                              const __nv_bfloat16* __restrict__ H, __nv_bfloat16* __restrict__ dZb,
                              float* __restrict__ dZ) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const float g = __bfloat162float(H[i]) > 0.f ? dH[i] : 0.f;
  dZ[i] = g;
  dZb[i] = __float2bfloat16_rn(g);
}

// Weight-gradient partials: part[b][r][c] = sum over block b's vertices of
// X[v][r] * G[v][c] (X BF16 [n x R], G FP32 [n x C]); one thread per (r, c).
__global__ void net_outer_part(int n, int R, int C, const __nv_bfloat16* __restrict__ X,
                               const float* __restrict__ G, int chunk, float* __restrict__ part) {
  const int rc = threadIdx.x + blockIdx.y * blockDim.x;
  if (rc >= R * C) return;
  const int r = rc / C, c = rc % C;
  const int v0 = blockIdx.x * chunk, v1 = min(n, v0 + chunk);
  float s = 0.f;
  for (int v = v0; v < v1; ++v) s = fmaf(__bfloat162float(X[(size_t)v * R + r]), G[(size_t)v * C + c], s);
  part[(size_t)blockIdx.x * R * C + rc] = s;
}

// Column sums partials (bias gradients): part[b][c] = sum of G[v][c].
__global__ void net_colsum_part(int n, int C, const float* __restrict__ G, int chunk,
                                float* __restrict__ part) {
  const int c = threadIdx.x;
  if (c >= C) return;
  const int v0 = blockIdx.x * chunk, v1 = min(n, v0 + chunk);
  float s = 0.f;
  for (int v = v0; v < v1; ++v) s += G[(size_t)v * C + c];
  part[(size_t)blockIdx.x * C + c] = s;
}

// Fixed-order sum of `parts` partial arrays of length m into out (FP32).
__global__ void net_reduce_parts(int parts, int m, const float* __restrict__ part, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double s = 0.0;
  for (int b = 0; b < parts; ++b) s += part[(size_t)b * m + i];
  out[i] = (float)s;
}

// dH_prev[w] = dHc[w][0:64] + sum over neighbours v of dHc[v][64:128] / deg(v)
// (the transpose of the mean aggregation; the graph is symmetric).
__global__ void net_agg_back(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const float* __restrict__ dHc, float* __restrict__ dH) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= n) return;
  float a0 = dHc[(size_t)w * 2 * kH + lane], a1 = dHc[(size_t)w * 2 * kH + 32 + lane];
  for (int k = rp[w]; k < rp[w + 1]; ++k) {
    const int v = col[k];
    const float inv = 1.f / (float)(rp[v + 1] - rp[v]);
    a0 = fmaf(dHc[(size_t)v * 2 * kH + kH + lane], inv, a0);
    a1 = fmaf(dHc[(size_t)v * 2 * kH + kH + 32 + lane], inv, a1);
  }
  dH[(size_t)w * kH + lane] = a0;
  dH[(size_t)w * kH + 32 + lane] = a1;
}

// Adam (Kingma and Ba 2015) on the FP32 masters.
__global__ void net_adam(int m, float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M1,
                         float* __restrict__ M2, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const float g = G[i];
  const float a = 0.9f * M1[i] + 0.1f * g;
  const float b = 0.999f * M2[i] + 0.001f * g * g;
  M1[i] = a;
  M2[i] = b;
  P[i] -= lr * (a / c1) / (sqrtf(b / c2) + 1e-8f);
}

// BF16 copies of W_l [rows x 64]: Wt = W^T [64 x rows] (forward B operand)
// and Wb = W [rows x 64] (backward B operand).
__global__ void net_cast_w(int rows, const float* __restrict__ W, __nv_bfloat16* __restrict__ Wt,
                           __nv_bfloat16* __restrict__ Wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * kH) return;
  const int r = i / kH, c = i % kH;
  const __nv_bfloat16 v = __float2bfloat16_rn(W[i]);
  Wt[(size_t)c * rows + r] = v;
  if (Wb) Wb[i] = v;
}

}  // namespace

// ----------------------------------------------------------------- host side
// Parameter offsets in the flat FP32 array: W0 [16x64], b0, W1 [128x64], b1,
// W2 [128x64], b2, Wo [64x4], bo.
void net_offsets(int off[9]) {
  int o = 0;
  const int rows[3] = {2 * kF, 2 * kH, 2 * kH};
  for (int l = 0; l < 3; ++l) {
    off[2 * l] = o;
    o += rows[l] * kH;
    off[2 * l + 1] = o;
    o += kH;
  }
  off[6] = o;
  o += kH * kO;
  off[7] = o;
  o += kO;
  off[8] = o;
}

mm_status net_alloc(Net& net, int max_n) {
  int off[9];
  net_offsets(off);
  const int P = off[8];
  if (!net.P) {
    MM_CK(cudaMalloc(&net.P, sizeof(float) * P));
    MM_CK(cudaMalloc(&net.G, sizeof(float) * P));
    MM_CK(cudaMalloc(&net.M1, sizeof(float) * P));
    MM_CK(cudaMalloc(&net.M2, sizeof(float) * P));
    MM_CK(cudaMemset(net.M1, 0, sizeof(float) * P));
    MM_CK(cudaMemset(net.M2, 0, sizeof(float) * P));
    const int rows[3] = {2 * kF, 2 * kH, 2 * kH};
    for (int l = 0; l < 3; ++l) {
      MM_CK(cudaMalloc(&net.Wt[l], sizeof(__nv_bfloat16) * rows[l] * kH));
      MM_CK(cudaMalloc(&net.Wb[l], sizeof(__nv_bfloat16) * rows[l] * kH));
    }
    MM_CK(cudaMalloc(&net.err, sizeof(int)));
    MM_CK(cudaMemset(net.err, 0, sizeof(int)));
    MM_CK(cudaMalloc(&net.stat, sizeof(float) * 4));
  }
  if (max_n > net.cap) {
    void* bufs[] = {net.f, net.basis, net.Hc, net.H[0], net.H[1], net.H[2], net.dbeta, net.dH,
                    net.dZ, net.dZb, net.dHc, net.part, net.loss_part};
    for (void* b : bufs)
      if (b) cudaFree(b);
    const size_t N = (size_t)max_n;
    MM_CK(cudaMalloc(&net.f, sizeof(__nv_bfloat16) * N * kF));
    MM_CK(cudaMalloc(&net.basis, sizeof(float2) * N * kO));
    MM_CK(cudaMalloc(&net.Hc, sizeof(__nv_bfloat16) * N * 2 * kH));
    for (int l = 0; l < 3; ++l) MM_CK(cudaMalloc(&net.H[l], sizeof(__nv_bfloat16) * N * kH));
    MM_CK(cudaMalloc(&net.dbeta, sizeof(float) * N * kO));
    MM_CK(cudaMalloc(&net.dH, sizeof(float) * N * kH));
    MM_CK(cudaMalloc(&net.dZ, sizeof(float) * N * kH));
    MM_CK(cudaMalloc(&net.dZb, sizeof(__nv_bfloat16) * N * kH));
    MM_CK(cudaMalloc(&net.dHc, sizeof(float) * N * 2 * kH));
    MM_CK(cudaMalloc(&net.part, sizeof(float) * (size_t)kNetParts * 2 * kH * kH));
    MM_CK(cudaMalloc(&net.loss_part, sizeof(double) * (size_t)ceil_div(N, 256)));
    net.cap = max_n;
  }
  return MM_OK;
}

void net_free(Net& net) {
  void* bufs[] = {net.P, net.G, net.M1, net.M2, net.Wt[0], net.Wt[1], net.Wt[2], net.Wb[0],
                  net.Wb[1], net.Wb[2], net.err, net.stat, net.f, net.basis, net.Hc, net.H[0], net.H[1],
                  net.H[2], net.dbeta, net.dH, net.dZ, net.dZb, net.dHc, net.part,
                  net.loss_part};
  for (void* b : bufs)
    if (b) cudaFree(b);
  net = Net();
}

mm_status net_sync_weights(Net& net, cudaStream_t s) {
  int off[9];
  net_offsets(off);
  const int rows[3] = {2 * kF, 2 * kH, 2 * kH};
  for (int l = 0; l < 3; ++l)
    net_cast_w<<<ceil_div(rows[l] * kH, 256), 256, 0, s>>>(rows[l], net.P + off[2 * l],
                                                           (__nv_bfloat16*)net.Wt[l],
                                                           (__nv_bfloat16*)net.Wb[l]);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

// Forward pass.  With `target`: the loss (per-block partials in
// net.loss_part) and dbeta.  Positions go to xout, or -- no xout and no
// target -- to smp.xc.next() (the prolongation step of a layout).
mm_status net_forward(Net& net, const NetSample& smp, float2* xout, const float2* target,
                      cudaStream_t s) {
  const int n = smp.n;
  if (n < 1) return MM_OK;
  if (n > net.cap) {
    set_error("network workspace holds %d vertices, sample has %d", net.cap, n);
    return MM_ERR_INVALID_ARG;
  }
  if (smp.nc < 1) {
    set_error("prolongation sample without coarse vertices");
    return MM_ERR_INVALID_ARG;
  }
  int off[9];
  net_offsets(off);
  net_stat<<<1, kStatThreads, 0, s>>>(smp.nc, smp.xc, net.stat);
  net_features<<<ceil_div(n, 256), 256, 0, s>>>(
      n, smp.rp, smp.col, smp.map, smp.xc, smp.crp, smp.ccol, smp.cc, net.stat,
      (uint32_t)(smp.seed & 0xffffffffu), (uint32_t)(smp.seed >> 32), (uint32_t)smp.level,
      (__nv_bfloat16*)net.f, net.basis);
  const __nv_bfloat16* Hin = (const __nv_bfloat16*)net.f;
  for (int l = 0; l < 3; ++l) {
    if (l == 0)
      net_aggregate<kF><<<ceil_div((int64_t)n * 32, 256), 256, 0, s>>>(
          n, smp.rp, smp.col, Hin, (__nv_bfloat16*)net.Hc);
    else
      net_aggregate<kH><<<ceil_div((int64_t)n * 32, 256), 256, 0, s>>>(
          n, smp.rp, smp.col, Hin, (__nv_bfloat16*)net.Hc);
    const int K = l == 0 ? 2 * kF : 2 * kH;
    MM_TRY(gemm_bf16(net.Hc, n, K, net.Wt[l], kH, net.P + off[2 * l + 1], 1, net.H[l], nullptr,
                     net.err, s));
    Hin = (const __nv_bfloat16*)net.H[l];
    // the backward pass needs every layer's Hcat: recompute it there
  }
  net_head<<<ceil_div(n, 256), 256, 0, s>>>(n, (const __nv_bfloat16*)net.H[2], net.P + off[6],
                                            net.P + off[7], net.basis, smp.map, smp.xc, smp.cc,
                                            xout, target, net.dbeta,
                                            target ? net.loss_part : nullptr);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

// Gradients of the loss into net.G (after net_forward with a target).
mm_status net_backward(Net& net, const NetSample& smp, cudaStream_t s) {
  const int n = smp.n;
  int off[9];
  net_offsets(off);
  const int parts = std::min(kNetParts, ceil_div(n, 64));
  const int chunk = ceil_div(n, parts);
  // head: dWo = H3^T dbeta, dbo = sum dbeta, dH3 = dbeta Wo^T
  net_outer_part<<<dim3(parts, 1), 256, 0, s>>>(n, kH, kO, (const __nv_bfloat16*)net.H[2],
                                                net.dbeta, chunk, net.part);
  net_reduce_parts<<<1, 256, 0, s>>>(parts, kH * kO, net.part, net.G + off[6]);
  net_colsum_part<<<parts, 32, 0, s>>>(n, kO, net.dbeta, chunk, net.part);
  net_reduce_parts<<<1, 32, 0, s>>>(parts, kO, net.part, net.G + off[7]);
  net_head_back<<<ceil_div((int64_t)n * kH, 256), 256, 0, s>>>(n, net.dbeta, net.P + off[6],
                                                               net.dH);
  for (int l = 2; l >= 0; --l) {
    const int D = l == 0 ? kF : kH;
    const int R = 2 * D;
    // rebuild Hcat of layer l from H_{l-1} (or the features)
    const __nv_bfloat16* Hin = l == 0 ? (const __nv_bfloat16*)net.f
                                      : (const __nv_bfloat16*)net.H[l - 1];
    if (l == 0)
      net_aggregate<kF><<<ceil_div((int64_t)n * 32, 256), 256, 0, s>>>(
          n, smp.rp, smp.col, Hin, (__nv_bfloat16*)net.Hc);
    else
      net_aggregate<kH><<<ceil_div((int64_t)n * 32, 256), 256, 0, s>>>(
          n, smp.rp, smp.col, Hin, (__nv_bfloat16*)net.Hc);
    net_relu_back<<<ceil_div((int64_t)n * kH, 256), 256, 0, s>>>(
        n * kH, net.dH, (const __nv_bfloat16*)net.H[l], (__nv_bfloat16*)net.dZb, net.dZ);
    // dW_l = Hcat^T dZ on the tensor cores (BF16 operands, FP32 accumulation
    // per vertex range, partials added in a fixed order); db_l = sum dZ
    const int tparts = gemm_tn_parts(n);
    MM_TRY(gemm_tn_partials(net.Hc, n, R, net.dZb, net.part, tparts, net.err, s));
    net_reduce_parts<<<ceil_div(R * kH, 256), 256, 0, s>>>(tparts, R * kH, net.part,
                                                           net.G + off[2 * l]);
    net_colsum_part<<<parts, kH, 0, s>>>(n, kH, net.dZ, chunk, net.part);
    net_reduce_parts<<<1, kH, 0, s>>>(parts, kH, net.part, net.G + off[2 * l + 1]);
    if (l == 0) break;
    // dHcat = dZ W_l^T on the tensor cores: A = dZ [n x 64], B = W_l [128 x 64]
    MM_TRY(gemm_bf16(net.dZb, n, kH, net.Wb[l], R, nullptr, 0, nullptr, net.dHc, net.err, s));
    net_agg_back<<<ceil_div((int64_t)n * 32, 256), 256, 0, s>>>(n, smp.rp, smp.col, net.dHc,
                                                               net.dH);
  }
  MM_CK(cudaGetLastError());
  return MM_OK;
}

mm_status net_adam_step(Net& net, float lr, cudaStream_t s) {
  int off[9];
  net_offsets(off);
  net.step += 1;
  const double c1 = 1.0 - std::pow(0.9, net.step), c2 = 1.0 - std::pow(0.999, net.step);
  net_adam<<<ceil_div(off[8], 256), 256, 0, s>>>(off[8], net.P, net.G, net.M1, net.M2, lr,
                                                 (float)c1, (float)c2);
  MM_TRY(net_sync_weights(net, s));
  return MM_OK;
}

}  // namespace mm
