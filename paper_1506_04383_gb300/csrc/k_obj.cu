// Maxent-stress objective, Eq. 1, over the pair set S of a level:
//   M(x) = sum_{{u,v} in S} w_uv (|x_u - x_v| - d_uv)^2
//        - alpha sum_{{u,v} not in S} ln |x_u - x_v|.
// The ln-sum over pairs outside S is the all-pairs ln-sum (tiles of 256 x 256
// positions in shared memory, upper triangle only, FP32 terms summed per
// tile and accumulated in FP64) minus the ln-sum over S.  Coincident pairs
// contribute 0.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mm_internal.cuh"

namespace mm {

namespace {

constexpr int kT = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kT / 32; ++w) t += sh[w];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(kT) pairs_ln_kernel(const float2* __restrict__ x, int n,
                                                      int nt, int64_t npairs, double* partials) {
  __shared__ float2 tile[kT];
  double acc = 0.0;
  for (int64_t t = blockIdx.x; t < npairs; t += gridDim.x) {
    // tile pair (I, J), I <= J, from the row-major upper-triangle index t
    int I = (int)floor(((2.0 * nt + 1.0) - sqrt((2.0 * nt + 1.0) * (2.0 * nt + 1.0) - 8.0 * t)) / 2.0);
    I = max(0, min(I, nt - 1));
    auto first = [&](int r) { return (int64_t)r * nt - (int64_t)r * (r - 1) / 2; };
    while (I > 0 && first(I) > t) --I;
    while (I + 1 < nt && first(I + 1) <= t) ++I;
    const int J = I + (int)(t - first(I));
    const int v0 = J * kT;
    const int cnt = min(kT, n - v0);
    __syncthreads();
    if ((int)threadIdx.x < cnt) tile[threadIdx.x] = x[v0 + threadIdx.x];
    __syncthreads();
    const int u = I * kT + threadIdx.x;
    if (u < n) {
      const float2 xu = x[u];
      float s = 0.f;
      for (int k = 0; k < cnt; ++k) {
        if (I == J && v0 + k <= u) continue;
        const float dx = xu.x - tile[k].x, dy = xu.y - tile[k].y;
        const float q = fmaf(dx, dx, dy * dy);
        if (q > 0.f) s += logf(q);
      }
      acc += 0.5 * (double)s;
    }
  }
  const double b = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

__global__ void __launch_bounds__(kT) s_pairs_kernel(const float2* __restrict__ x, int n,
                                                     const int32_t* __restrict__ sp,
                                                     const SEnt* __restrict__ S,
                                                     double* partials) {
  double st = 0.0, ln = 0.0;
  for (int u = blockIdx.x * kT + threadIdx.x; u < n; u += gridDim.x * kT) {
    const float2 xu = x[u];
    for (int e = sp[u]; e < sp[u + 1]; ++e) {
      const SEnt en = S[e];
      if (en.col <= u) continue;
      const float2 xv = x[en.col];
      const double dx = (double)xu.x - xv.x, dy = (double)xu.y - xv.y;
      const double q = dx * dx + dy * dy;
      const double dist = sqrt(q);
      const double d = en.d;
      st += (dist - d) * (dist - d) / (d * d);
      if (q > 0) ln += 0.5 * log(q);
    }
  }
  const double a = block_sum(st);
  const double b = block_sum(ln);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

__global__ void __launch_bounds__(kT) sum_phi_kernel(const float* __restrict__ phi, int n,
                                                     double* partials) {
  double acc = 0.0;
  for (int u = blockIdx.x * kT + threadIdx.x; u < n; u += gridDim.x * kT) acc += phi[u];
  const double b = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

}  // namespace

// Eq. 1 with the ln-sum over all pairs from per-vertex log potentials
// Phi[u] = sum_{v != u} ln|x_u - x_v| (a Barnes-Hut estimate): all-pairs
// ln-sum = (1/2) sum_u Phi[u]; stress and the ln-sum over S exact.
mm_status objective_from_phi(const Level& L, const float2* x, const float* phi, double alpha,
                             double out[3], cudaStream_t s) {
  const int n = L.n;
  const int pb = std::max(1, std::min(ceil_div(n, kT), num_sms() * 4));
  const int sb = std::max(1, std::min(ceil_div(n, kT), num_sms() * 4));
  double* parts = nullptr;
  MM_CK(cudaMalloc(&parts, sizeof(double) * (size_t)(pb + 2 * sb)));
  sum_phi_kernel<<<pb, kT, 0, s>>>(phi, n, parts);
  s_pairs_kernel<<<sb, kT, 0, s>>>(x, n, L.sp, L.s, parts + pb);
  cudaError_t e = cudaGetLastError();
  std::vector<double> h((size_t)(pb + 2 * sb));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), parts, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(parts);
  MM_CK(e);
  double all = 0, stress = 0, lnS = 0;
  for (int i = 0; i < pb; ++i) all += h[i];
  all *= 0.5;
  for (int i = 0; i < sb; ++i) {
    stress += h[pb + 2 * i];
    lnS += h[pb + 2 * i + 1];
  }
  out[0] = stress;
  out[1] = all - lnS;
  out[2] = stress - alpha * (all - lnS);
  return MM_OK;
}

mm_status objective_exact(const Level& L, const float2* x, double alpha, double out[3],
                          cudaStream_t s) {
  const int n = L.n;
  const int nt = ceil_div(std::max(n, 1), kT);
  const int64_t npairs = (int64_t)nt * (nt + 1) / 2;
  const int pb = (int)std::min<int64_t>(npairs, num_sms() * 8);
  const int sb = std::max(1, std::min(ceil_div(n, kT), num_sms() * 4));
  double* parts = nullptr;
  MM_CK(cudaMalloc(&parts, sizeof(double) * (size_t)(pb + 2 * sb)));
  pairs_ln_kernel<<<pb, kT, 0, s>>>(x, n, nt, npairs, parts);
  s_pairs_kernel<<<sb, kT, 0, s>>>(x, n, L.sp, L.s, parts + pb);
  cudaError_t e = cudaGetLastError();
  std::vector<double> h((size_t)(pb + 2 * sb));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), parts, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(parts);
  MM_CK(e);
  double all = 0, stress = 0, lnS = 0;
  for (int i = 0; i < pb; ++i) all += h[i];
  for (int i = 0; i < sb; ++i) {
    stress += h[pb + 2 * i];
    lnS += h[pb + 2 * i + 1];
  }
  out[0] = stress;
  out[1] = all - lnS;
  out[2] = stress - alpha * (all - lnS);
  return MM_OK;
}

}  // namespace mm
