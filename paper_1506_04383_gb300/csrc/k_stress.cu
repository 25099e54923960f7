// Full stress and its optimal scale (Sec. 4, methodology):
//
//   F(x) = sum over unordered pairs {u,v} of w_uv (|x_u - x_v| - d_uv)^2,
//   d_uv the hop distance, w_uv = d_uv^-2, and the scalar s minimising
//   sum w (s |x_u - x_v| - d)^2:  s = sum w d |dx| / sum w |dx|^2,
//   F(s x) = sum w d^2 - (sum w d |dx|)^2 / sum w |dx|^2.
//
// All-pairs distances come from breadth-first searches run 64 sources at a
// time: every vertex keeps one 64-bit word per role (reached, frontier, next
// frontier), bit j standing for source 64b + j.  One level of all 64
// searches is one pass over the CSR: next[v] = OR of frontier[u] over the
// neighbours u, minus what v has already seen; each newly set bit is a pair
// (source, v) at distance = level, whose terms are added right there (no
// distance matrix is stored).  A block runs whole batches (persistent over
// batches); its three word arrays live in global scratch.  Each unordered
// pair is counted once, from its smaller endpoint.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "mm_internal.cuh"

namespace mm {

namespace {

constexpr int kStressThreads = 1024;
constexpr int kStressSums = 5;  // F, A = sum w d L, B = sum w L^2, C = sum w d^2, pairs

__global__ void __launch_bounds__(kStressThreads) stress_bfs_kernel(
    int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
    const float2* __restrict__ x, int batches, unsigned long long* scratch, double* part) {
  __shared__ float2 src[64];
  __shared__ double red[kStressSums][kStressThreads / 32];
  unsigned long long* vis = scratch + (size_t)blockIdx.x * 3 * (size_t)n;
  unsigned long long* cur = vis + n;
  unsigned long long* nxt = cur + n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int b = blockIdx.x; b < batches; b += gridDim.x) {
    const int s0 = b * 64;
    const int ns = min(64, n - s0);
    if (tid < ns) src[tid] = x[s0 + tid];
    for (int v = tid; v < n; v += kStressThreads) {
      const unsigned long long m = (v >= s0 && v < s0 + ns) ? (1ull << (v - s0)) : 0ull;
      vis[v] = m;
      cur[v] = m;
    }
    __syncthreads();
    double acc[kStressSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int level = 1; level < n; ++level) {
      float f = 0.f, a = 0.f, bb = 0.f, c = 0.f;
      int cnt = 0;
      bool any = false;
      const float d = (float)level, w = 1.f / (d * d);
      for (int v = tid; v < n; v += kStressThreads) {
        unsigned long long nb = 0ull;
        for (int e = rp[v]; e < rp[v + 1]; ++e) nb |= cur[col[e]];
        unsigned long long fresh = nb & ~vis[v];
        nxt[v] = fresh;
        if (!fresh) continue;
        any = true;
        vis[v] |= fresh;
        const float2 xv = x[v];
        while (fresh) {
          const int j = __ffsll((long long)fresh) - 1;
          fresh &= fresh - 1;
          if (s0 + j >= v) continue;  // the pair is counted from its smaller end
          const float dx = src[j].x - xv.x, dy = src[j].y - xv.y;
          const float L = sqrtf(fmaf(dx, dx, dy * dy));
          const float r = L - d;
          f = fmaf(w * r, r, f);
          a = fmaf(w * d, L, a);
          bb = fmaf(w * L, L, bb);
          c += w * d * d;
          ++cnt;
        }
      }
      if (cnt) {
        acc[0] += f;
        acc[1] += a;
        acc[2] += bb;
        acc[3] += c;
        acc[4] += cnt;
      }
      // every next word is written and no thread reads this frontier again
      const bool more = __syncthreads_or(any) != 0;
      unsigned long long* t = cur;
      cur = nxt;
      nxt = t;
      if (!more) break;
    }
    // fixed-order block sums of the batch (FP64), one record per batch
#pragma unroll
    for (int k = 0; k < kStressSums; ++k) {
      double v = acc[k];
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (tid < kStressSums) {
      double t = 0.0;
      for (int w2 = 0; w2 < kStressThreads / 32; ++w2) t += red[tid][w2];
      part[(size_t)b * kStressSums + tid] = t;
    }
    __syncthreads();
  }
}

}  // namespace

mm_status full_stress(int n, const int32_t* rp, const int32_t* col, const float2* x,
                      double out[4], cudaStream_t s) {
  if (n < 1) {
    out[0] = out[1] = out[2] = out[3] = 0.0;
    return MM_OK;
  }
  const int batches = ceil_div(n, 64);
  const int grid = std::min(batches, 2 * num_sms());
  unsigned long long* scratch = nullptr;
  double* part = nullptr;
  MM_CK(cudaMallocAsync(&scratch, sizeof(unsigned long long) * 3 * (size_t)n * grid, s));
  MM_CK(cudaMallocAsync(&part, sizeof(double) * kStressSums * (size_t)batches, s));
  stress_bfs_kernel<<<grid, kStressThreads, 0, s>>>(n, rp, col, x, batches, scratch, part);
  cudaError_t e = cudaGetLastError();
  std::vector<double> h((size_t)kStressSums * batches);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(scratch, s);
  cudaFreeAsync(part, s);
  MM_CK(e);
  double F = 0, A = 0, B = 0, C = 0, P = 0;
  for (int b = 0; b < batches; ++b) {
    F += h[(size_t)b * kStressSums];
    A += h[(size_t)b * kStressSums + 1];
    B += h[(size_t)b * kStressSums + 2];
    C += h[(size_t)b * kStressSums + 3];
    P += h[(size_t)b * kStressSums + 4];
  }
  out[0] = F;
  out[1] = B > 0 ? A / B : 0.0;
  out[2] = B > 0 ? C - A * A / B : C;
  out[3] = P;
  return MM_OK;
}

}  // namespace mm
