// FP32 FMA throughput of the device, measured (the denominator of the
// ALU-bound rooflines: the Barnes-Hut walk, the exact pair sums and the
// Eq. 3 sums).  No paper counterpart; a measurement aid.
//
// Every thread runs kChains independent FMA chains (enough independent work
// to cover the FMA latency), unrolled so that the loop overhead is a few
// percent; the grid holds 4 blocks of 512 threads per SM.  Flops counted:
// 2 per FMA.
#include <cuda_runtime.h>

#include "mm_internal.cuh"

namespace mm {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 32;
constexpr int kPeakThreads = 512;

__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(float* out, int iters, float a,
                                                               float b) {
  float v[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) v[j] = (float)(threadIdx.x + j) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) v[j] = fmaf(v[j], a, b);
    }
  }
  float sum = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) sum += v[j];
  // a store the compiler cannot prove dead (a = 1, b = 0 keeps v finite)
  if (sum == -1.2345f) out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

}  // namespace
}  // namespace mm

using namespace mm;

extern "C" mm_status mm_measure_fp32_peak(int32_t reps, double* tflops, double* ms_per_launch,
                                          void* stream) {
  if (reps < 1 || !tflops) {
    set_error("mm_measure_fp32_peak: need reps >= 1 and tflops");
    return MM_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = 4 * num_sms();
  const int iters = 2048;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  MM_CK(cudaMallocAsync(&out, sizeof(float) * (size_t)blocks * kPeakThreads, s));
  mm_status st = MM_OK;
  float ms = 0.f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = cuda_status(cudaGetLastError(), "cudaEventCreate", __FILE__, __LINE__);
  } else {
    fma_peak_kernel<<<blocks, kPeakThreads, 0, s>>>(out, iters, 1.0f, 0.0f);  // warm-up
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r)
      fma_peak_kernel<<<blocks, kPeakThreads, 0, s>>>(out, iters, 1.0f, 0.0f);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) st = cuda_status(e, "fma_peak_kernel", __FILE__, __LINE__);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  if (st != MM_OK) return st;
  const double per = (double)ms / reps;
  const double flops = 2.0 * kChains * kUnroll * (double)iters * blocks * kPeakThreads;
  *tflops = flops / (per * 1e-3) / 1e12;
  if (ms_per_launch) *ms_per_launch = per;
  return MM_OK;
}
