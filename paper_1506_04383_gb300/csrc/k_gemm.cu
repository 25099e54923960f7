// BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05) with an
// FP32 accumulator in tensor memory, for the dense layers of the learned
// prolongation:   C[M x N] = A[M x K] * B[N x K]^T  (+ bias, ReLU)
// A and B are row-major with K contiguous (both "K-major").  One CTA of 128
// threads computes a 128-row tile:
//   * warp 0 allocates N tensor-memory columns (128 lanes x N FP32);
//   * all threads stage A (128 x K) and B (N x K) in shared memory in the
//     canonical no-swizzle K-major layout of 8 x 16-byte core matrices
//     (K-adjacent core matrices 128 B apart, M/N-adjacent ones 256 B apart,
//     one 16-wide K slice after another);
//   * one thread issues K/16 tcgen05.mma (kind::f16, BF16 x BF16 -> FP32,
//     M = 128) and commits them to an mbarrier;
//   * after the (bounded) wait every warp reads its 32 accumulator rows with
//     tcgen05.ld 32x32b and runs the epilogue (bias, ReLU, BF16 or FP32
//     store); warp 0 frees the tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "mm_internal.cuh"

namespace mm {

namespace {

constexpr int kGemmThreads = 128;
constexpr int kTileM = 128;
constexpr int kSpin = 1 << 26;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (K direction), stride-dimension byte offset (M/N direction), the
// descriptor version bit (46), no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3ffffu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t make_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// Bytes of the staged tiles: A = (K/16) slices x 4096 B, B = (K/16) x N x 32 B.
__host__ __device__ constexpr int gemm_smem_bytes(int n, int k) {
  return (k / 16) * 4096 + (k / 16) * n * 32;
}

template <int N>
__global__ void __launch_bounds__(kGemmThreads) gemm_tc_kernel(
    const __nv_bfloat16* __restrict__ A, int M, int K, const __nv_bfloat16* __restrict__ B,
    const float* __restrict__ bias, int relu, __nv_bfloat16* __restrict__ outb,
    float* __restrict__ outf, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTileM;
  const int ks = K / 16;
  unsigned char* sA = smem;
  unsigned char* sB = smem + ks * 4096;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // stage A: 128 rows x K/8 chunks of 16 bytes (rows beyond M are zero)
  const int kc = K / 8;
  for (int c = tid; c < kTileM * kc; c += kGemmThreads) {
    const int m = c / kc, k8 = c % kc;
    const int row = m0 + m;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (row < M) v = *reinterpret_cast<const uint4*>(A + (size_t)row * K + k8 * 8);
    const int off = (k8 >> 1) * 4096 + (m >> 3) * 256 + (k8 & 1) * 128 + (m & 7) * 16;
    *reinterpret_cast<uint4*>(sA + off) = v;
  }
  // stage B: N rows x K/8 chunks
  for (int c = tid; c < N * kc; c += kGemmThreads) {
    const int r = c / kc, k8 = c % kc;
    const uint4 v = *reinterpret_cast<const uint4*>(B + (size_t)r * K + k8 * 8);
    const int off = (k8 >> 1) * (N * 32) + (r >> 3) * 256 + (k8 & 1) * 128 + (r & 7) * 16;
    *reinterpret_cast<uint4*>(sB + off) = v;
  }
  // generic-proxy shared stores -> visible to the tensor cores (async proxy)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {
    const uint32_t idesc = make_idesc(kTileM, N);
    const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
    for (int s = 0; s < ks; ++s) {
      const uint64_t ad = make_desc(a0 + s * 4096, 128, 256);
      const uint64_t bd = make_desc(b0 + s * (N * 32), 128, 256);
      const uint32_t acc = s > 0 ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
          "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(&mbar)));
  }
  // wait for the MMAs (phase 0), bounded
  bool ok = false;
  for (int spin = 0; spin < kSpin; ++spin) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
        " selp.b32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(&mbar)));
    if (done) {
      ok = true;
      break;
    }
  }
  // tcgen05.ld is warp-collective: the whole warp reads or none of it
  ok = __all_sync(0xffffffffu, ok);
  if (!ok && lane == 0 && err) atomicOr(err, 4);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t r[16];
      ld16(tbase + (uint32_t)c0, r);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float v = __uint_as_float(r[j]);
          if (bias) v += bias[c0 + j];
          if (relu) v = fmaxf(v, 0.f);
          if (outb) outb[(size_t)row * N + c0 + j] = __float2bfloat16_rn(v);
          if (outf) outf[(size_t)row * N + c0 + j] = v;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(N));
  }
}

template <int N>
mm_status launch_gemm(const __nv_bfloat16* A, int M, int K, const __nv_bfloat16* B,
                      const float* bias, int relu, __nv_bfloat16* outb, float* outf, int* err,
                      cudaStream_t s) {
  const int smem = gemm_smem_bytes(N, K);
  gemm_tc_kernel<N><<<ceil_div(M, kTileM), kGemmThreads, smem, s>>>(A, M, K, B, bias, relu, outb,
                                                                    outf, err);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

}  // namespace

// Opt-in to the shared memory of the largest tiles (K = 128); call once per
// device before the first GEMM (outside stream capture).
mm_status gemm_setup() {
  MM_CK(cudaFuncSetAttribute(gemm_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             gemm_smem_bytes(64, 128)));
  MM_CK(cudaFuncSetAttribute(gemm_tc_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             gemm_smem_bytes(128, 128)));
  return MM_OK;
}

mm_status gemm_bf16(const void* A, int M, int K, const void* B, int N, const float* bias,
                    int relu, void* outb, float* outf, int* err, cudaStream_t s) {
  if (M < 0 || K < 16 || K > 128 || K % 16 || (N != 64 && N != 128) || !A || !B ||
      (!outb && !outf)) {
    set_error("gemm: need 16 <= K <= 128 (multiple of 16), N in {64, 128}");
    return MM_ERR_INVALID_ARG;
  }
  if (((uintptr_t)A & 15) || ((uintptr_t)B & 15)) {
    set_error("gemm: A and B must be 16-byte aligned");
    return MM_ERR_INVALID_ARG;
  }
  if (M == 0) return MM_OK;
  if (N == 64)
    return launch_gemm<64>((const __nv_bfloat16*)A, M, K, (const __nv_bfloat16*)B, bias, relu,
                           (__nv_bfloat16*)outb, outf, err, s);
  return launch_gemm<128>((const __nv_bfloat16*)A, M, K, (const __nv_bfloat16*)B, bias, relu,
                          (__nv_bfloat16*)outb, outf, err, s);
}

}  // namespace mm
