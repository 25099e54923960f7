// BF16 tensor-core GEMMs on the 5th-generation tensor cores (tcgen05) with an
// FP32 accumulator in tensor memory, for the dense layers of the learned
// prolongation: the layer products (gemm_tc_kernel, below) and the weight
// gradients (gemm_tn_partial_kernel, further down).
//   C[M x N] = A[M x K] * B[N x K]^T  (+ bias, ReLU)
// A and B are row-major with K contiguous (both "K-major").  The layer
// product is persistent, one CTA of 256 threads per SM over 128-row tiles:
//   * warp 0 allocates 2 N tensor-memory columns (two 128 x N FP32
//     accumulators);
//   * B (N x K) is staged once and the A tiles (128 x K) stream through a
//     ring of shared-memory stages by cp.async, all in the canonical
//     no-swizzle K-major layout of 8 x 16-byte core matrices (K-adjacent
//     core matrices 128 B apart, M/N-adjacent ones 256 B apart, one 16-wide
//     K slice after another);
//   * per tile one thread issues K/16 tcgen05.mma (kind::f16, BF16 x BF16 ->
//     FP32, M = 128) into the tile's accumulator and commits them to that
//     accumulator's mbarrier;
//   * while they run, every warp drains the previous tile's accumulator
//     (bounded mbarrier wait, tcgen05.ld 32x32b, bias, ReLU, BF16 or FP32
//     store); warp 0 frees the tensor memory at the end.
#include <cuda_bf16.h>

#include <algorithm>
#include <cuda_runtime.h>

#include "mm_internal.cuh"

namespace mm {

namespace {

constexpr int kGemmThreads = 128;  // weight-gradient CTAs
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

// Shared memory: B = (K/16) x N x 32 B once, then kPipeStages A stages of
// (K/16) x 4096 B (128 rows).
constexpr int kPipeStages = 5;  // A tiles in shared memory: 3 in flight, 1 in the MMA, 1 spare
__host__ __device__ constexpr int gemm_smem_bytes(int n, int k) {
  return (k / 16) * n * 32 + kPipeStages * (k / 16) * 4096;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes)
               : "memory");
}

constexpr int kPipeThreads = 256;

// The copies of A tile t (rows 128 t ...) into a stage, in the K-major core-
// matrix layout; rows beyond M are zero-filled (no bytes read).  K / 8 is a
// power of two (K in {16, 32, 64, 128}): lg_kc = log2(K / 8).
__device__ __forceinline__ void load_a_tile(const __nv_bfloat16* __restrict__ A, int M, int K,
                                            int lg_kc, int t, uint32_t sA, int tid) {
  const int kc = K / 8;
  const int m0 = t * kTileM;
  for (int c = tid; c < kTileM * kc; c += kPipeThreads) {
    const int m = c >> lg_kc, k8 = c & (kc - 1);
    const int row = m0 + m;
    const bool in = row < M;
    const __nv_bfloat16* src = A + (size_t)(in ? row : 0) * K + k8 * 8;
    const uint32_t off = (k8 >> 1) * 4096 + (m >> 3) * 256 + (k8 & 1) * 128 + (m & 7) * 16;
    cp_async16(sA + off, src, in ? 16u : 0u);
  }
}

// Persistent: CTA b takes the 128-row tiles b, b + grid, ... .  The A tiles
// stream through a ring of kPipeStages shared-memory stages by cp.async
// (three tiles ahead of the one in the MMA), B is staged once, and the
// accumulator alternates between two TMEM buffers, so the MMAs of tile j run
// while the epilogue of tile j - 1 drains the other buffer and later tiles
// are in flight.  A stage is refilled only after the MMA that read it has
// completed (its mbarrier was waited on one iteration earlier).  Eight warps:
// warps w and w + 4 share TMEM lane quarter w (rows 32 w ..) and take one
// half of the columns each.
template <int N>
__global__ void __launch_bounds__(kPipeThreads, 1) gemm_tc_kernel(
    const __nv_bfloat16* __restrict__ A, int M, int K, const __nv_bfloat16* __restrict__ B,
    const float* __restrict__ bias, int relu, __nv_bfloat16* __restrict__ outb,
    float* __restrict__ outf, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ float sbias[N];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, half = warp >> 2;
  const int ks = K / 16;
  const int lg_kc = __ffs(K / 8) - 1;
  const int tiles = (M + kTileM - 1) / kTileM;
  const int my = (tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int stage_bytes = ks * 4096;
  unsigned char* sB = smem;
  const uint32_t sA0 = smem_addr(smem + ks * N * 32);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(2 * N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  for (int c = tid; c < N; c += kPipeThreads) sbias[c] = bias ? bias[c] : 0.f;
  // B: N rows x K/8 chunks, once
  const int kc = K / 8;
  for (int c = tid; c < N * kc; c += kPipeThreads) {
    const int r = c / kc, k8 = c % kc;
    const uint4 v = *reinterpret_cast<const uint4*>(B + (size_t)r * K + k8 * 8);
    const int off = (k8 >> 1) * (N * 32) + (r >> 3) * 256 + (k8 & 1) * 128 + (r & 7) * 16;
    *reinterpret_cast<uint4*>(sB + off) = v;
  }
  constexpr int kAhead = kPipeStages - 2;
  for (int j = 0; j < kAhead; ++j) {
    if (j < my)
      load_a_tile(A, M, K, lg_kc, blockIdx.x + j * gridDim.x,
                  sA0 + (j % kPipeStages) * stage_bytes, tid);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = make_idesc(kTileM, N);

  // epilogue of tile jj: wait for its MMAs (bounded), drain its accumulator
  auto epilogue = [&](int jj) {
    const uint32_t bar = smem_addr(&mbar[jj & 1]);
    const uint32_t parity = (uint32_t)((jj >> 1) & 1);
    bool ok = false;
    for (int spin = 0; spin < kSpin; ++spin) {
      uint32_t done;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
          " selp.b32 %0, 1, 0, p;\n}"
          : "=r"(done)
          : "r"(bar), "r"(parity));
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
      const int row = (blockIdx.x + jj * gridDim.x) * kTileM + quarter * 32 + lane;
      const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((jj & 1) * N);
#pragma unroll
      for (int c0 = half * (N / 2); c0 < (half + 1) * (N / 2); c0 += 16) {
        uint32_t r[16];
        ld16(tbase + (uint32_t)c0, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < M) {
          // the lane's 16 consecutive outputs of its row, written as whole
          // 16-byte vectors (every 32-byte sector filled by one thread)
          float v[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            v[q] = __uint_as_float(r[q]) + sbias[c0 + q];
            if (relu) v[q] = fmaxf(v[q], 0.f);
          }
          if (outb) {
            uint32_t pk[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
              pk[q] = *reinterpret_cast<const uint32_t*>(&h2);
            }
            uint4* dst = reinterpret_cast<uint4*>(outb + (size_t)row * N + c0);
            dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
          }
          if (outf) {
            float4* dst = reinterpret_cast<float4*>(outf + (size_t)row * N + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  };

  for (int j = 0; j < my; ++j) {
    // tile j + kAhead into the stage of tile j - 2, whose MMAs were waited
    // for in the previous iteration's epilogue
    const int jn = j + kAhead;
    if (jn < my)
      load_a_tile(A, M, K, lg_kc, blockIdx.x + jn * gridDim.x,
                  sA0 + (jn % kPipeStages) * stage_bytes, tid);
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group %0;" ::"n"(kAhead) : "memory");
    // every thread's copies of tile j (and B) -> visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      const uint32_t a0 = sA0 + (j % kPipeStages) * stage_bytes, b0 = smem_addr(sB);
      const uint32_t d = tmem + (uint32_t)((j & 1) * N);
      for (int s = 0; s < ks; ++s) {
        const uint64_t ad = make_desc(a0 + s * 4096, 128, 256);
        const uint64_t bd = make_desc(b0 + s * (N * 32), 128, 256);
        const uint32_t acc = s > 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_addr(&mbar[j & 1])));
    }
    if (j > 0) epilogue(j - 1);
  }
  if (my > 0) epilogue(my - 1);
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * N));
  }
}

// ------------------------------------------------------------------------
// Weight gradients of the dense layers on the tensor cores:
//   part[b][r][c] = sum over CTA b's vertices v of A[v][r] * B[v][c]
// with A = Hcat (BF16 [n x R], R = 16 or 128) and B = dZ (BF16 [n x 64]);
// the caller adds the per-CTA partials in a fixed order.  In GEMM terms the
// contraction runs over the vertices, so both operands arrive with the
// contracted index slowest (row-major over vertices).  Each CTA (128
// threads, three per SM, a contiguous range of vertices) stages 64 vertices
// at a time: the warps load 8 x 8 BF16 blocks in the matrix-fragment layout
// and store them transposed with stmatrix .trans, so that A^T (R rows,
// padded to 128 with zeros) and B^T (64 rows) land in the same K-major
// no-swizzle layout as gemm_tc_kernel's operands; one thread issues the four
// K = 16 MMAs (M = 128, N = 64) of the chunk into one FP32 accumulator in
// tensor memory and commits them to an mbarrier, which every thread waits
// on (bounded) before the buffers are refilled.  Finally each warp reads its
// 32 accumulator rows with tcgen05.ld and writes the first R rows.
constexpr int kTnChunk = 64;                              // vertices per stage
constexpr int kTnSmem = (kTnChunk / 16) * (4096 + 64 * 32);  // A + B tiles

__global__ void __launch_bounds__(kGemmThreads, 3) gemm_tn_partial_kernel(
    const __nv_bfloat16* __restrict__ A, int n, int R, const __nv_bfloat16* __restrict__ B,
    float* __restrict__ part, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  constexpr int N = 64;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x;
  const int v0 = (int)((int64_t)n * blockIdx.x / G), v1 = (int)((int64_t)n * (blockIdx.x + 1) / G);
  unsigned char* sA = smem;
  unsigned char* sB = smem + (kTnChunk / 16) * 4096;
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
  // rows R..127 of A^T stay zero for the whole run
  for (int i = tid; i < kTnSmem / 16; i += kGemmThreads)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = make_idesc(kTileM, N);
  // The chunk's R + 64 blocks of 8 vertices x 8 columns (of A, then of B),
  // four per warp operation: lane t holds the 32-bit pair (vertex t / 4,
  // columns 2 (t % 4) ..) of each of the operation's blocks -- the fragment
  // layout of an 8 x 8 BF16 matrix -- and stmatrix .trans stores each block
  // transposed, its row j (16 bytes: column j over the 8 vertices) at the
  // address lane 8 i + j gives for block i: row m of the K-major operand,
  // K chunk vg.  The eight rows of a block are 128 contiguous bytes, so the
  // stores do not conflict.  A chunk's fragments are loaded into registers
  // while the previous chunk's MMAs run.
  const int na = (R / 8) * 8;  // A blocks: R/8 column groups x 8 vertex groups
  const int nops = (na + 64) / 4;
  constexpr int kWarpsTn = kGemmThreads / 32;
  constexpr int kOps = (128 + 64) / 4 / kWarpsTn;  // operations per warp, at most
  uint32_t frag[kOps][4];
  auto load_chunk = [&](int base) {
#pragma unroll
    for (int k = 0; k < kOps; ++k) {
      const int op = warp + k * kWarpsTn;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int tb = op * 4 + i;
        const bool isA = tb < na;
        const int t = isA ? tb : tb - na;
        const int cg = t >> 3, vg = t & 7;  // column group, vertex group
        const int v = base + vg * 8 + (lane >> 2);
        // element offset in 32 bits (n x 128 < 2^31 for every level the
        // network sees); one base pointer per operand
        const int off = v * (isA ? R : N) + cg * 8 + 2 * (lane & 3);
        frag[k][i] = op < nops && v < v1
                         ? __ldg(reinterpret_cast<const uint32_t*>((isA ? A : B) + off))
                         : 0u;
      }
    }
  };
  bool ok = true;
  int chunks = 0;
  if (v0 < v1) load_chunk(v0);
  for (int base = v0; base < v1 && ok; base += kTnChunk, ++chunks) {
#pragma unroll
    for (int k = 0; k < kOps; ++k) {
      const int op = warp + k * kWarpsTn;
      if (op >= nops) continue;  // warp-uniform
      const int tb = op * 4 + (lane >> 3);
      const bool isA = tb < na;
      const int t = isA ? tb : tb - na;
      const int cg = t >> 3, vg = t & 7;
      const int m = cg * 8 + (lane & 7);
      const int slice = isA ? 4096 : N * 32;
      const uint32_t addr = smem_addr((isA ? sA : sB) + (vg >> 1) * slice + (m >> 3) * 256 +
                                      (vg & 1) * 128 + (m & 7) * 16);
      asm volatile("stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1, %2, %3, %4};" ::"r"(
                       addr),
                   "r"(frag[k][0]), "r"(frag[k][1]), "r"(frag[k][2]), "r"(frag[k][3])
                   : "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
#pragma unroll
      for (int s = 0; s < kTnChunk / 16; ++s) {
        const uint64_t ad = make_desc(a0 + s * 4096, 128, 256);
        const uint64_t bd = make_desc(b0 + s * (N * 32), 128, 256);
        const uint32_t acc = (chunks > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_addr(&mbar)));
    }
    // the next chunk's fragments in flight while these MMAs run
    if (base + kTnChunk < v1) load_chunk(base + kTnChunk);
    // the chunk's MMAs done (phase = chunk parity) before the buffers are
    // refilled or the accumulator read; bounded
    bool done = false;
    const uint32_t par = (uint32_t)(chunks & 1);
    for (int spin = 0; spin < kSpin && !done; ++spin) {
      uint32_t d;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
          " selp.b32 %0, 1, 0, p;\n}"
          : "=r"(d)
          : "r"(smem_addr(&mbar)), "r"(par));
      done = d != 0;
    }
    ok = __syncthreads_and(done ? 1 : 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (!ok && tid == 0 && err) atomicOr(err, 4);
  // epilogue: row m = warp * 32 + lane of the accumulator; rows < R kept
  const int m = warp * 32 + lane;
  float* out = part + (size_t)blockIdx.x * R * N;
  if (ok && chunks > 0) {
    const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t r[16];
      ld16(tbase + (uint32_t)c0, r);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < R) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(out + (size_t)m * N + c0 + j) =
              make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                          __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
      }
    }
  } else if (m < R) {
    for (int c = 0; c < N; c += 4)
      *reinterpret_cast<float4*>(out + (size_t)m * N + c) = make_float4(0.f, 0.f, 0.f, 0.f);
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
  const int grid = std::max(1, std::min(ceil_div(M, kTileM), num_sms()));
  gemm_tc_kernel<N><<<grid, kPipeThreads, smem, s>>>(A, M, K, B, bias, relu, outb, outf, err);
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

mm_status gemm_tn_partials(const void* A, int n, int R, const void* B, float* part, int parts,
                           int* err, cudaStream_t s) {
  if (n < 0 || (R != 16 && R != 128) || parts < 1 || !A || !B || !part) {
    set_error("gemm_tn: need R in {16, 128}, parts >= 1");
    return MM_ERR_INVALID_ARG;
  }
  if (((uintptr_t)A & 15) || ((uintptr_t)B & 15) || ((uintptr_t)part & 15)) {
    set_error("gemm_tn: A, B and part must be 16-byte aligned");
    return MM_ERR_INVALID_ARG;
  }
  gemm_tn_partial_kernel<<<parts, kGemmThreads, kTnSmem, s>>>(
      (const __nv_bfloat16*)A, n, R, (const __nv_bfloat16*)B, part, err);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

namespace {
// out[i] = sum over p of part[p][i], in order p = 0, 1, ... (FP32)
__global__ void sum_parts_kernel(int parts, int m, const float* __restrict__ part,
                                 float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  float s = 0.f;
  for (int p = 0; p < parts; ++p) s += part[(size_t)p * m + i];
  out[i] = s;
}
}  // namespace

// Three CTAs per SM (24 KB of shared memory and 64 TMEM columns each) keep
// enough operand loads in flight; at most kNetParts partials.
int gemm_tn_parts(int n) {
  return std::max(1, std::min(std::min(3 * num_sms(), kNetParts), ceil_div(n, kTnChunk)));
}

mm_status gemm_tn_bf16(const void* A, int n, int R, const void* B, float* out, float* part,
                       int* err, cudaStream_t s) {
  const int parts = gemm_tn_parts(n);
  MM_TRY(gemm_tn_partials(A, n, R, B, part, parts, err, s));
  sum_parts_kernel<<<ceil_div(R * 64, 256), 256, 0, s>>>(parts, R * 64, part, out);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

mm_status gemm_bf16(const void* A, int M, int K, const void* B, int N, const float* bias,
                    int relu, void* outb, float* outf, int* err, cudaStream_t s) {
  if (M < 0 || (K != 16 && K != 32 && K != 64 && K != 128) || (N != 64 && N != 128) || !A ||
      !B || (!outb && !outf)) {
    set_error("gemm: need K in {16, 32, 64, 128}, N in {64, 128}");
    return MM_ERR_INVALID_ARG;
  }
  if (((uintptr_t)A & 15) || ((uintptr_t)B & 15) || ((uintptr_t)outb & 15) ||
      ((uintptr_t)outf & 15)) {
    set_error("gemm: A, B and the outputs must be 16-byte aligned");
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
