// Device primitives: stable LSD radix sort of (key, int32) pairs and
// exclusive scans.  Written for sm_103a: one tile of 2048 items per 256-thread
// block, 8-bit digits, warp-level stable ranking with match.any.
#include <cuda_runtime.h>

#include "mm_internal.cuh"

namespace mm {

namespace {

constexpr int kRadix = 256;
constexpr int kWarps = kSortThreads / 32;

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K key, int shift) {
  return (uint32_t)(key >> shift) & (kRadix - 1);
}

// counts[d * tiles + b] = number of items of tile b with digit d.
template <typename K>
__global__ void __launch_bounds__(kSortThreads) rs_upsweep(const K* __restrict__ keys, int n,
                                                           int shift, uint32_t* counts,
                                                           int tiles) {
  __shared__ uint32_t hist[kRadix];
  for (int i = threadIdx.x; i < kRadix; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kSortTile + warp * (32 * kSortIPT);
#pragma unroll
  for (int j = 0; j < kSortIPT; ++j) {
    const int64_t idx = base + j * 32 + lane;
    const unsigned valid = __ballot_sync(0xffffffffu, idx < n);
    if (idx < n) {
      const uint32_t d = digit_of(keys[idx], shift);
      const unsigned peers = __match_any_sync(valid, d);
      if (lane == __ffs(peers) - 1) atomicAdd(&hist[d], (uint32_t)__popc(peers));
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kRadix; i += blockDim.x)
    counts[(int64_t)i * tiles + blockIdx.x] = hist[i];
}

// One block per digit: exclusive scan of counts[d][*] in place, totals[d].
__global__ void __launch_bounds__(1024) rs_scan_digits(uint32_t* counts, int tiles,
                                                       uint32_t* totals) {
  __shared__ uint32_t part[1024];
  uint32_t* row = counts + (int64_t)blockIdx.x * tiles;
  const int per = (tiles + blockDim.x - 1) / blockDim.x;
  const int beg = threadIdx.x * per;
  const int end = min(beg + per, tiles);
  uint32_t s = 0;
  for (int i = beg; i < end; ++i) s += row[i];
  part[threadIdx.x] = s;
  __syncthreads();
  // Hillis-Steele inclusive scan over the 1024 partial sums
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int i = beg; i < end; ++i) {
    uint32_t c = row[i];
    row[i] = run;
    run += c;
  }
  if (threadIdx.x == blockDim.x - 1) totals[blockIdx.x] = part[threadIdx.x];
}

// Stable scatter of one tile.  Items of a warp's sub-tile are ranked round by
// round (32 consecutive items per round) with match.any, so the output order
// of equal digits follows the input order.
template <typename K>
__global__ void __launch_bounds__(kSortThreads) rs_downsweep(
    const K* __restrict__ kin, const int32_t* __restrict__ vin, K* __restrict__ kout,
    int32_t* __restrict__ vout, int n, int shift, const uint32_t* __restrict__ counts,
    const uint32_t* __restrict__ totals, int tiles) {
  __shared__ uint32_t whist[kWarps][kRadix];
  __shared__ uint32_t dbase[kRadix];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * kRadix; i += blockDim.x) (&whist[0][0])[i] = 0;
  if (threadIdx.x < 32) {
    // exclusive scan of the 256 digit totals by one warp (8 per lane)
    uint32_t v[8], s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      v[j] = totals[lane * 8 + j];
      s += v[j];
    }
    uint32_t inc = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += t;
    }
    uint32_t run = inc - s;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      dbase[lane * 8 + j] = run;
      run += v[j];
    }
  }
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile + warp * (32 * kSortIPT);
  K key[kSortIPT];
  int32_t val[kSortIPT];
  uint32_t dig[kSortIPT];
  unsigned peers[kSortIPT];
#pragma unroll
  for (int j = 0; j < kSortIPT; ++j) {
    const int64_t idx = base + j * 32 + lane;
    const unsigned valid = __ballot_sync(0xffffffffu, idx < n);
    peers[j] = 0;
    if (idx < n) {
      key[j] = kin[idx];
      val[j] = vin[idx];
      dig[j] = digit_of(key[j], shift);
      peers[j] = __match_any_sync(valid, dig[j]);
      if (lane == __ffs(peers[j]) - 1) whist[warp][dig[j]] += __popc(peers[j]);
    }
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive prefix over warps plus the tile's global offset
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
    uint32_t run = dbase[d] + counts[(int64_t)d * tiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      uint32_t c = whist[w][d];
      whist[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < kSortIPT; ++j) {
    uint32_t pos = 0;
    const bool valid = peers[j] != 0;
    if (valid) pos = whist[warp][dig[j]] + __popc(peers[j] & lt);
    __syncwarp();
    if (valid && lane == __ffs(peers[j]) - 1) whist[warp][dig[j]] += __popc(peers[j]);
    __syncwarp();
    if (valid) {
      kout[pos] = key[j];
      vout[pos] = val[j];
    }
  }
}

template <typename K>
mm_status radix_sort(K* k0, K* k1, int32_t* v0, int32_t* v1, int n, int begin_bit,
                     int end_bit, SortWS& ws, cudaStream_t s, K** ko, int32_t** vo) {
  K* kin = k0;
  K* kalt = k1;
  int32_t* vin = v0;
  int32_t* valt = v1;
  if (n > 1) {
    const int tiles = ceil_div(n, kSortTile);
    if (tiles > ws.max_tiles) {
      set_error("radix sort of %d items exceeds its workspace", n);
      return MM_ERR_INVALID_ARG;
    }
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
      rs_upsweep<K><<<tiles, kSortThreads, 0, s>>>(kin, n, shift, ws.counts, tiles);
      rs_scan_digits<<<kRadix, 1024, 0, s>>>(ws.counts, tiles, ws.totals);
      rs_downsweep<K><<<tiles, kSortThreads, 0, s>>>(kin, vin, kalt, valt, n, shift, ws.counts,
                                                     ws.totals, tiles);
      K* tk = kin; kin = kalt; kalt = tk;
      int32_t* tv = vin; vin = valt; valt = tv;
    }
    MM_CK(cudaGetLastError());
  }
  *ko = kin;
  *vo = vin;
  return MM_OK;
}

// ------------------------------------------------------------------ scan --
constexpr int kScanThreads = 256;
constexpr int kScanIPT = 16;
constexpr int kScanTile = kScanThreads * kScanIPT;

template <typename T>
__device__ __forceinline__ T block_exclusive(T v, T* sh, T* total) {
  // sh: kScanThreads/32 entries
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T inc = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += t;
  }
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < kScanThreads / 32 ? sh[lane] : 0;
    T winc = w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      T t = __shfl_up_sync(0xffffffffu, winc, off);
      if (lane >= off) winc += t;
    }
    if (lane < kScanThreads / 32) sh[lane] = winc - w;
    if (lane == kScanThreads / 32 - 1) *total = winc;
  }
  __syncthreads();
  T r = sh[warp] + inc - v;
  __syncthreads();
  return r;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_tiles(const int32_t* __restrict__ in,
                                                           T* __restrict__ out, int n,
                                                           T* __restrict__ tile_sums) {
  __shared__ T sh[kScanThreads / 32];
  __shared__ T total;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanIPT;
  T v[kScanIPT];
  T s = 0;
#pragma unroll
  for (int j = 0; j < kScanIPT; ++j) {
    v[j] = base + j < n ? (T)in[base + j] : (T)0;
    s += v[j];
  }
  T run = block_exclusive<T>(s, sh, &total);
#pragma unroll
  for (int j = 0; j < kScanIPT; ++j) {
    if (base + j < n) out[base + j] = run;
    run += v[j];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

template <typename T>
__global__ void __launch_bounds__(1024) scan_sums(T* sums, int m, T* grand) {
  __shared__ T part[1024];
  const int per = (m + blockDim.x - 1) / blockDim.x;
  const int beg = threadIdx.x * per;
  const int end = min(beg + per, m);
  T s = 0;
  for (int i = beg; i < end; ++i) s += sums[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    T v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  T run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int i = beg; i < end; ++i) {
    T c = sums[i];
    sums[i] = run;
    run += c;
  }
  if (threadIdx.x == blockDim.x - 1) *grand = part[threadIdx.x];
}

template <typename T>
__global__ void scan_add(T* out, int n, const T* tile_offsets) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += tile_offsets[i / kScanTile];
}

template <typename T>
mm_status scan_exclusive(const int32_t* in, T* out, int n, void* ws, cudaStream_t s) {
  const int tiles = ceil_div(n, kScanTile);
  T* sums = (T*)ws;
  if (n <= 0) {
    MM_CK(cudaMemsetAsync(out, 0, sizeof(T), s));
    return MM_OK;
  }
  scan_tiles<T><<<tiles, kScanThreads, 0, s>>>(in, out, n, sums);
  scan_sums<T><<<1, 1024, 0, s>>>(sums, tiles, out + n);
  if (tiles > 1) scan_add<T><<<ceil_div(n, 256), 256, 0, s>>>(out, n, sums);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

}  // namespace

mm_status sort_ws_alloc(SortWS& ws, int64_t max_n) {
  ws.max_tiles = ceil_div(max_n > 0 ? max_n : 1, kSortTile);
  MM_CK(cudaMalloc(&ws.counts, sizeof(uint32_t) * kRadix * (size_t)ws.max_tiles));
  MM_CK(cudaMalloc(&ws.totals, sizeof(uint32_t) * kRadix));
  return MM_OK;
}

void sort_ws_free(SortWS& ws) {
  cudaFree(ws.counts);
  cudaFree(ws.totals);
  ws = SortWS();
}

mm_status radix_sort_u32(uint32_t* k0, uint32_t* k1, int32_t* v0, int32_t* v1, int n,
                         int begin_bit, int end_bit, SortWS& ws, cudaStream_t s,
                         uint32_t** keys_out, int32_t** vals_out) {
  return radix_sort<uint32_t>(k0, k1, v0, v1, n, begin_bit, end_bit, ws, s, keys_out, vals_out);
}

mm_status radix_sort_u64(uint64_t* k0, uint64_t* k1, int32_t* v0, int32_t* v1, int n,
                         int begin_bit, int end_bit, SortWS& ws, cudaStream_t s,
                         uint64_t** keys_out, int32_t** vals_out) {
  return radix_sort<uint64_t>(k0, k1, v0, v1, n, begin_bit, end_bit, ws, s, keys_out, vals_out);
}

size_t scan_ws_bytes(int64_t n) {
  return sizeof(int64_t) * (size_t)(ceil_div(n > 0 ? n : 1, kScanTile) + 1);
}

mm_status scan_exclusive_i32(const int32_t* in, int32_t* out, int n, void* ws, cudaStream_t s) {
  return scan_exclusive<int32_t>(in, out, n, ws, s);
}

mm_status scan_exclusive_i64(const int32_t* in, int64_t* out, int n, void* ws, cudaStream_t s) {
  return scan_exclusive<int64_t>(in, out, n, ws, s);
}

}  // namespace mm
