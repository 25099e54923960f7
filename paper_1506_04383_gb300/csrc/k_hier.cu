// Hierarchy construction on the device (Sec. 3.1) and the per-level pair
// set S (Sec. 2.3 footnote, Sec. 3.2):
//   * input validation (CSR shape, sorted rows, symmetry, no self-loops);
//   * k-hop S with shortest <=k-hop distances (k = 1 copies E; k = 2
//     enumerates 1- and 2-hop paths, sorts (u, v) keys and keeps the minimum
//     length per pair);
//   * size-constrained label propagation (synchronous rounds in two seeded
//     halves, warp per vertex with a shared-memory hash of neighbouring
//     clusters, concurrent moves into a cluster admitted in seeded priority
//     order while the size bound holds);
//   * contraction (rank relabelling, sorted coarse edge keys, weights summed
//     in fine-entry order).
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <vector>

#include "mm_internal.cuh"

namespace mm {

namespace {

// RAII device buffer for temporaries of the build phase, stream-ordered
// (cudaMallocAsync / cudaFreeAsync never synchronise the device, so builds on
// different streams -- the graphs of a batch -- overlap).
struct Tmp {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  ~Tmp() {
    if (p) cudaFreeAsync(p, s);
  }
  template <typename T>
  T* as() const { return (T*)p; }
};

mm_status tmp_alloc(Tmp& t, size_t bytes, cudaStream_t s) {
  t.s = s;
  MM_CK(cudaMallocAsync(&t.p, bytes > 0 ? bytes : 16, s));
  return MM_OK;
}

// Sort workspace on the stream's pool.
struct TmpSort {
  SortWS ws;
  cudaStream_t s = nullptr;
  ~TmpSort() {
    if (ws.counts) cudaFreeAsync(ws.counts, s);
    if (ws.totals) cudaFreeAsync(ws.totals, s);
  }
};

mm_status tmp_sort(TmpSort& t, int64_t max_n, cudaStream_t s) {
  t.s = s;
  t.ws.max_tiles = ceil_div(max_n > 0 ? max_n : 1, kSortTile);
  MM_CK(cudaMallocAsync(&t.ws.counts, sizeof(uint32_t) * 256 * (size_t)t.ws.max_tiles, s));
  MM_CK(cudaMallocAsync(&t.ws.totals, sizeof(uint32_t) * 256, s));
  return MM_OK;
}

int bits_for(int64_t v) {  // bits needed to hold values in [0, v]
  int b = 1;
  while (b < 62 && ((int64_t)1 << b) <= v) ++b;
  return b;
}

// ------------------------------------------------------------ validation --
enum : int {
  kBadRowPtr = 1, kBadCol = 2, kSelfLoop = 4, kUnsorted = 8, kAsym = 16
};

__global__ void validate_kernel(int n, int64_t nnz, const int64_t* __restrict__ rp,
                                const int32_t* __restrict__ col, int32_t* rp32, int* flags) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u > n) return;
  const int64_t b = rp[u];
  rp32[u] = (int32_t)b;
  if (u == 0 && b != 0) atomicOr(flags, kBadRowPtr);
  if (u == n) {
    if (b != nnz) atomicOr(flags, kBadRowPtr);
    return;
  }
  const int64_t e = rp[u + 1];
  if (e < b || e > nnz) {
    atomicOr(flags, kBadRowPtr);
    return;
  }
  int prev = -1;
  for (int64_t i = b; i < e; ++i) {
    const int v = col[i];
    if (v < 0 || v >= n) { atomicOr(flags, kBadCol); return; }
    if (v == u) atomicOr(flags, kSelfLoop);
    if (v <= prev) atomicOr(flags, kUnsorted);
    prev = v;
    // symmetry: u must appear in row v (binary search; rows sorted)
    int64_t lo = rp[v], hi = rp[v + 1] - 1;
    if (lo < 0 || hi >= nnz) { atomicOr(flags, kBadRowPtr); return; }
    bool found = false;
    while (lo <= hi) {
      const int64_t mid = (lo + hi) >> 1;
      const int w = col[mid];
      if (w == u) { found = true; break; }
      if (w < u) lo = mid + 1; else hi = mid - 1;
    }
    if (!found) atomicOr(flags, kAsym);
  }
}

// ------------------------------------------------------------ k-hop S ---
__device__ __forceinline__ float edge_length(const float* c, const float* elen, int e, int a,
                                             int b) {
  if (c) return sqrtf(c[a]) + sqrtf(c[b]);
  return elen ? elen[e] : 1.f;
}

__global__ void khop1_kernel(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const float* __restrict__ c, const float* __restrict__ elen,
                             int32_t* sp, SEnt* S, float* rho) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u > n) return;
  sp[u] = rp[u];
  if (u == n) return;
  float r = 0.f;
  for (int e = rp[u]; e < rp[u + 1]; ++e) {
    const int v = col[e];
    const float d = edge_length(c, elen, e, u, v);
    S[e].col = v;
    S[e].d = d;
    r += 1.f / (d * d);
  }
  rho[u] = r;
}

__global__ void khop2_count(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                            int32_t* cnt) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  int64_t s = rp[u + 1] - rp[u];
  for (int e = rp[u]; e < rp[u + 1]; ++e) {
    const int w = col[e];
    s += rp[w + 1] - rp[w];
  }
  cnt[u] = (int32_t)min(s, (int64_t)0x7fffffff);
}

// Emits (u, v, length) for every path of one or two edges out of u.
__global__ void khop2_emit(int n, int vb, const int32_t* __restrict__ rp,
                           const int32_t* __restrict__ col, const float* __restrict__ c,
                           const float* __restrict__ elen, const int64_t* __restrict__ off,
                           uint64_t* keys, int32_t* dbits) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  int64_t o = off[u];
  for (int e = rp[u]; e < rp[u + 1]; ++e) {
    const int w = col[e];
    const float l1 = edge_length(c, elen, e, u, w);
    keys[o] = ((uint64_t)u << vb) | (uint64_t)w;
    dbits[o] = __float_as_int(l1);
    ++o;
    for (int f = rp[w]; f < rp[w + 1]; ++f) {
      const int v = col[f];
      const float l2 = l1 + edge_length(c, elen, f, w, v);
      // the path back to u itself is padded with an impossible key (u, u)
      keys[o] = ((uint64_t)u << vb) | (uint64_t)(v == u ? u : v);
      dbits[o] = v == u ? __float_as_int(CUDART_INF_F) : __float_as_int(l2);
      ++o;
    }
  }
}

__global__ void run_heads(int m, const uint64_t* __restrict__ keys, int32_t* head) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

// One thread per run of equal (u, v) keys: minimum length, skipping (u, u).
__global__ void khop2_reduce(int m, int vb, const uint64_t* __restrict__ keys,
                             const int32_t* __restrict__ dbits, const int32_t* __restrict__ head,
                             const int32_t* __restrict__ pos, SEnt* S, int32_t* rowcnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m || !head[i]) return;
  const uint64_t k = keys[i];
  const int u = (int)(k >> vb);
  const int v = (int)(k & (((uint64_t)1 << vb) - 1));
  float d = __int_as_float(dbits[i]);
  for (int j = i + 1; j < m && keys[j] == k; ++j) d = fminf(d, __int_as_float(dbits[j]));
  S[pos[i]].col = v;
  S[pos[i]].d = d;
  if (u != v) atomicAdd(&rowcnt[u], 1);
}

// Removes the (u, u) padding entries while copying into the final rows.
__global__ void khop2_finish(int n, const int32_t* __restrict__ sp_tmp, const SEnt* __restrict__ S_tmp,
                             const int32_t* __restrict__ sp, SEnt* S, float* rho) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  int o = sp[u];
  float r = 0.f;
  for (int i = sp_tmp[u]; i < sp_tmp[u + 1]; ++i) {
    const SEnt en = S_tmp[i];
    if (en.col == u) continue;
    S[o++] = en;
    r += 1.f / (en.d * en.d);
  }
  rho[u] = r;
}

// Row starts of the unique (u, v) runs: counts every run including (u, u).
__global__ void count_runs(int m, int vb, const uint64_t* __restrict__ keys,
                           const int32_t* __restrict__ head, int32_t* cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m || !head[i]) return;
  atomicAdd(&cnt[(int)(keys[i] >> vb)], 1);
}

// ------------------------------------------------- label propagation ----
constexpr int kLPWarps = 4;
constexpr int kLPHash = 1024;  // distinct neighbouring clusters per vertex
constexpr int kLPHeavyDeg = kLPHash / 2;  // longer rows: a block and a global hash each
constexpr int kLPHeavyT = 256;

__global__ void __launch_bounds__(kLPWarps * 32) lp_propose(
    int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
    const float* __restrict__ omega, const float* __restrict__ c, const float* __restrict__ W,
    const int32_t* __restrict__ labels, float U, uint32_t k0, uint32_t k1, uint32_t round,
    uint32_t level, uint32_t half, int tb, uint64_t* keys, int32_t* vals) {
  __shared__ int32_t hk[kLPWarps][kLPHash];
  __shared__ float hv[kLPWarps][kLPHash];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int v = blockIdx.x * kLPWarps + wl;
  if (v >= n) return;
  uint32_t z[4];
  philox4x32_10((uint32_t)v, round, level, 2u, k0, k1, z);
  const uint64_t none = ~(uint64_t)0;
  vals[v] = v;
  if ((z[0] & 1u) != half) {
    if (lane == 0) keys[v] = none;
    return;
  }
  // more neighbours than half the hash: lp_propose_heavy decides
  if (rp[v + 1] - rp[v] > kLPHeavyDeg) return;
  for (int i = lane; i < kLPHash; i += 32) { hk[wl][i] = -1; hv[wl][i] = 0.f; }
  __syncwarp();
  for (int e = rp[v] + lane; e < rp[v + 1]; e += 32) {
    const int L = labels[col[e]];
    const float w = omega ? omega[e] : 1.f;
    uint32_t hsh = ((uint32_t)L * 2654435761u) & (kLPHash - 1);
    for (int probe = 0; probe < kLPHash; ++probe) {
      const int prev = atomicCAS(&hk[wl][hsh], -1, L);
      if (prev == -1 || prev == L) {
        atomicAdd(&hv[wl][hsh], w);
        break;
      }
      hsh = (hsh + 1) & (kLPHash - 1);
    }
  }
  __syncwarp();
  const int own = labels[v];
  const float cv = c[v];
  // best eligible cluster: max connection, then smallest label
  float best = -1.f;
  int bestL = 0x7fffffff;
  float ownc = 0.f;
  for (int i = lane; i < kLPHash; i += 32) {
    const int L = hk[wl][i];
    if (L < 0) continue;
    const float cn = hv[wl][i];
    if (L == own) { ownc = cn; continue; }
    if (W[L] + cv > U) continue;
    if (cn > best || (cn == best && L < bestL)) { best = cn; bestL = L; }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oL = __shfl_xor_sync(0xffffffffu, bestL, o);
    ownc += __shfl_xor_sync(0xffffffffu, ownc, o);
    if (ob > best || (ob == best && oL < bestL)) { best = ob; bestL = oL; }
  }
  if (lane == 0) {
    // stay unless another eligible cluster is strictly better connected
    if (best > ownc && bestL != 0x7fffffff)
      keys[v] = ((uint64_t)bestL << 8) | (uint64_t)(z[1] >> 24);
    else
      keys[v] = none;
  }
  (void)tb;
}

// The proposal of a vertex with more than kLPHeavyDeg neighbours (hubs of
// power-law graphs): one block per vertex, connection weights per
// neighbouring cluster in an open-addressing hash of T >= 2 deg slots in
// global scratch, then the same choice as lp_propose (best eligible
// cluster, ties to the smallest label, stay unless strictly better).
__global__ void __launch_bounds__(kLPHeavyT) lp_propose_heavy(
    const int32_t* __restrict__ hl, const int64_t* __restrict__ hoff,
    const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
    const float* __restrict__ omega, const float* __restrict__ c, const float* __restrict__ W,
    const int32_t* __restrict__ labels, float U, uint32_t k0, uint32_t k1, uint32_t round,
    uint32_t level, uint32_t half, int32_t* hkey, float* hval, uint64_t* keys) {
  const int v = hl[blockIdx.x];
  uint32_t z[4];
  philox4x32_10((uint32_t)v, round, level, 2u, k0, k1, z);
  if ((z[0] & 1u) != half) return;  // lp_propose wrote "stay"
  const int64_t base = hoff[blockIdx.x];
  const int T = (int)(hoff[blockIdx.x + 1] - base);  // a power of two
  int32_t* hk = hkey + base;
  float* hv = hval + base;
  for (int i = threadIdx.x; i < T; i += kLPHeavyT) {
    hk[i] = -1;
    hv[i] = 0.f;
  }
  __syncthreads();
  for (int e = rp[v] + threadIdx.x; e < rp[v + 1]; e += kLPHeavyT) {
    const int L = labels[col[e]];
    const float w = omega ? omega[e] : 1.f;
    uint32_t h = ((uint32_t)L * 2654435761u) & (uint32_t)(T - 1);
    for (int probe = 0; probe < T; ++probe) {
      const int prev = atomicCAS(&hk[h], -1, L);
      if (prev == -1 || prev == L) {
        atomicAdd(&hv[h], w);
        break;
      }
      h = (h + 1) & (uint32_t)(T - 1);
    }
  }
  __syncthreads();
  const int own = labels[v];
  const float cv = c[v];
  float best = -1.f, ownc = 0.f;
  int bestL = 0x7fffffff;
  for (int i = threadIdx.x; i < T; i += kLPHeavyT) {
    const int L = __ldcg(&hk[i]);
    if (L < 0) continue;
    const float cn = __ldcg(&hv[i]);
    if (L == own) { ownc = cn; continue; }
    if (W[L] + cv > U) continue;
    if (cn > best || (cn == best && L < bestL)) { best = cn; bestL = L; }
  }
  __shared__ float sb[kLPHeavyT / 32], so[kLPHeavyT / 32];
  __shared__ int sl[kLPHeavyT / 32];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oL = __shfl_xor_sync(0xffffffffu, bestL, o);
    ownc += __shfl_xor_sync(0xffffffffu, ownc, o);
    if (ob > best || (ob == best && oL < bestL)) { best = ob; bestL = oL; }
  }
  if (lane == 0) { sb[wp] = best; sl[wp] = bestL; so[wp] = ownc; }
  __syncthreads();
  if (threadIdx.x == 0) {
    best = sb[0]; bestL = sl[0]; ownc = so[0];
    for (int k = 1; k < kLPHeavyT / 32; ++k) {
      ownc += so[k];
      if (sb[k] > best || (sb[k] == best && sl[k] < bestL)) { best = sb[k]; bestL = sl[k]; }
    }
    keys[v] = (best > ownc && bestL != 0x7fffffff) ? (((uint64_t)bestL << 8) | (uint64_t)(z[1] >> 24))
                                                  : ~(uint64_t)0;
  }
}

// Hash size of heavy vertex i: the power of two >= 2 deg.
__global__ void lp_heavy_sizes(int m, const int32_t* __restrict__ hl,
                               const int32_t* __restrict__ rp, int32_t* size) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int d = rp[hl[i] + 1] - rp[hl[i]];
  int T = 1;
  while (T < 2 * d) T <<= 1;
  size[i] = T;
}

__global__ void max_row_kernel(int n, const int32_t* __restrict__ rp, int32_t* out) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n) atomicMax(out, rp[u + 1] - rp[u]);
}

// One thread per run of movers into the same cluster (sorted by priority):
// admit while the cluster weight stays <= U.
__global__ void lp_admit(int n, const uint64_t* __restrict__ keys, const int32_t* __restrict__ vals,
                         const float* __restrict__ c, const float* __restrict__ W, float U,
                         int32_t* labels, int* moved) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t k = keys[i];
  if (k == ~(uint64_t)0) return;
  const int T = (int)(k >> 8);
  if (i > 0 && (int)(keys[i - 1] >> 8) == T && keys[i - 1] != ~(uint64_t)0) return;
  float acc = W[T];
  for (int j = i; j < n && keys[j] != ~(uint64_t)0 && (int)(keys[j] >> 8) == T; ++j) {
    const int v = vals[j];
    if (acc + c[v] <= U) {
      acc += c[v];
      labels[v] = T;
      atomicAdd(moved, 1);
    }
  }
}

// The whole label propagation of a level of at most kLPSmallN vertices in
// one CTA, with the semantics of the multi-kernel rounds above: per round
// two seeded halves; per half, every active vertex proposes its best
// eligible neighbouring cluster (shared-memory hash per warp), movers are
// ordered by (target, priority, vertex) with a bitonic sort and admitted
// while the target's weight stays <= U, weights are recomputed.  Stops after
// a round without moves (the labels are then a fixed point).
constexpr int kLPSmallN = 4096;
constexpr int kLPSmallT = 1024;
constexpr int kLPSmallHash = 512;

struct LPSmem {
  int32_t hk[kLPSmallT / 32][kLPSmallHash];
  float hv[kLPSmallT / 32][kLPSmallHash];
  unsigned long long key[kLPSmallN];
  int32_t lab[kLPSmallN];
  float W[kLPSmallN];
  float cv[kLPSmallN];
};

__global__ void __launch_bounds__(kLPSmallT, 1) lp_small_kernel(
    int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
    const float* __restrict__ omega, const float* __restrict__ c, float U, int rounds,
    uint32_t k0, uint32_t k1, uint32_t level, int32_t* labels) {
  extern __shared__ __align__(16) unsigned char lp_raw[];
  LPSmem& s = *reinterpret_cast<LPSmem*>(lp_raw);
  __shared__ int moved;
  const int tid = threadIdx.x, lane = tid & 31, wl = tid >> 5;
  const unsigned long long none = ~0ull;
  for (int v = tid; v < n; v += kLPSmallT) {
    s.lab[v] = v;
    s.W[v] = c[v];
    s.cv[v] = c[v];
  }
  int np = 2;
  while (np < n) np <<= 1;
  __syncthreads();
  for (int r = 0; r < rounds; ++r) {
    if (tid == 0) moved = 0;
    for (uint32_t half = 0; half < 2; ++half) {
      // proposals, one warp per vertex
      for (int v = wl; v < np; v += kLPSmallT / 32) {
        if (v >= n) {
          if (lane == 0) s.key[v] = none;
          continue;
        }
        uint32_t z[4];
        philox4x32_10((uint32_t)v, (uint32_t)r, level, 2u, k0, k1, z);
        if ((z[0] & 1u) != half) {
          if (lane == 0) s.key[v] = none;
          continue;
        }
        for (int i = lane; i < kLPSmallHash; i += 32) { s.hk[wl][i] = -1; s.hv[wl][i] = 0.f; }
        __syncwarp();
        for (int e = rp[v] + lane; e < rp[v + 1]; e += 32) {
          const int L = s.lab[col[e]];
          const float w = omega ? omega[e] : 1.f;
          uint32_t hsh = ((uint32_t)L * 2654435761u) & (kLPSmallHash - 1);
          for (int probe = 0; probe < kLPSmallHash; ++probe) {
            const int prev = atomicCAS(&s.hk[wl][hsh], -1, L);
            if (prev == -1 || prev == L) {
              atomicAdd(&s.hv[wl][hsh], w);
              break;
            }
            hsh = (hsh + 1) & (kLPSmallHash - 1);
          }
        }
        __syncwarp();
        const int own = s.lab[v];
        const float cvv = s.cv[v];
        float best = -1.f, ownc = 0.f;
        int bestL = 0x7fffffff;
        for (int i = lane; i < kLPSmallHash; i += 32) {
          const int L = s.hk[wl][i];
          if (L < 0) continue;
          const float cn = s.hv[wl][i];
          if (L == own) { ownc = cn; continue; }
          if (s.W[L] + cvv > U) continue;
          if (cn > best || (cn == best && L < bestL)) { best = cn; bestL = L; }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          const float ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oL = __shfl_xor_sync(0xffffffffu, bestL, o);
          ownc += __shfl_xor_sync(0xffffffffu, ownc, o);
          if (ob > best || (ob == best && oL < bestL)) { best = ob; bestL = oL; }
        }
        if (lane == 0)
          s.key[v] = (best > ownc && bestL != 0x7fffffff)
                         ? ((unsigned long long)bestL << 44) |
                               ((unsigned long long)(z[1] >> 24) << 12) | (unsigned long long)v
                         : none;
        __syncwarp();
      }
      __syncthreads();
      // order movers by (target, priority, vertex)
      for (int k = 2; k <= np; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int i = tid; i < np; i += kLPSmallT) {
            const int ij = i ^ j;
            if (ij > i) {
              const unsigned long long a = s.key[i], b = s.key[ij];
              if ((a > b) == ((i & k) == 0)) { s.key[i] = b; s.key[ij] = a; }
            }
          }
          __syncthreads();
        }
      // admission per target run
      for (int i = tid; i < n; i += kLPSmallT) {
        const unsigned long long k = s.key[i];
        if (k == none) continue;
        const int T = (int)(k >> 44);
        if (i > 0 && s.key[i - 1] != none && (int)(s.key[i - 1] >> 44) == T) continue;
        float acc = s.W[T];
        for (int j = i; j < n && s.key[j] != none && (int)(s.key[j] >> 44) == T; ++j) {
          const int v = (int)(s.key[j] & 0xfffull);
          if (acc + s.cv[v] <= U) {
            acc += s.cv[v];
            s.lab[v] = T;
            atomicAdd(&moved, 1);
          }
        }
      }
      __syncthreads();
      for (int v = tid; v < n; v += kLPSmallT) s.W[v] = 0.f;
      __syncthreads();
      for (int v = tid; v < n; v += kLPSmallT) atomicAdd(&s.W[s.lab[v]], s.cv[v]);
      __syncthreads();
    }
    if (moved == 0) break;
    __syncthreads();
  }
  for (int v = tid; v < n; v += kLPSmallT) labels[v] = s.lab[v];
}

__global__ void lp_init(int n, const float* __restrict__ c, int32_t* labels, float* W) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  labels[v] = v;
  W[v] = c[v];
}

__global__ void lp_weights(int n, const float* __restrict__ c, const int32_t* __restrict__ labels,
                           float* W) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  atomicAdd(&W[labels[v]], c[v]);
}

// ------------------------------------------------------------ contraction --
__global__ void mark_used(int n, const int32_t* __restrict__ labels, int32_t* used) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) used[labels[v]] = 1;
}

__global__ void apply_map(int n, const int32_t* __restrict__ labels, const int32_t* __restrict__ rank,
                          const float* __restrict__ c, int32_t* map, float* cc) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int m = rank[labels[v]];
  map[v] = m;
  atomicAdd(&cc[m], c[v]);
}

__global__ void cut_flags(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const int32_t* __restrict__ map, int32_t* flag) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  const int mu = map[u];
  for (int e = rp[u]; e < rp[u + 1]; ++e) flag[e] = map[col[e]] != mu ? 1 : 0;
}

__global__ void cut_emit(int n, int cb, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                         const int32_t* __restrict__ map, const int32_t* __restrict__ pos,
                         uint64_t* keys, int32_t* vals) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  const int mu = map[u];
  for (int e = rp[u]; e < rp[u + 1]; ++e) {
    const int mv = map[col[e]];
    if (mv == mu) continue;
    keys[pos[e]] = ((uint64_t)mu << cb) | (uint64_t)mv;
    vals[pos[e]] = e;
  }
}

__global__ void coarse_reduce(int m, int cb, const uint64_t* __restrict__ keys,
                              const int32_t* __restrict__ vals, const float* __restrict__ omega,
                              const int32_t* __restrict__ head, const int32_t* __restrict__ pos,
                              int32_t* ccol, float* comega, int32_t* rowcnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m || !head[i]) return;
  const uint64_t k = keys[i];
  float w = 0.f;
  for (int j = i; j < m && keys[j] == k; ++j) w += omega ? omega[vals[j]] : 1.f;
  ccol[pos[i]] = (int)(k & (((uint64_t)1 << cb) - 1));
  comega[pos[i]] = w;
  atomicAdd(&rowcnt[(int)(k >> cb)], 1);
}

// Rows longer than thr are "heavy": flag them (and track the longest row).
__global__ void heavy_flags_kernel(int n, const int32_t* __restrict__ sp, int thr,
                                   int32_t* flag, int32_t* maxdeg) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  const int d = sp[u + 1] - sp[u];
  atomicMax(maxdeg, d);
  flag[u] = d > thr ? 1 : 0;
}

// Ordered compaction: heavy row u goes to slot pos[u] (ascending u).
__global__ void heavy_list_kernel(int n, const int32_t* __restrict__ flag,
                                  const int32_t* __restrict__ pos, int32_t* list) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n && flag[u]) list[pos[u]] = u;
}

}  // namespace

mm_status validate_graph(int n, int64_t nnz, const int64_t* rp64, const int32_t* col,
                         int32_t* rp32_out, cudaStream_t s) {
  Tmp fl;
  MM_TRY(tmp_alloc(fl, sizeof(int), s));
  MM_CK(cudaMemsetAsync(fl.p, 0, sizeof(int), s));
  validate_kernel<<<ceil_div(n + 1, 256), 256, 0, s>>>(n, nnz, rp64, col, rp32_out, fl.as<int>());
  MM_CK(cudaGetLastError());
  int flags = 0;
  MM_TRY(read_scalar(fl.p, &flags, s));
  MM_CK(cudaStreamSynchronize(s));
  if (flags) {
    set_error("malformed graph:%s%s%s%s%s", (flags & kBadRowPtr) ? " row_ptr" : "",
              (flags & kBadCol) ? " col-out-of-range" : "", (flags & kSelfLoop) ? " self-loop" : "",
              (flags & kUnsorted) ? " unsorted-or-duplicate-row" : "",
              (flags & kAsym) ? " asymmetric" : "");
    return MM_ERR_INVALID_ARG;
  }
  return MM_OK;
}

mm_status build_khop(int n, const int32_t* rp, const int32_t* col, const float* elen,
                     const float* c, int k, int32_t** sp_out, SEnt** s_out, float** rho_out,
                     int64_t* nnz_out, cudaStream_t s) {
  if (k != 1 && k != 2) {
    set_error("k = %d: the device S builder supports k = 1 and k = 2", k);
    return MM_ERR_UNSUPPORTED;
  }
  int32_t nnzE = 0;
  MM_TRY(read_scalar(rp + n, &nnzE, s));
  MM_CK(cudaStreamSynchronize(s));
  int32_t* sp = nullptr;
  SEnt* S = nullptr;
  float* rho = nullptr;
  MM_CK(cudaMallocAsync(&sp, sizeof(int32_t) * (size_t)(n + 1), s));
  MM_CK(cudaMallocAsync(&rho, sizeof(float) * (size_t)std::max(n, 1), s));
  *sp_out = sp;
  *rho_out = rho;
  if (k == 1) {
    MM_CK(cudaMallocAsync(&S, sizeof(SEnt) * (size_t)std::max(nnzE, 1), s));
    *s_out = S;
    khop1_kernel<<<ceil_div(n + 1, 256), 256, 0, s>>>(n, rp, col, c, elen, sp, S, rho);
    MM_CK(cudaGetLastError());
    *nnz_out = nnzE;
    return MM_OK;
  }
  // k = 2: enumerate paths of one and two edges
  Tmp cnt, off, scan_ws;
  MM_TRY(tmp_alloc(cnt, sizeof(int32_t) * (size_t)(n + 1), s));
  MM_TRY(tmp_alloc(off, sizeof(int64_t) * (size_t)(n + 1), s));
  MM_TRY(tmp_alloc(scan_ws, scan_ws_bytes(std::max<int64_t>(n, 1)) + 64, s));
  khop2_count<<<ceil_div(n, 256), 256, 0, s>>>(n, rp, col, cnt.as<int32_t>());
  MM_TRY(scan_exclusive_i64(cnt.as<int32_t>(), off.as<int64_t>(), n, scan_ws.p, s));
  int64_t m64 = 0;
  MM_TRY(read_scalar(off.as<int64_t>() + n, &m64, s));
  MM_CK(cudaStreamSynchronize(s));
  if (m64 >= 0x7fffffffLL) {
    set_error("2-hop enumeration has %lld paths (limit 2^31-1)", (long long)m64);
    return MM_ERR_UNSUPPORTED;
  }
  const int m = (int)m64;
  const int vb = bits_for(std::max(n - 1, 1));
  const int ub = bits_for(std::max(n - 1, 1));
  Tmp k0, k1, d0, d1, head, pos, rowcnt, sp_tmp, S_tmp, ws2;
  MM_TRY(tmp_alloc(k0, sizeof(uint64_t) * (size_t)std::max(m, 1), s));
  MM_TRY(tmp_alloc(k1, sizeof(uint64_t) * (size_t)std::max(m, 1), s));
  MM_TRY(tmp_alloc(d0, sizeof(int32_t) * (size_t)std::max(m, 1), s));
  MM_TRY(tmp_alloc(d1, sizeof(int32_t) * (size_t)std::max(m, 1), s));
  khop2_emit<<<ceil_div(n, 256), 256, 0, s>>>(n, vb, rp, col, c, elen, off.as<int64_t>(),
                                              k0.as<uint64_t>(), d0.as<int32_t>());
  MM_CK(cudaGetLastError());
  TmpSort sws;
  MM_TRY(tmp_sort(sws, std::max(m, 1), s));
  uint64_t* keys;
  int32_t* dbits;
  MM_TRY(radix_sort_u64(k0.as<uint64_t>(), k1.as<uint64_t>(), d0.as<int32_t>(),
                        d1.as<int32_t>(), m, 0, ub + vb, sws.ws, s, &keys, &dbits));
  MM_TRY(tmp_alloc(head, sizeof(int32_t) * (size_t)std::max(m, 1), s));
  MM_TRY(tmp_alloc(pos, sizeof(int32_t) * (size_t)(m + 1), s));
  MM_TRY(tmp_alloc(ws2, scan_ws_bytes(std::max(m, 1)) + 64, s));
  MM_TRY(tmp_alloc(rowcnt, sizeof(int32_t) * (size_t)(n + 1), s));
  MM_TRY(tmp_alloc(sp_tmp, sizeof(int32_t) * (size_t)(n + 1), s));
  run_heads<<<ceil_div(std::max(m, 1), 256), 256, 0, s>>>(m, keys, head.as<int32_t>());
  MM_TRY(scan_exclusive_i32(head.as<int32_t>(), pos.as<int32_t>(), m, ws2.p, s));
  int32_t uniq = 0;
  MM_TRY(read_scalar(pos.as<int32_t>() + m, &uniq, s));
  MM_CK(cudaStreamSynchronize(s));
  MM_TRY(tmp_alloc(S_tmp, sizeof(SEnt) * (size_t)std::max(uniq, 1), s));
  // temporary rows include the (u, u) padding runs
  MM_CK(cudaMemsetAsync(rowcnt.p, 0, sizeof(int32_t) * (size_t)(n + 1), s));
  count_runs<<<ceil_div(std::max(m, 1), 256), 256, 0, s>>>(m, vb, keys, head.as<int32_t>(),
                                                          rowcnt.as<int32_t>());
  MM_TRY(scan_exclusive_i32(rowcnt.as<int32_t>(), sp_tmp.as<int32_t>(), n, ws2.p, s));
  MM_CK(cudaMemsetAsync(rowcnt.p, 0, sizeof(int32_t) * (size_t)(n + 1), s));
  khop2_reduce<<<ceil_div(std::max(m, 1), 256), 256, 0, s>>>(
      m, vb, keys, dbits, head.as<int32_t>(), pos.as<int32_t>(), S_tmp.as<SEnt>(),
      rowcnt.as<int32_t>());
  MM_TRY(scan_exclusive_i32(rowcnt.as<int32_t>(), sp, n, ws2.p, s));
  int32_t nnzS = 0;
  MM_TRY(read_scalar(sp + n, &nnzS, s));
  MM_CK(cudaStreamSynchronize(s));
  MM_CK(cudaMallocAsync(&S, sizeof(SEnt) * (size_t)std::max(nnzS, 1), s));
  *s_out = S;
  khop2_finish<<<ceil_div(n, 256), 256, 0, s>>>(n, sp_tmp.as<int32_t>(), S_tmp.as<SEnt>(), sp, S,
                                                rho);
  MM_CK(cudaGetLastError());
  MM_CK(cudaStreamSynchronize(s));
  *nnz_out = nnzS;
  return MM_OK;
}

mm_status cluster_lp(int n, const int32_t* rp, const int32_t* col, const float* omega,
                     const float* c, float U, int rounds, uint64_t seed, int level,
                     int32_t* labels, cudaStream_t s) {
  if (n <= 0) return MM_OK;
  const uint32_t key0 = (uint32_t)(seed & 0xffffffffu), key1 = (uint32_t)(seed >> 32);
  int32_t maxdeg = 0;
  {
    Tmp md;
    MM_TRY(tmp_alloc(md, sizeof(int32_t), s));
    MM_CK(cudaMemsetAsync(md.p, 0, sizeof(int32_t), s));
    max_row_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, rp, md.as<int32_t>());
    MM_TRY(read_scalar(md.p, &maxdeg, s));
    MM_CK(cudaStreamSynchronize(s));
  }
  // the single-CTA path holds every row's clusters in a 512-slot hash
  if (n <= kLPSmallN && maxdeg <= kLPSmallHash / 2) {
    static_assert(sizeof(LPSmem) <= 227 * 1024, "LP kernel exceeds shared memory");
    MM_CK(cudaFuncSetAttribute(lp_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sizeof(LPSmem)));
    lp_small_kernel<<<1, kLPSmallT, sizeof(LPSmem), s>>>(n, rp, col, omega, c, U, rounds, key0,
                                                         key1, (uint32_t)level, labels);
    MM_CK(cudaGetLastError());
    MM_CK(cudaStreamSynchronize(s));
    return MM_OK;
  }
  Tmp W, k0, k1, v0, v1, mv;
  MM_TRY(tmp_alloc(mv, sizeof(int), s));
  MM_TRY(tmp_alloc(W, sizeof(float) * (size_t)n, s));
  MM_TRY(tmp_alloc(k0, sizeof(uint64_t) * (size_t)n, s));
  MM_TRY(tmp_alloc(k1, sizeof(uint64_t) * (size_t)n, s));
  MM_TRY(tmp_alloc(v0, sizeof(int32_t) * (size_t)n, s));
  MM_TRY(tmp_alloc(v1, sizeof(int32_t) * (size_t)n, s));
  TmpSort sws;
  MM_TRY(tmp_sort(sws, n, s));
  // vertices with more than kLPHeavyDeg neighbours: ordered list, hash
  // offsets (2 deg rounded up to a power of two each) and scratch
  Tmp hflag, hpos, hws, hl, hsz, hoff, hkey, hval;
  int32_t nh = 0;
  if (maxdeg > kLPHeavyDeg) {
    MM_TRY(tmp_alloc(hflag, sizeof(int32_t) * (size_t)n, s));
    MM_TRY(tmp_alloc(hpos, sizeof(int32_t) * ((size_t)n + 1), s));
    MM_TRY(tmp_alloc(hws, scan_ws_bytes(n), s));
    MM_TRY(tmp_alloc(hl, sizeof(int32_t) * (size_t)n, s));
    Tmp dummy;
    MM_TRY(tmp_alloc(dummy, sizeof(int32_t), s));
    heavy_flags_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, rp, kLPHeavyDeg, hflag.as<int32_t>(),
                                                        dummy.as<int32_t>());
    MM_TRY(scan_exclusive_i32(hflag.as<int32_t>(), hpos.as<int32_t>(), n, hws.p, s));
    heavy_list_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, hflag.as<int32_t>(),
                                                       hpos.as<int32_t>(), hl.as<int32_t>());
    MM_TRY(read_scalar(hpos.as<int32_t>() + n, &nh, s));
    MM_CK(cudaStreamSynchronize(s));
  }
  if (nh > 0) {
    MM_TRY(tmp_alloc(hsz, sizeof(int32_t) * (size_t)nh, s));
    MM_TRY(tmp_alloc(hoff, sizeof(int64_t) * ((size_t)nh + 1), s));
    Tmp sws2;
    MM_TRY(tmp_alloc(sws2, scan_ws_bytes(nh), s));
    lp_heavy_sizes<<<ceil_div(nh, 256), 256, 0, s>>>(nh, hl.as<int32_t>(), rp, hsz.as<int32_t>());
    MM_TRY(scan_exclusive_i64(hsz.as<int32_t>(), hoff.as<int64_t>(), nh, sws2.p, s));
    int64_t total = 0;
    MM_TRY(read_scalar(hoff.as<int64_t>() + nh, &total, s));
    MM_CK(cudaStreamSynchronize(s));
    MM_TRY(tmp_alloc(hkey, sizeof(int32_t) * (size_t)std::max<int64_t>(total, 1), s));
    MM_TRY(tmp_alloc(hval, sizeof(float) * (size_t)std::max<int64_t>(total, 1), s));
  }
  lp_init<<<ceil_div(n, 256), 256, 0, s>>>(n, c, labels, W.as<float>());
  const int tb = bits_for(n) + 1;
  mm_status st = MM_OK;
  for (int r = 0; r < rounds && st == MM_OK; ++r) {
    MM_CK(cudaMemsetAsync(mv.p, 0, sizeof(int), s));
    for (uint32_t half = 0; half < 2 && st == MM_OK; ++half) {
      lp_propose<<<ceil_div(n, kLPWarps), kLPWarps * 32, 0, s>>>(
          n, rp, col, omega, c, W.as<float>(), labels, U, key0, key1, (uint32_t)r,
          (uint32_t)level, half, tb, k0.as<uint64_t>(), v0.as<int32_t>());
      if (nh > 0)
        lp_propose_heavy<<<nh, kLPHeavyT, 0, s>>>(
            hl.as<int32_t>(), hoff.as<int64_t>(), rp, col, omega, c, W.as<float>(), labels, U,
            key0, key1, (uint32_t)r, (uint32_t)level, half, hkey.as<int32_t>(),
            hval.as<float>(), k0.as<uint64_t>());
      uint64_t* keys;
      int32_t* vals;
      st = radix_sort_u64(k0.as<uint64_t>(), k1.as<uint64_t>(), v0.as<int32_t>(), v1.as<int32_t>(),
                          n, 0, 8 + tb, sws.ws, s, &keys, &vals);
      if (st != MM_OK) break;
      // keys equal to all ones sort last only if every bit is compared: the
      // sort above covers bits [0, 8 + tb) and targets are < 2^(tb-1)
      lp_admit<<<ceil_div(n, 256), 256, 0, s>>>(n, keys, vals, c, W.as<float>(), U, labels,
                                                 mv.as<int>());
      cudaMemsetAsync(W.p, 0, sizeof(float) * (size_t)n, s);
      lp_weights<<<ceil_div(n, 256), 256, 0, s>>>(n, c, labels, W.as<float>());
    }
    // a round without moves leaves a fixed point: every later round would
    // make the same (no) choices
    int moved = 0;
    MM_TRY(read_scalar(mv.p, &moved, s));
    MM_CK(cudaStreamSynchronize(s));
    if (moved == 0) break;
  }
  if (st != MM_OK) return st;
  MM_CK(cudaGetLastError());
  MM_CK(cudaStreamSynchronize(s));
  return MM_OK;
}

mm_status contract(int n, const int32_t* rp, const int32_t* col, const float* omega,
                   const float* c, const int32_t* labels, int32_t* map, Level& out,
                   cudaStream_t s) {
  int32_t nnz = 0;
  MM_TRY(read_scalar(rp + n, &nnz, s));
  MM_CK(cudaStreamSynchronize(s));
  Tmp used, rank, ws, flag, pos, k0, k1, v0, v1, head, hpos, rowcnt;
  MM_TRY(tmp_alloc(used, sizeof(int32_t) * (size_t)(n + 1), s));
  MM_TRY(tmp_alloc(rank, sizeof(int32_t) * (size_t)(n + 1), s));
  MM_TRY(tmp_alloc(ws, scan_ws_bytes(std::max(std::max(n, nnz), 1)) + 64, s));
  MM_CK(cudaMemsetAsync(used.p, 0, sizeof(int32_t) * (size_t)(n + 1), s));
  mark_used<<<ceil_div(n, 256), 256, 0, s>>>(n, labels, used.as<int32_t>());
  MM_TRY(scan_exclusive_i32(used.as<int32_t>(), rank.as<int32_t>(), n, ws.p, s));
  int32_t nc = 0;
  MM_TRY(read_scalar(rank.as<int32_t>() + n, &nc, s));
  MM_CK(cudaStreamSynchronize(s));
  out.n = nc;
  MM_CK(cudaMallocAsync(&out.c, sizeof(float) * (size_t)std::max(nc, 1), s));
  MM_CK(cudaMemsetAsync(out.c, 0, sizeof(float) * (size_t)std::max(nc, 1), s));
  apply_map<<<ceil_div(n, 256), 256, 0, s>>>(n, labels, rank.as<int32_t>(), c, map, out.c);
  MM_TRY(tmp_alloc(flag, sizeof(int32_t) * (size_t)std::max(nnz, 1), s));
  MM_TRY(tmp_alloc(pos, sizeof(int32_t) * (size_t)(nnz + 1), s));
  cut_flags<<<ceil_div(n, 256), 256, 0, s>>>(n, rp, col, map, flag.as<int32_t>());
  MM_TRY(scan_exclusive_i32(flag.as<int32_t>(), pos.as<int32_t>(), nnz, ws.p, s));
  int32_t m = 0;
  MM_TRY(read_scalar(pos.as<int32_t>() + nnz, &m, s));
  MM_CK(cudaStreamSynchronize(s));
  const int cb = bits_for(std::max(nc - 1, 1));
  MM_TRY(tmp_alloc(k0, sizeof(uint64_t) * (size_t)std::max(m, 1), s));
  MM_TRY(tmp_alloc(k1, sizeof(uint64_t) * (size_t)std::max(m, 1), s));
  MM_TRY(tmp_alloc(v0, sizeof(int32_t) * (size_t)std::max(m, 1), s));
  MM_TRY(tmp_alloc(v1, sizeof(int32_t) * (size_t)std::max(m, 1), s));
  cut_emit<<<ceil_div(n, 256), 256, 0, s>>>(n, cb, rp, col, map, pos.as<int32_t>(),
                                            k0.as<uint64_t>(), v0.as<int32_t>());
  TmpSort sws;
  MM_TRY(tmp_sort(sws, std::max(m, 1), s));
  uint64_t* keys;
  int32_t* vals;
  MM_TRY(radix_sort_u64(k0.as<uint64_t>(), k1.as<uint64_t>(), v0.as<int32_t>(),
                        v1.as<int32_t>(), m, 0, 2 * cb, sws.ws, s, &keys, &vals));
  MM_TRY(tmp_alloc(head, sizeof(int32_t) * (size_t)std::max(m, 1), s));
  MM_TRY(tmp_alloc(hpos, sizeof(int32_t) * (size_t)(m + 1), s));
  run_heads<<<ceil_div(std::max(m, 1), 256), 256, 0, s>>>(m, keys, head.as<int32_t>());
  MM_TRY(scan_exclusive_i32(head.as<int32_t>(), hpos.as<int32_t>(), m, ws.p, s));
  int32_t cnnz = 0;
  MM_TRY(read_scalar(hpos.as<int32_t>() + m, &cnnz, s));
  MM_CK(cudaStreamSynchronize(s));
  out.nnzE = cnnz;
  MM_CK(cudaMallocAsync(&out.col, sizeof(int32_t) * (size_t)std::max(cnnz, 1), s));
  MM_CK(cudaMallocAsync(&out.omega, sizeof(float) * (size_t)std::max(cnnz, 1), s));
  MM_CK(cudaMallocAsync(&out.rp, sizeof(int32_t) * (size_t)(nc + 1), s));
  MM_TRY(tmp_alloc(rowcnt, sizeof(int32_t) * (size_t)(nc + 1), s));
  MM_CK(cudaMemsetAsync(rowcnt.p, 0, sizeof(int32_t) * (size_t)(nc + 1), s));
  coarse_reduce<<<ceil_div(std::max(m, 1), 256), 256, 0, s>>>(
      m, cb, keys, vals, omega, head.as<int32_t>(), hpos.as<int32_t>(), out.col, out.omega,
      rowcnt.as<int32_t>());
  MM_TRY(scan_exclusive_i32(rowcnt.as<int32_t>(), out.rp, nc, ws.p, s));
  MM_CK(cudaGetLastError());
  MM_CK(cudaStreamSynchronize(s));
  return MM_OK;
}

mm_status gather_config(Level& L, const mm_params& p, cudaStream_t s) {
  const double avg = L.n > 0 ? (double)L.nnzS / L.n : 0.0;
  int lanes = p.gather_lanes;
  if (lanes <= 0) {
    // enough lanes to fill the GPU (SMs x 2048 threads) when n is small,
    // never more than the mean row length
    lanes = 1;
    const int64_t want = (int64_t)num_sms() * 2048 / std::max(L.n, 1);
    while (lanes < 32 && 2 * lanes <= want && lanes < avg) lanes <<= 1;
  }
  if (lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32) {
    set_error("gather_lanes must be a power of two <= 32 (got %d)", lanes);
    return MM_ERR_INVALID_ARG;
  }
  L.lanes = lanes;
  if (p.traverse_warps > 0) {
    L.walk_warps = p.traverse_warps;
  } else if (p.bh_group) {
    // warps sharing one task: about 24 warps per SM in all (measured: more
    // helpers per task only add seed overhead once the SMs are full)
    const int64_t tasks = std::max<int64_t>(1, (L.n + 31) / 32);
    int w = 1;
    while (w < 16 && (int64_t)w * tasks < (int64_t)24 * num_sms()) w <<= 1;
    L.walk_warps = w;
  } else {
    L.walk_warps = L.n >= 20000 ? 16 : 8;  // per-point walk: warps per block
  }
  L.heavy_degree = p.heavy_degree > 0 ? p.heavy_degree : std::max(512, 32 * lanes);
  // heavy rows in ascending order (a deterministic processing order):
  // flags, exclusive scan (the total lands in pos[n]), ordered scatter
  const int n = std::max(L.n, 1);
  Tmp flag, pos, ws, mx;
  MM_TRY(tmp_alloc(flag, sizeof(int32_t) * (size_t)n, s));
  MM_TRY(tmp_alloc(pos, sizeof(int32_t) * ((size_t)n + 1), s));
  MM_TRY(tmp_alloc(ws, scan_ws_bytes(n), s));
  MM_TRY(tmp_alloc(mx, sizeof(int32_t), s));
  MM_CK(cudaMemsetAsync(mx.p, 0, sizeof(int32_t), s));
  MM_CK(cudaMallocAsync(&L.heavy, sizeof(int32_t) * (size_t)n, s));
  int32_t h[2] = {0, 0};
  if (L.n > 0) {
    heavy_flags_kernel<<<ceil_div(L.n, 256), 256, 0, s>>>(L.n, L.sp, L.heavy_degree,
                                                          flag.as<int32_t>(), mx.as<int32_t>());
    MM_TRY(scan_exclusive_i32(flag.as<int32_t>(), pos.as<int32_t>(), L.n, ws.p, s));
    heavy_list_kernel<<<ceil_div(L.n, 256), 256, 0, s>>>(L.n, flag.as<int32_t>(),
                                                         pos.as<int32_t>(), L.heavy);
    MM_CK(cudaGetLastError());
    MM_TRY(read_scalar(pos.as<int32_t>() + L.n, &h[0], s));
    MM_TRY(read_scalar(mx.p, &h[1], s));
  }
  MM_CK(cudaStreamSynchronize(s));
  L.n_heavy = h[0];
  L.max_deg = h[1];
  // the sums over S on a parallel branch of the sweep pay off where they
  // are a large part of it (hubs, long rows); otherwise the extra update
  // launch costs what the overlap saves (measured: R-MAT 2^20 -20 %,
  // Delaunay 2^20 and the 100k RGG unchanged)
  L.split_gather = L.n_heavy > 0 || avg >= 24.0;
  return MM_OK;
}

}  // namespace mm
