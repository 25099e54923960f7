// Hierarchy order of the vertices of every level (a data-layout step; the
// paper has no counterpart).
//
// The Eq. 2 gather reads, for every vertex u, the positions of the vertices
// of S_u.  In the input numbering of a large graph those are scattered over
// the whole position array, and every 8-byte read touches its own 32-byte
// sector.  After coarsening, each level is renumbered so that the vertices
// of one cluster are consecutive and the clusters follow the order of the
// coarser level: the coarsest level keeps its numbering, and level l is
// sorted stably by the new index of its coarse vertex (ties by old index).
// Neighbours in the graph then mostly share clusters, so the positions a
// warp's S rows read lie in a few sectors, and the sorted points of the tree
// build and the walk's force scatter follow the same order.
//
// Per level the CSR rows, their columns, the edge weights omega, the input
// edge lengths (level 0), the node weights c and the map to the next level
// are rewritten; everything derived from them (pair sets S, gather
// configuration, Eq. 3 groups) is built afterwards.  The level-0
// permutation is kept: positions at level 0 cross the C-ABI in the caller's
// numbering and are mapped on the way in and out.
#include <cuda_runtime.h>

#include <algorithm>

#include "mm_internal.cuh"

namespace mm {

namespace {

__global__ void order_keys(int n, const int32_t* __restrict__ map,
                           const int32_t* __restrict__ pi_next, uint32_t* __restrict__ key,
                           int32_t* __restrict__ val) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int32_t p = map[v];
  key[v] = (uint32_t)(pi_next ? pi_next[p] : p);
  val[v] = v;
}

__global__ void invert_perm(int n, const int32_t* __restrict__ sigma, int32_t* __restrict__ pi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) pi[sigma[i]] = i;
}

__global__ void row_degrees(int n, const int32_t* __restrict__ rp,
                            const int32_t* __restrict__ sigma, int32_t* __restrict__ deg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) deg[i] = rp[sigma[i] + 1] - rp[sigma[i]];
}

// New row i is old row sigma[i] with its columns relabelled by pi; one warp
// per row.
__global__ void permute_csr(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const float* __restrict__ om, const float* __restrict__ el,
                            const int32_t* __restrict__ sigma, const int32_t* __restrict__ pi,
                            const int32_t* __restrict__ nrp, int32_t* __restrict__ ncol,
                            float* __restrict__ nom, float* __restrict__ nel) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const int i = (int)w;
  const int o = sigma[i];
  const int a = rp[o], b = rp[o + 1], d = nrp[i];
  for (int e = a + lane; e < b; e += 32) {
    ncol[d + (e - a)] = pi[col[e]];
    nom[d + (e - a)] = om[e];
    if (el) nel[d + (e - a)] = el[e];
  }
}

__global__ void gather_f32(int n, const int32_t* __restrict__ idx, const float* __restrict__ in,
                           float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[idx[i]];
}

__global__ void permute_map(int n, const int32_t* __restrict__ map,
                            const int32_t* __restrict__ sigma, const int32_t* __restrict__ pi_next,
                            int32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t p = map[sigma[i]];
  out[i] = pi_next ? pi_next[p] : p;
}

__global__ void gather_f2(int n, const int32_t* __restrict__ idx, const float2* __restrict__ in,
                          float2* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[idx[i]];
}

int bits_of(int64_t v) {  // bits needed to hold values in [0, v]
  int b = 1;
  while (b < 31 && ((int64_t)1 << b) <= v) ++b;
  return b;
}

}  // namespace

mm_status permute_positions(int n, const int32_t* idx, const float2* in, float2* out,
                            cudaStream_t s) {
  if (n <= 0) return MM_OK;
  gather_f2<<<ceil_div(n, 256), 256, 0, s>>>(n, idx, in, out);
  MM_CK(cudaGetLastError());
  return MM_OK;
}

mm_status renumber_levels(std::vector<Level>& levels, LevelOrder& ord, cudaStream_t s) {
  const int L = (int)levels.size();
  if (L < 2) return MM_OK;  // a single level keeps the input numbering
  int nmax = 1;
  for (const Level& V : levels) nmax = std::max(nmax, V.n);
  SortWS ws;
  MM_TRY(sort_ws_alloc(ws, nmax));
  uint32_t *k0 = nullptr, *k1 = nullptr;
  int32_t *v0 = nullptr, *v1 = nullptr, *deg = nullptr;
  void* scan_ws = nullptr;
  mm_status st = MM_OK;
  auto ck = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == MM_OK) st = cuda_status(e, what, __FILE__, __LINE__);
  };
  ck(cudaMallocAsync(&k0, sizeof(uint32_t) * nmax, s), "alloc");
  ck(cudaMallocAsync(&k1, sizeof(uint32_t) * nmax, s), "alloc");
  ck(cudaMallocAsync(&v0, sizeof(int32_t) * nmax, s), "alloc");
  ck(cudaMallocAsync(&v1, sizeof(int32_t) * nmax, s), "alloc");
  ck(cudaMallocAsync(&deg, sizeof(int32_t) * nmax, s), "alloc");
  ck(cudaMallocAsync(&scan_ws, scan_ws_bytes(nmax), s), "alloc");
  int32_t* pi_next = nullptr;  // new index of each vertex of level l + 1
  for (int l = L - 2; l >= 0 && st == MM_OK; --l) {
    Level& V = levels[l];
    const int n = V.n, nn = levels[l + 1].n;
    const int64_t m = V.nnzE;
    // sigma: old vertex at new index i (stable sort by the coarse vertex's
    // new index); pi: its inverse
    order_keys<<<ceil_div(n, 256), 256, 0, s>>>(n, V.map, pi_next, k0, v0);
    uint32_t* ko = nullptr;
    int32_t* sigma = nullptr;
    st = radix_sort_u32(k0, k1, v0, v1, n, 0, bits_of(std::max(nn - 1, 1)), ws, s, &ko, &sigma);
    if (st != MM_OK) break;
    int32_t *pi = nullptr, *sig = nullptr, *nrp = nullptr, *ncol = nullptr, *nmap = nullptr;
    float *nom = nullptr, *nel = nullptr, *nc = nullptr;
    ck(cudaMallocAsync(&pi, sizeof(int32_t) * n, s), "alloc");
    ck(cudaMallocAsync(&sig, sizeof(int32_t) * n, s), "alloc");
    ck(cudaMallocAsync(&nrp, sizeof(int32_t) * (size_t)(n + 1), s), "alloc");
    ck(cudaMallocAsync(&ncol, sizeof(int32_t) * (size_t)std::max<int64_t>(m, 1), s), "alloc");
    ck(cudaMallocAsync(&nom, sizeof(float) * (size_t)std::max<int64_t>(m, 1), s), "alloc");
    if (V.elen) ck(cudaMallocAsync(&nel, sizeof(float) * (size_t)std::max<int64_t>(m, 1), s),
                   "alloc");
    ck(cudaMallocAsync(&nc, sizeof(float) * n, s), "alloc");
    ck(cudaMallocAsync(&nmap, sizeof(int32_t) * n, s), "alloc");
    if (st != MM_OK) break;
    ck(cudaMemcpyAsync(sig, sigma, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s), "copy");
    invert_perm<<<ceil_div(n, 256), 256, 0, s>>>(n, sig, pi);
    row_degrees<<<ceil_div(n, 256), 256, 0, s>>>(n, V.rp, sig, deg);
    st = scan_exclusive_i32(deg, nrp, n, scan_ws, s);
    if (st != MM_OK) break;
    permute_csr<<<ceil_div((int64_t)n * 32, 256), 256, 0, s>>>(n, V.rp, V.col, V.omega, V.elen,
                                                               sig, pi, nrp, ncol, nom, nel);
    gather_f32<<<ceil_div(n, 256), 256, 0, s>>>(n, sig, V.c, nc);
    permute_map<<<ceil_div(n, 256), 256, 0, s>>>(n, V.map, sig, pi_next, nmap);
    ck(cudaGetLastError(), "renumber kernels");
    if (l == 0) {
      // level 0 keeps the caller's CSR for export; positions are mapped
      ord.rp_user = V.rp;
      ord.col_user = V.col;
      ord.omega_user = V.omega;
      ord.elen_user = V.elen;
      ord.perm0 = pi;
      ord.inv0 = sig;
    } else {
      cudaFreeAsync(V.rp, s);
      cudaFreeAsync(V.col, s);
      cudaFreeAsync(V.omega, s);
      if (V.elen) cudaFreeAsync(V.elen, s);
      cudaFreeAsync(sig, s);
    }
    cudaFreeAsync(V.c, s);
    cudaFreeAsync(V.map, s);
    V.rp = nrp;
    V.col = ncol;
    V.omega = nom;
    V.elen = nel;
    V.c = nc;
    V.map = nmap;
    if (pi_next) cudaFreeAsync(pi_next, s);
    pi_next = l == 0 ? nullptr : pi;
  }
  if (pi_next) cudaFreeAsync(pi_next, s);
  cudaFreeAsync(k0, s);
  cudaFreeAsync(k1, s);
  cudaFreeAsync(v0, s);
  cudaFreeAsync(v1, s);
  cudaFreeAsync(deg, s);
  cudaFreeAsync(scan_ws, s);
  ck(cudaStreamSynchronize(s), "renumber");
  sort_ws_free(ws);
  return st;
}

}  // namespace mm
