// mm_repulsion_noalloc: the Barnes-Hut long-range sum with every byte of its
// scratch in one fixed, file-scope device array, so the call itself never
// allocates.
//
// Who needs it: callers that must not call cudaMalloc/cudaFree on their hot
// path -- code running under a custom or pool allocator that forbids other
// allocations, real-time loops that cannot afford the implicit device
// synchronisation cudaFree brings, and hosts that hand the library a fixed
// device-memory budget up front.  They pass their own input and output
// buffers; the tree workspace (sort buffers, radix tree, node records) comes
// from the static array below.
//
// Cost of the array: kScratchBytes of device memory on every GPU that loads
// this library, held until the process exits.
//
// Set-up: the first call on a device, with that device current, resolves the
// array's device address with cudaGetSymbolAddress (a host-side name of a
// __device__ array is only a host stand-in, not a usable device pointer).
// Make that first call before any stream capture.
//
// Every call synchronises the stream before it returns (it reads the walk's
// error flag back to the host).
//
// Sharing: every call uses the same array and it keeps the previous call's
// contents; the walk's error flag is cleared at the start of each call.
// The sort's look-back status words rely on the zero fill at module load:
// they are tagged with a build epoch that starts at 0 and that every call
// advances, so no word left by an earlier call (or the initial zeros) can be
// taken for one of the current call.  Node records of an earlier, larger
// call stay in the array; the walk never reads past the current call's
// 2n - 1 records.
// Calls whose GPU work overlaps (different streams, different host threads)
// race on the array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "mm_internal.cuh"

namespace mm {

namespace {

constexpr int kNoAllocMaxN = 32768;   // largest point set accepted
constexpr size_t kAlign = 256;

constexpr size_t up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

// Byte offsets of the workspace pieces inside the array.
struct Carve {
  size_t keys0, keys1, vals0, vals1, xs, lo, hi, left, right, delta, owner, parent, incl,
      tile_sum, status, hist, counters, walk_next, node, partials, root, ticket, err, zero,
      total;
};

constexpr Carve carve() {
  constexpr size_t N = kNoAllocMaxN;
  constexpr size_t tiles = (N + kSortMinTile - 1) / kSortMinTile;
  Carve c{};
  size_t o = 0;
  c.keys0 = o; o += up(4 * N);
  c.keys1 = o; o += up(4 * N);
  c.vals0 = o; o += up(4 * N);
  c.vals1 = o; o += up(4 * N);
  c.xs = o; o += up(8 * N);
  c.lo = o; o += up(4 * N);
  c.hi = o; o += up(4 * N);
  c.left = o; o += up(4 * N);
  c.right = o; o += up(4 * N);
  c.delta = o; o += up(4 * N);
  c.owner = o; o += up(4 * N);
  c.parent = o; o += up(4 * 2 * N);
  c.incl = o; o += up(16 * N);
  c.tile_sum = o; o += up(16 * tiles);
  c.status = o; o += up(8 * 4 * tiles * 256);
  c.hist = o; o += up(4 * 4 * 256);
  c.counters = o; o += up(4 * 4);
  c.walk_next = o; o += up(4);
  c.node = o; o += up(32 * 2 * N);
  c.partials = o; o += up(16 * 2 * kMaxSMs);
  c.root = o; o += up(16);
  c.ticket = o; o += up(8);
  c.err = o; o += up(4);
  c.zero = o; o += up(4);
  c.total = o;
  return c;
}

constexpr Carve kCarve = carve();
constexpr size_t kScratchBytes = kCarve.total;
static_assert(kScratchBytes < (8u << 20), "no-allocation scratch stays under 8 MiB");
static_assert(kCarve.node % alignof(NodeRec) == 0, "cell records are read with 256-bit loads");

// The scratch array (zero at module load).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[64] = {nullptr};

// Device address of g_scratch for the current device (resolved once).
mm_status scratch_address(void** out) {
  int dev = 0;
  MM_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range", dev);
    return MM_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      set_error("cudaGetSymbolAddress of the no-allocation scratch failed: %s",
                cudaGetErrorString(e));
      return MM_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return MM_OK;
}

}  // namespace

}  // namespace mm

using namespace mm;

extern "C" mm_status mm_repulsion_noalloc(int32_t n, const float* x, float theta, float* F_out,
                                          void* stream) {
  if (n < 1 || !x || !F_out || !(theta >= 0.f)) {
    set_error("mm_repulsion_noalloc: need n >= 1, device x and F_out, theta >= 0");
    return MM_ERR_INVALID_ARG;
  }
  if (n > kNoAllocMaxN) {
    set_error("mm_repulsion_noalloc: n = %d exceeds the fixed scratch limit of %d points", n,
              kNoAllocMaxN);
    return MM_ERR_INVALID_ARG;
  }
  // x and F_out must be device memory of the current device: that is the
  // device whose copy of the array is resolved below and used by the kernels
  int dev = 0;
  MM_CK(cudaGetDevice(&dev));
  const void* ptrs[2] = {x, F_out};
  for (const void* q : ptrs) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, q) != cudaSuccess ||
        (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) ||
        at.device != dev) {
      cudaGetLastError();
      set_error("mm_repulsion_noalloc: x and F_out must be device memory of the current "
                "device (%d)", dev);
      return MM_ERR_INVALID_ARG;
    }
  }
  void* base = nullptr;
  MM_TRY(scratch_address(&base));
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* b = (unsigned char*)base;
  const Carve& c = kCarve;
  TreeWS ws;
  ws.cap = kNoAllocMaxN;
  ws.keys[0] = (uint32_t*)(b + c.keys0);
  ws.keys[1] = (uint32_t*)(b + c.keys1);
  ws.vals[0] = (int32_t*)(b + c.vals0);
  ws.vals[1] = (int32_t*)(b + c.vals1);
  ws.xs = (float2*)(b + c.xs);
  ws.lo = (int32_t*)(b + c.lo);
  ws.hi = (int32_t*)(b + c.hi);
  ws.left = (int32_t*)(b + c.left);
  ws.right = (int32_t*)(b + c.right);
  ws.delta = (int32_t*)(b + c.delta);
  ws.owner = (int32_t*)(b + c.owner);
  ws.parent = (int32_t*)(b + c.parent);
  ws.incl = (ulonglong2*)(b + c.incl);
  ws.tile_sum = (ulonglong2*)(b + c.tile_sum);
  ws.status = (unsigned long long*)(b + c.status);
  ws.hist = (uint32_t*)(b + c.hist);
  ws.counters = (uint32_t*)(b + c.counters);
  ws.walk_next = (unsigned*)(b + c.walk_next);
  ws.node = (NodeRec*)(b + c.node);
  ws.partials = (float4*)(b + c.partials);
  ws.root = (float4*)(b + c.root);
  ws.ticket = (uint32_t*)(b + c.ticket);
  ws.err = (int*)(b + c.err);
  // the error flag and the bounding-box ticket must start at zero; the
  // build epoch (ticket[1]) must persist, since the sort's look-back status
  // words are tagged with it
  MM_CK(cudaMemsetAsync(ws.err, 0, sizeof(int), s));
  MM_CK(cudaMemsetAsync(ws.ticket, 0, sizeof(uint32_t), s));
  XSel xs{(const float2*)x, (const float2*)x, (const int32_t*)(b + c.zero)};
  // the library's default walk (leaf buckets, group acceptance), as
  // mm_repulsion on a hierarchy built with mm_default_params
  mm_params d;
  mm_default_params(&d);
  MM_TRY(walk_setup(ws));
  MM_TRY(bh_build(xs, n, theta, leaf_of(d), ws, s, nullptr, true, group_of(d)));
  MM_TRY(bh_traverse(n, ws, (float2*)F_out, 0, nullptr, s, group_of(d)));
  int err = 0;
  MM_CK(cudaMemcpyAsync(&err, ws.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  MM_CK(cudaStreamSynchronize(s));
  if (err & 2) {
    set_error("a bounded device wait gave up (the sort's look-back)");
    return MM_ERR_TIMEOUT;
  }
  if (err) {
    set_error("internal error: Barnes-Hut walk met an inconsistent tree");
    return MM_ERR_CUDA;
  }
  return MM_OK;
}
