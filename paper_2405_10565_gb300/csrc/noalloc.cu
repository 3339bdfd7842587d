// Morton clustering of strand roots that allocates no device memory.
//
// Some callers cannot let a library allocate: a host application that owns
// every device allocation under a fixed memory budget (a game engine's frame
// loop, a host framework whose own allocator must see all memory), or a
// real-time loop where cudaMalloc / cudaFree are off limits because they
// synchronise the device.  For them this entry point runs the root-bounds,
// Morton-code and cluster kernels of hr_build_clusters with all of its scratch
// in one file-scope device array of fixed size, and writes only the caller's
// output buffers.  Its stable radix sort is the four-kernel-per-digit sort
// (digit histogram per 2,048-key tile, scan, scatter), not the single-sweep
// sort of hr_build_clusters, because its scratch has a fixed size; both sorts
// are stable, so the order and cluster ids are the same.
//
// The array's name is meaningful to device code only; on the host it is a
// stand-in, so host code takes its device address with cudaGetSymbolAddress
// once per device (with that device current) and passes that address on.
#include <mutex>

#include "common.cuh"

namespace hr {
namespace {

constexpr uint32_t kMaxN = HR_NOALLOC_MAX_STRANDS;
constexpr uint32_t kAlignWords = 64;  // 256 bytes
constexpr uint32_t round_up(uint32_t x) { return (x + kAlignWords - 1) / kAlignWords * kAlignWords; }
constexpr uint32_t kSortTileKeys = 2048;                      // keys per sort block
constexpr uint32_t kMaxCounts = (kMaxN + kSortTileKeys - 1) / kSortTileKeys * 256;
constexpr uint32_t kOffBounds = 0;
constexpr uint32_t kOffKeys = kOffBounds + kAlignWords;
constexpr uint32_t kOffKeysTmp = kOffKeys + round_up(kMaxN);
constexpr uint32_t kOffValsTmp = kOffKeysTmp + round_up(kMaxN);
constexpr uint32_t kOffCounts = kOffValsTmp + round_up(kMaxN);
constexpr uint32_t kOffSums = kOffCounts + round_up(kMaxCounts);
constexpr uint32_t kWords = kOffSums + round_up(1024);

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t* g_dev_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set up on the
// first call on each device).
cudaError_t scratch_address(uint32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_dev_ptr[dev];
  return cudaSuccess;
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace hr

extern "C" hr_status hr_morton_clusters_noalloc(const float* vertices, uint32_t n_strands,
                                                uint32_t n_segments, uint32_t n_clusters,
                                                uint32_t* order_out, uint32_t* cluster_of_out,
                                                void* cuda_stream) {
  using namespace hr;
  if (!vertices || !order_out || !cluster_of_out) return HR_EINVAL;
  if (n_strands < 1 || n_strands > kMaxN) return HR_EINVAL;
  if (n_segments < 1 || n_segments > 4096) return HR_EINVAL;
  if (n_clusters < 1 || n_clusters > n_strands) return HR_EINVAL;
  if (!on_device(vertices) || !on_device(order_out) || !on_device(cluster_of_out)) return HR_EINVAL;
  uint32_t* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) {
    cudaGetLastError();
    return HR_ECUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // every word read below is written first in this call (bounds are reset,
  // keys and counts fully rewritten), so no clearing pass is needed
  const cudaError_t e = morton_clusters_with(
      reinterpret_cast<const float4*>(vertices), n_strands, n_segments, n_clusters, order_out,
      cluster_of_out, base + kOffBounds, base + kOffKeys, base + kOffKeysTmp, base + kOffValsTmp,
      base + kOffCounts, base + kOffSums, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HR_ECUDA;
  }
  return HR_OK;
}
