// Device-wide exclusive scan and stable LSD radix sort of (uint32 key, uint32
// value) pairs.  Used by the Morton clustering of strands and by the linear
// BVH build.
#include "common.cuh"

namespace hr {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;  // 1024 values per block

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total
// through *total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = warp_incl_scan(v);
  if (lane == 31) warp_sums[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
    s = warp_incl_scan(s);
    if (lane < kScanThreads / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  uint32_t off = wid ? warp_sums[wid - 1] : 0;
  *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return off + inc - v;
}

__global__ void k_scan_tiles(uint32_t* data, uint32_t n, uint32_t* block_sums) {
  const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? data[base + i] : 0u;
    s += v[i];
  }
  uint32_t total;
  uint32_t off = block_excl_scan(s, &total);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) data[base + i] = off;
    off += v[i];
  }
  if (threadIdx.x == 0 && block_sums) block_sums[blockIdx.x] = total;
}

__global__ void k_scan_add(uint32_t* data, uint32_t n, const uint32_t* block_offs) {
  const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  const uint32_t add = block_offs[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) data[base + i] += add;
}

// ------------------------------------------------------------- radix sort

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;  // keys per thread
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048 keys per block
constexpr int kRadix = 256;

// Per-block digit histogram; counts laid out digit-major: counts[d * B + b].
__global__ void k_digit_hist(const uint32_t* __restrict__ keys, uint32_t n, int shift,
                             uint32_t* __restrict__ counts, uint32_t nblocks) {
  __shared__ uint32_t h[kRadix];
  for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const uint32_t base = blockIdx.x * kSortTile;
  for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
    uint32_t p = base + i;
    if (p < n) atomicAdd(&h[(keys[p] >> shift) & 0xffu], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) counts[d * nblocks + blockIdx.x] = h[d];
}

// Stable scatter: each warp ranks its 256 contiguous keys in order with
// __match_any_sync, warps are combined by a per-digit prefix in shared
// memory, and the block's global digit offsets come from the scanned
// histogram.
__global__ void __launch_bounds__(kSortThreads)
    k_digit_scatter(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, uint32_t n,
                    int shift, const uint32_t* __restrict__ offsets, uint32_t nblocks) {
  __shared__ uint32_t whist[kSortWarps][kRadix];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads)
    (&whist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t base = blockIdx.x * kSortTile + wid * (32 * kSortItems);
  uint32_t k[kSortItems], v[kSortItems], local[kSortItems];
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    const uint32_t p = base + j * 32 + lane;
    const bool valid = p < n;
    k[j] = valid ? keys[p] : 0u;
    v[j] = valid ? vals[p] : 0u;
    const uint32_t d = valid ? ((k[j] >> shift) & 0xffu) : 256u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank_in = __popc(peers & lt_mask);
    uint32_t prior = 0;
    if (valid) prior = whist[wid][d];
    local[j] = prior + rank_in;
    __syncwarp();
    if (valid && rank_in == 0) whist[wid][d] = prior + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // exclusive prefix over warps for each digit
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      uint32_t t = whist[w][d];
      whist[w][d] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    const uint32_t p = base + j * 32 + lane;
    if (p < n) {
      const uint32_t d = (k[j] >> shift) & 0xffu;
      const uint32_t dst = offsets[d * nblocks + blockIdx.x] + whist[wid][d] + local[j];
      keys_out[dst] = k[j];
      vals_out[dst] = v[j];
    }
  }
}

}  // namespace

hr_status scan_u32(hr_ctx* ctx, uint32_t* data, uint32_t n, cudaStream_t st) {
  if (n == 0) return HR_OK;
  const uint32_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 1) {
    k_scan_tiles<<<1, kScanThreads, 0, st>>>(data, n, nullptr);
    HR_LAUNCHED(ctx);
    return HR_OK;
  }
  // levels of block sums; each level uses its own scratch slot (10, 11, 12)
  uint32_t* sums = nullptr;
  static const int kMaxLevels = 3;
  uint32_t counts[kMaxLevels + 1];
  uint32_t* bufs[kMaxLevels + 1];
  counts[0] = n;
  bufs[0] = data;
  int lv = 0;
  while (counts[lv] > (uint32_t)kScanTile) {
    if (lv >= kMaxLevels) return set_error(ctx, HR_EINVAL, "scan: input too large");
    const uint32_t b = (counts[lv] + kScanTile - 1) / kScanTile;
    HR_TRY(scratch(ctx, 10 + lv, (size_t)b * 4, (void**)&sums));
    k_scan_tiles<<<b, kScanThreads, 0, st>>>(bufs[lv], counts[lv], sums);
    HR_LAUNCHED(ctx);
    bufs[lv + 1] = sums;
    counts[lv + 1] = b;
    ++lv;
  }
  k_scan_tiles<<<1, kScanThreads, 0, st>>>(bufs[lv], counts[lv], nullptr);
  HR_LAUNCHED(ctx);
  for (int l = lv - 1; l >= 0; --l) {
    const uint32_t b = (counts[l] + kScanTile - 1) / kScanTile;
    k_scan_add<<<b, kScanThreads, 0, st>>>(bufs[l], counts[l], bufs[l + 1]);
    HR_LAUNCHED(ctx);
  }
  return HR_OK;
}

hr_status radix_sort_pairs(hr_ctx* ctx, uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp,
                           uint32_t* vals_tmp, uint32_t n, int bits, cudaStream_t st) {
  if (n <= 1) return HR_OK;
  const uint32_t nb = (n + kSortTile - 1) / kSortTile;
  uint32_t* counts = nullptr;
  HR_TRY(scratch(ctx, 13, (size_t)nb * kRadix * 4, (void**)&counts));
  uint32_t *ki = keys, *vi = vals, *ko = keys_tmp, *vo = vals_tmp;
  int passes = 0;
  for (int shift = 0; shift < bits; shift += 8, ++passes) {
    k_digit_hist<<<nb, kSortThreads, 0, st>>>(ki, n, shift, counts, nb);
    HR_LAUNCHED(ctx);
    HR_TRY(scan_u32(ctx, counts, nb * kRadix, st));
    k_digit_scatter<<<nb, kSortThreads, 0, st>>>(ki, vi, ko, vo, n, shift, counts, nb);
    HR_LAUNCHED(ctx);
    uint32_t* t;
    t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  if (passes & 1) {
    HR_CUDA(ctx, cudaMemcpyAsync(keys, ki, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    HR_CUDA(ctx, cudaMemcpyAsync(vals, vi, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
  }
  return HR_OK;
}

}  // namespace hr

namespace hr {

// Scan and radix sort on caller-provided scratch (no allocation).  `sums`
// holds ceil(n / 1024) words; n <= 1024 * 1024.
cudaError_t scan_u32_with(uint32_t* data, uint32_t n, uint32_t* sums, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const uint32_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb > (uint32_t)kScanTile) return cudaErrorInvalidValue;
  if (nb == 1) {
    k_scan_tiles<<<1, kScanThreads, 0, st>>>(data, n, nullptr);
    return cudaGetLastError();
  }
  k_scan_tiles<<<nb, kScanThreads, 0, st>>>(data, n, sums);
  k_scan_tiles<<<1, kScanThreads, 0, st>>>(sums, nb, nullptr);
  k_scan_add<<<nb, kScanThreads, 0, st>>>(data, n, sums);
  return cudaGetLastError();
}

cudaError_t radix_sort_pairs_with(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp,
                                  uint32_t* vals_tmp, uint32_t n, int bits, uint32_t* counts,
                                  uint32_t* sums, cudaStream_t st) {
  if (n <= 1) return cudaSuccess;
  const uint32_t nb = (n + kSortTile - 1) / kSortTile;
  uint32_t *ki = keys, *vi = vals, *ko = keys_tmp, *vo = vals_tmp;
  int passes = 0;
  for (int shift = 0; shift < bits; shift += 8, ++passes) {
    k_digit_hist<<<nb, kSortThreads, 0, st>>>(ki, n, shift, counts, nb);
    cudaError_t e = scan_u32_with(counts, nb * kRadix, sums, st);
    if (e != cudaSuccess) return e;
    k_digit_scatter<<<nb, kSortThreads, 0, st>>>(ki, vi, ko, vo, n, shift, counts, nb);
    uint32_t* t;
    t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  if (passes & 1) {
    cudaMemcpyAsync(keys, ki, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(vals, vi, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
  }
  return cudaGetLastError();
}

}  // namespace hr
