// Device-wide exclusive scan and stable LSD radix sort of (uint32 key, uint32
// value) pairs.  Used by the Morton clustering of strands and by the linear
// BVH build.  Two forms of the sort: a single sweep per digit pass (the
// library's), and histogram / scan / scatter kernels per pass on
// caller-provided buffers (the allocation-free clustering entry point).
#include <algorithm>

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

// ------------------------------------------------ single-sweep radix sort
//
// The stable LSD sort with one kernel per digit pass (Merrill and Garland's
// decoupled look-back applied to radix sorting, as in Adinets and Merrill's
// Onesweep): the digit totals of every pass come from one histogram kernel,
// and each tile finds the offsets of its digits among the earlier tiles by
// reading their published counts instead of through a device-wide scan.

constexpr uint32_t kFlagAgg = 1u << 30;  // tile's own digit count
constexpr uint32_t kFlagInc = 2u << 30;  // count of this and every earlier tile
constexpr uint32_t kCountMask = kFlagAgg - 1u;
constexpr int kLookbackWindow = 8;
constexpr int kSweepItems = 12;  // keys per thread
constexpr uint32_t kSweepTile = kSortThreads * kSweepItems;

// Digit totals of every pass in one read of the keys: hist[q * 256 + d].
__global__ void k_pass_hist(const uint32_t* __restrict__ keys, uint32_t n, int bits,
                            uint32_t* __restrict__ hist) {
  const int passes = (bits + 7) / 8;
  const uint32_t low = bits >= 32 ? 0xffffffffu : (1u << bits) - 1u;  // only the low bits count
  __shared__ uint32_t h[4][kRadix];
  for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const uint32_t k = keys[p];
    for (int q = 0; q < passes; ++q) atomicAdd(&h[q][((k & low) >> (8 * q)) & 0xffu], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) {
    const uint32_t v = (&h[0][0])[i];
    if (v) atomicAdd(hist + i, v);
  }
}

// One digit pass.  Tiles are numbered in the order their blocks start, so a
// tile only ever waits for tiles whose blocks are already running.  Tile t
// ranks its keys stably (per-warp digit counts; lanes with equal digits found
// by one vote per digit bit), publishes its digit counts, then
// (thread d for digit d) walks back over the earlier tiles' published words,
// adding counts until it meets a word that already holds an inclusive count.
// If a wait outlasts max_polls reads (kLookbackPolls in the library) the
// block counts the digits of all earlier keys itself, which gives the same
// offsets.
__global__ void __launch_bounds__(kSortThreads)
    k_sweep(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
            uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, uint32_t n, int shift,
            const uint32_t* __restrict__ totals, uint32_t* status, uint32_t* tile_ctr,
            int max_polls, uint32_t dm) {
  static_assert(kSortThreads == kRadix && kSortThreads == kScanThreads, "one thread per digit");
  __shared__ uint32_t whist[kSortWarps][kRadix];
  __shared__ uint32_t s_off[kRadix];
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_key[kSweepTile], s_val[kSweepTile];  // the tile in digit order
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
  for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&whist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t t = s_tile;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t base = t * kSweepTile + wid * (32 * kSweepItems);
  uint32_t k[kSweepItems], v[kSweepItems], local[kSweepItems];
#pragma unroll
  for (int j = 0; j < kSweepItems; ++j) {  // every load in flight before the ranking
    const uint32_t p = base + j * 32 + lane;
    k[j] = p < n ? keys[p] : 0u;
    v[j] = p < n ? vals[p] : 0u;
  }
#pragma unroll
  for (int j = 0; j < kSweepItems; ++j) {
    const bool valid = base + j * 32 + lane < n;
    const uint32_t d = valid ? ((k[j] >> shift) & dm) : 0u;
    // lanes with the same digit: one vote per digit bit, and one for validity
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
    if (!valid) peers = ~peers;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const bool bit = (d >> b) & 1u;
      const uint32_t vote = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? vote : ~vote;
    }
    const uint32_t rank_in = __popc(peers & lt_mask);
    uint32_t prior = 0;
    if (valid) prior = whist[wid][d];
    local[j] = prior + rank_in;
    __syncwarp();
    if (valid && rank_in == 0) whist[wid][d] = prior + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  const uint32_t d = threadIdx.x;
  uint32_t c = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {
    const uint32_t x = whist[w][d];
    whist[w][d] = c;
    c += x;
  }
  volatile uint32_t* vs = status;
  vs[(size_t)t * kRadix + d] = (t == 0 ? kFlagInc : kFlagAgg) | c;
  uint32_t all;
  const uint32_t dstart = block_excl_scan(__ldg(totals + d), &all);
  uint32_t excl = 0;
  bool gave_up = t > 0 && max_polls == 0;  // 0: always count (tests the path below)
  if (t > 0 && !gave_up) {
    // kLookbackWindow earlier tiles per read, nearest first: counts are added
    // up to the first inclusive word; a tile not yet published stops the walk
    // there until a later read finds it
    int kt = (int)t - 1;
    int polls = 0;
    for (;;) {
      uint32_t w[kLookbackWindow];
#pragma unroll
      for (int i = 0; i < kLookbackWindow; ++i)
        w[i] = kt - i >= 0 ? (uint32_t)vs[(size_t)(kt - i) * kRadix + d] : (uint32_t)kFlagInc;
      int used = 0;
      bool inc = false;
#pragma unroll
      for (int i = 0; i < kLookbackWindow; ++i) {
        if (used == i && w[i] != 0u && !inc) {
          excl += w[i] & kCountMask;
          inc = (w[i] & kFlagInc) != 0u;
          ++used;
        }
      }
      if (inc) break;
      kt -= used;  // tile 0 publishes an inclusive count, so kt stays >= 0
      if (used == 0 && ++polls > max_polls) {
        gave_up = true;
        break;
      }
    }
  }
  if (__syncthreads_or(gave_up)) {
    uint32_t* cnt = s_off;
    cnt[d] = 0;
    __syncthreads();
    for (uint32_t p = threadIdx.x; p < t * kSweepTile; p += kSortThreads)
      atomicAdd(&cnt[(keys[p] >> shift) & dm], 1u);
    __syncthreads();
    excl = cnt[d];
    __syncthreads();
  }
  if (t > 0) vs[(size_t)t * kRadix + d] = kFlagInc | (excl + c);
  // digit d's keys take places [tstart, tstart + c) of the tile in digit
  // order, and the output from dstart + excl on
  const uint32_t tstart = block_excl_scan(c, &all);
  s_off[d] = dstart + excl - tstart;  // output index = s_off[digit] + tile place
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) whist[w][d] += tstart;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kSweepItems; ++j) {
    if (base + j * 32 + lane < n) {
      const uint32_t q = whist[wid][(k[j] >> shift) & dm] + local[j];
      s_key[q] = k[j];
      s_val[q] = v[j];
    }
  }
  __syncthreads();
  // the tile in digit order: consecutive threads write consecutive places of
  // each digit's run
  const uint32_t tile_n = min(kSweepTile, n - t * kSweepTile);
  for (uint32_t i = threadIdx.x; i < tile_n; i += kSortThreads) {
    const uint32_t key = s_key[i];
    const uint32_t dst = s_off[(key >> shift) & dm] + i;
    keys_out[dst] = key;
    vals_out[dst] = s_val[i];
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
                           uint32_t* vals_tmp, uint32_t n, int bits, cudaStream_t st,
                           int max_polls, uint32_t** keys_out, uint32_t** vals_out) {
  if (keys_out) *keys_out = keys;
  if (vals_out) *vals_out = vals;
  if (n <= 1) return HR_OK;
  if (n >= kFlagAgg || bits < 1 || bits > 32) return set_error(ctx, HR_EINVAL, "sort: size out of range");
  const int passes = (bits + 7) / 8;
  const uint32_t nb = (n + kSweepTile - 1) / kSweepTile;
  // pass totals (passes x 256), tile counters (64 words), then the tiles'
  // published counts (passes x nb x 256), all cleared here
  const size_t words = (size_t)passes * kRadix + 64 + (size_t)passes * nb * kRadix;
  uint32_t* ws = nullptr;
  HR_TRY(scratch(ctx, 14, words * 4, (void**)&ws));
  HR_CUDA(ctx, cudaMemsetAsync(ws, 0, words * 4, st));
  uint32_t* totals = ws;
  uint32_t* ctr = ws + (size_t)passes * kRadix;
  uint32_t* status = ctr + 64;
  const uint32_t hb = std::min<uint32_t>(nb, 1024u);
  k_pass_hist<<<hb, kSortThreads, 0, st>>>(keys, n, bits, totals);
  HR_LAUNCHED(ctx);
  uint32_t *ki = keys, *vi = vals, *ko = keys_tmp, *vo = vals_tmp;
  for (int q = 0; q < passes; ++q) {
    // digit q holds key bits [8q, min(8q + 8, bits))
    const uint32_t dm = bits - 8 * q >= 8 ? 0xffu : (1u << (bits - 8 * q)) - 1u;
    k_sweep<<<nb, kSortThreads, 0, st>>>(ki, vi, ko, vo, n, 8 * q, totals + q * kRadix,
                                         status + (size_t)q * nb * kRadix, ctr + q, max_polls, dm);
    HR_LAUNCHED(ctx);
    uint32_t* t;
    t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  if (keys_out && vals_out) {  // the caller takes the result where the last pass left it
    *keys_out = ki;
    *vals_out = vi;
  } else if (passes & 1) {
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
