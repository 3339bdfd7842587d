// Batched persistent serving kernel: one launch renders warp tiles of several
// requests.  Warps take batch tiles from a work counter until the batch is
// exhausted (no warp ever waits on another), locate the owning item by binary
// search over the items' first batch tiles, and render that warp tile with
// the item's own scene, camera and output, as the frame kernel does: only the
// tiles over a request's projected scene rectangle are enumerated, the rest
// of its image having been cleared to background at admission.
#include <algorithm>

#include "serve.h"
#include "trace_core.cuh"

namespace hr {
namespace {

__global__ void k_serve_rect(const FrameArgs fa, float4* rect) { tr::scene_rect_warp(fa, rect); }

template <int KMAX, int PREC>
// 4 blocks per SM (at most 128 registers), as for the frame kernel.
__global__ void __launch_bounds__(kBlock, 4)
    k_serve(const ServeItem* __restrict__ items, const uint32_t* __restrict__ item_start,
            uint32_t n_items, uint32_t total, uint32_t* work) {
  const uint32_t lane = threadIdx.x & 31;
  for (;;) {
    uint32_t bt = 0;
    if (lane == 0) bt = atomicAdd(work, 1u);
    bt = __shfl_sync(0xffffffffu, bt, 0);
    if (bt >= total) return;
    uint32_t lo = 0, hi = n_items;  // last item with start <= bt
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (item_start[mid] <= bt) lo = mid; else hi = mid;
    }
    const ServeItem& it = items[lo];
    const WarpGrid g = it.grid;
    const uint32_t t = it.wt0 + (bt - item_start[lo]);
    tr::Counts cn{0, 0, 0, 0, 0, 0, 0, 0};
    bool overflow = false;
    tr::render_warp_tile<KMAX, PREC, false>(it.fa, g.x0 + (t % g.nx) * g.wtw,
                                            g.y0 + (t / g.nx) * g.wth, g.wtw, it.rect, it.rgb, cn,
                                            overflow);
    if (overflow) atomicAdd(it.fa.overflow, 1u);
  }
}

template <int PREC>
hr_status launch_p(hr_ctx* ctx, int kmax, const ServeItem* items, const uint32_t* starts,
                   uint32_t n, uint32_t total, uint32_t* work, int grid, cudaStream_t st) {
  switch (kmax) {
    case 1: k_serve<1, PREC><<<grid, kBlock, 0, st>>>(items, starts, n, total, work); break;
    case 2: k_serve<2, PREC><<<grid, kBlock, 0, st>>>(items, starts, n, total, work); break;
    case 4: k_serve<4, PREC><<<grid, kBlock, 0, st>>>(items, starts, n, total, work); break;
    default: k_serve<8, PREC><<<grid, kBlock, 0, st>>>(items, starts, n, total, work); break;
  }
  HR_LAUNCHED(ctx);
  return HR_OK;
}

}  // namespace

int serve_grid(int kmax, int precision) {
  int dev = 0, sms = 1, blocks = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void* fn = nullptr;
  if (precision == HR_PREC_FP16) {
    fn = kmax <= 1 ? (const void*)k_serve<1, HR_PREC_FP16> : kmax <= 2 ? (const void*)k_serve<2, HR_PREC_FP16>
       : kmax <= 4 ? (const void*)k_serve<4, HR_PREC_FP16> : (const void*)k_serve<8, HR_PREC_FP16>;
  } else {
    fn = kmax <= 1 ? (const void*)k_serve<1, HR_PREC_FP32> : kmax <= 2 ? (const void*)k_serve<2, HR_PREC_FP32>
       : kmax <= 4 ? (const void*)k_serve<4, HR_PREC_FP32> : (const void*)k_serve<8, HR_PREC_FP32>;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, kBlock, 0) != cudaSuccess) {
    cudaGetLastError();
    blocks = 4;
  }
  return sms * std::max(1, blocks);
}

hr_status launch_scene_rect(hr_ctx* ctx, const FrameArgs& fa, float4* rect_dev, cudaStream_t st) {
  k_serve_rect<<<1, 32, 0, st>>>(fa, rect_dev);
  HR_LAUNCHED(ctx);
  return HR_OK;
}

hr_status launch_serve_batch(hr_ctx* ctx, int kmax, int precision, const ServeItem* items_dev,
                             const uint32_t* item_start_dev, uint32_t n_items,
                             uint32_t total_tiles, uint32_t* work_counter_dev, int grid,
                             cudaStream_t st) {
  if (n_items == 0 || total_tiles == 0) return HR_OK;
  return precision == HR_PREC_FP16
             ? launch_p<HR_PREC_FP16>(ctx, kmax, items_dev, item_start_dev, n_items, total_tiles,
                                      work_counter_dev, grid, st)
             : launch_p<HR_PREC_FP32>(ctx, kmax, items_dev, item_start_dev, n_items, total_tiles,
                                      work_counter_dev, grid, st);
}

}  // namespace hr
