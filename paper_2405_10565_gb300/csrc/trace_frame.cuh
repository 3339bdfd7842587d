// Frame kernel (hot path of hr_render) and its launcher, shared by the two
// translation units that instantiate it without and with shadow rays (so
// that they compile in parallel).
#pragma once

#include <algorithm>

#include "trace_core.cuh"

namespace hr {
namespace {

// Projected scene rectangle of the frame and a cleared work counter, once per
// launch (one warp).
__global__ void k_scene_rect(const FrameArgs fa, float4* rect, uint32_t* work) {
  tr::scene_rect_warp(fa, rect);
  if (threadIdx.x == 0) *work = 0u;
}

// Persistent frame kernel.  The image has been cleared to background; the
// warp tiles (32 / grp pixels each) that overlap the projected scene rectangle
// are handed out one at a time through an atomic counter, so the few tiles
// that see hair spread over every warp of the GPU and a warp that drew cheap
// tiles takes more.  No warp ever waits for another.
// The plain instantiations are held to 4 blocks per SM (128 registers, no
// spills in the traversal): at 5 blocks (96 registers) the k-buffer's depth
// pairs and the precise-decision state spill, and the full-head frame took
// 1.01 instead of 0.64 ms; 3 blocks or no bound were no faster.
template <int KMAX, int PREC, bool COUNT, bool SHADOW>
__global__ void __launch_bounds__(kBlock, SHADOW ? 1 : 4)
    k_frame(const FrameArgs fa, const float4* __restrict__ rect_p, uint32_t* work,
            float* __restrict__ rgb) {
  const float4 rect = *rect_p;
  const WarpGrid g = warp_grid(rect, (uint32_t)fa.cam.W, (uint32_t)fa.cam.H, fa.grp);
  tr::Counts cn{0, 0, 0, 0, 0, 0, 0, 0};
  bool overflow = false;
  const uint32_t lane = threadIdx.x & 31;
  if (COUNT && fa.tile_log && blockIdx.x == 0 && threadIdx.x == 0) *fa.tile_count = g.n;
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(work, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= g.n) break;
    uint64_t t0 = 0;
    uint32_t nodes0 = 0, tests0 = 0;
    if (COUNT && fa.tile_log) {
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      nodes0 = cn.nodes;
      tests0 = cn.tests;
    }
    tr::render_warp_tile<KMAX, PREC, COUNT, SHADOW>(fa, g.x0 + (t % g.nx) * g.wtw,
                                                    g.y0 + (t / g.nx) * g.wth, g.wtw, rect, rgb,
                                                    cn, overflow);
    if (COUNT && fa.tile_log) {
      uint32_t dn = cn.nodes - nodes0, dt = cn.tests - tests0;
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        dn = max(dn, __shfl_xor_sync(0xffffffffu, dn, o));
        dt = max(dt, __shfl_xor_sync(0xffffffffu, dt, o));
      }
      uint64_t t1;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
      if (lane == 0 && t < fa.tile_cap) {
        uint32_t sm;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
        fa.tile_log[t] = hr_tile_record{t0, t1, t, sm, dn, dt};
      }
    }
  }
  if (COUNT) tr::flush_counts(fa, cn);
  if (overflow) atomicAdd(fa.overflow, 1u);
}

template <int KMAX, int PREC, bool COUNT, bool SHADOW>
int frame_grid() {
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 1, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_frame<KMAX, PREC, COUNT, SHADOW>, kBlock,
                                                      0) != cudaSuccess) {
      cudaGetLastError();
      per = 4;
    }
    grid = sms * (per > 0 ? per : 1);
  }
  return grid;
}

template <int KMAX, int PREC, bool SHADOW>
hr_status launch_k(hr_ctx* ctx, const FrameArgs& fa, bool count, float* rgb, cudaStream_t st) {
  const uint32_t tiles = tiles_for(fa.cam.W, fa.cam.H, fa.spp);
  float4* rect = nullptr;
  HR_TRY(scratch(ctx, 47, 2 * sizeof(float4), (void**)&rect));
  uint32_t* work = reinterpret_cast<uint32_t*>(rect + 1);
  HR_CUDA(ctx, cudaMemsetAsync(rgb, 0, (size_t)fa.cam.W * fa.cam.H * 3 * sizeof(float), st));
  k_scene_rect<<<1, 32, 0, st>>>(fa, rect, work);
  HR_LAUNCHED(ctx);
  if (count) {
    const int g = (int)std::min<uint32_t>(tiles, frame_grid<KMAX, PREC, true, SHADOW>());
    k_frame<KMAX, PREC, true, SHADOW><<<g, kBlock, 0, st>>>(fa, rect, work, rgb);
  } else {
    const int g = (int)std::min<uint32_t>(tiles, frame_grid<KMAX, PREC, false, SHADOW>());
    k_frame<KMAX, PREC, false, SHADOW><<<g, kBlock, 0, st>>>(fa, rect, work, rgb);
  }
  HR_LAUNCHED(ctx);
  return HR_OK;
}

template <int PREC, bool SHADOW>
hr_status launch_p(hr_ctx* ctx, const FrameArgs& fa, bool count, float* rgb, cudaStream_t st) {
  switch (kmax_for(fa.k)) {
    case 1: return launch_k<1, PREC, SHADOW>(ctx, fa, count, rgb, st);
    case 2: return launch_k<2, PREC, SHADOW>(ctx, fa, count, rgb, st);
    case 4: return launch_k<4, PREC, SHADOW>(ctx, fa, count, rgb, st);
    default: return launch_k<8, PREC, SHADOW>(ctx, fa, count, rgb, st);
  }
}

template <bool SHADOW>
hr_status launch_frame_t(hr_ctx* ctx, const FrameArgs& fa, int precision, bool count,
                         float* rgb_dev, cudaStream_t st) {
  if (fa.cam.W <= 0 || fa.cam.H <= 0) return HR_OK;
  return precision == HR_PREC_FP16 ? launch_p<HR_PREC_FP16, SHADOW>(ctx, fa, count, rgb_dev, st)
                                   : launch_p<HR_PREC_FP32, SHADOW>(ctx, fa, count, rgb_dev, st);
}

}  // namespace
}  // namespace hr
