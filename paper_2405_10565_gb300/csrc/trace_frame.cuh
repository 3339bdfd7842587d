// Frame kernel (hot path of hr_render) and its launcher, shared by the two
// translation units that instantiate it without and with shadow rays (so
// that they compile in parallel).
#pragma once

#include <algorithm>

#include "trace_core.cuh"

namespace hr {
namespace {

// Projected scene rectangle of the frame and a cleared work counter, once per
// launch (warp 0).  With a tile schedule (fa.sched), the block also picks
// this frame's heavy tiles among the previous frame's candidates (TileSched):
// those whose slowest lane took at least kHeavyRelPct percent of the steps of
// that frame's slowest tile and more than kHeavyMinSteps, at most kHeavyMax
// of them (the heaviest), stored by their pixel origin heaviest first.  The
// previous frame's warp grid is rebuilt from its scene rectangle, which the
// block then replaces with this frame's, and the candidate threshold of this
// frame is set from the previous frame's largest count.  A previous frame of
// another size or spp, or a frame of more than kHeavyTilesPerWarp tiles per
// resident warp, gives no heavy tiles.  One thread per candidate.
constexpr int kRectThreads = (int)kCandMax;
__global__ void __launch_bounds__(kRectThreads) k_scene_rect(const FrameArgs fa, float4* rect,
                                                             uint32_t* work) {
  if (threadIdx.x < 32) tr::scene_rect_warp(fa, rect);
  if (threadIdx.x == 0) *work = 0u;
  TileSched* sc = fa.sched;
  if (!sc) return;
  __shared__ uint32_t s_hist[256], s_cut, s_n;
  __shared__ uint32_t s_tile[kHeavyMax], s_steps[kHeavyMax];
  const uint32_t tid = threadIdx.x;
  const bool have = sc->prev_n > 0 && sc->prev_W == (uint32_t)fa.cam.W &&
                    sc->prev_H == (uint32_t)fa.cam.H && sc->prev_grp == fa.grp;
  const uint32_t M = have ? sc->max_steps : 0u;
  if (tid == 0) {
    s_cut = 0u;
    s_n = 0u;
  }
  if (tid < 256) s_hist[tid] = 0u;
  __syncthreads();
  const float4 rc = *rect;  // written by warp 0 before the barrier
  const WarpGrid g = warp_grid(rc, (uint32_t)fa.cam.W, (uint32_t)fa.cam.H, fa.grp);
  const bool allow = (uint64_t)g.n <= (uint64_t)kHeavyTilesPerWarp * fa.frame_warps;
  const uint32_t nc = have && allow ? min(sc->cand_n, kCandMax) : 0u;
  const bool mine = tid < nc;
  const uint32_t c = mine ? sc->cand_steps[tid] : 0u;
  const uint32_t ct = mine ? sc->cand_tile[tid] : 0u;
  // steps in [lo, M] binned into 256 bins; the cut is the highest bin with
  // at least kHeavyMax candidates at or above it (else bin 0), and those
  // past kHeavyMax in the cut's bin are left out
  const uint32_t lo = max((uint32_t)((uint64_t)M * kHeavyRelPct / 100u), kHeavyMinSteps + 1);
  const uint32_t span = M >= lo ? M - lo + 1 : 1u;
  const bool cand = mine && c >= lo && ct < sc->prev_n;
  const uint32_t b = cand ? (uint32_t)((uint64_t)(min(c, M) - lo) * 256u / span) : 0u;
  if (cand) atomicAdd(&s_hist[b], 1u);
  __syncthreads();
  // suffix sums of the histogram (Hillis-Steele over 256 bins)
  for (uint32_t o = 1; o < 256; o <<= 1) {
    uint32_t v = 0;
    if (tid < 256) v = s_hist[tid] + (tid + o < 256 ? s_hist[tid + o] : 0u);
    __syncthreads();
    if (tid < 256) s_hist[tid] = v;
    __syncthreads();
  }
  if (tid < 256 && s_hist[tid] >= kHeavyMax) atomicMax(&s_cut, tid);
  __syncthreads();
  const uint32_t cut = s_cut;
  // the bins above the cut first (fewer than kHeavyMax candidates), then the cut's
  for (int pass = 0; pass < 2; ++pass) {
    if (cand && (pass == 0 ? b > cut : b == cut)) {
      const uint32_t k = atomicAdd(&s_n, 1u);
      if (k < kHeavyMax) {
        s_tile[k] = ct;
        s_steps[k] = c;
      }
    }
    __syncthreads();
  }
  const uint32_t nh = min(s_n, kHeavyMax);
  if (tid < nh) {  // heaviest first (ties by tile index): rank by counting
    uint32_t r = 0;
    for (uint32_t k = 0; k < nh; ++k)
      r += s_steps[k] > s_steps[tid] || (s_steps[k] == s_steps[tid] && s_tile[k] < s_tile[tid]);
    const WarpGrid pg = warp_grid(sc->prev_rect, (uint32_t)fa.cam.W, (uint32_t)fa.cam.H, fa.grp);
    const uint32_t t = s_tile[tid];
    sc->heavy[r] = (pg.x0 + (t % pg.nx) * pg.wtw) | ((pg.y0 + (t / pg.nx) * pg.wth) << 16);
  }
  if (tid < kHeavyMax) sc->done[tid] = 0u;
  __syncthreads();  // the previous frame's candidates and grid are no longer read
  if (tid == 0) {
    sc->n_heavy = nh;
    sc->grp = fa.grp;
    sc->thresh = lo;
    sc->max_steps = 0u;
    sc->cand_n = 0u;
    sc->prev_rect = rc;
    sc->prev_n = g.n;
    sc->prev_W = (uint32_t)fa.cam.W;
    sc->prev_H = (uint32_t)fa.cam.H;
    sc->prev_grp = fa.grp;
  }
}

// Persistent frame kernel.  The image has been cleared to background; the
// warp tiles (32 / grp pixels each) that overlap the projected scene rectangle
// are handed out one at a time through an atomic counter, so the few tiles
// that see hair spread over every warp of the GPU and a warp that drew cheap
// tiles takes more.  With a schedule, the hand-outs start with the heavy
// tiles (TileSched), kHeavyRays lanes each; the warp that finishes a heavy
// tile's last hand-out composites it.  No warp ever waits for another.
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
  // heavy tiles first, kHeavyRays rays per hand-out (kernels without a
  // schedule: none)
  TileSched* sc = fa.sched;
  const uint32_t nh = sc && sc->grp == fa.grp ? min(sc->n_heavy, kHeavyMax) : 0u;
  const uint32_t thresh = sc ? sc->thresh : 0u;
  uint32_t wmax = 0;  // the warp's largest tile step count
  // a tile's slowest-lane steps: the warp's maximum, and a candidate for the
  // next frame's heavy tiles at or above the threshold (lane 0)
  auto note = [&](uint32_t tile, uint32_t st) {
    wmax = max(wmax, st);
    if (lane == 0 && st >= thresh && __ldcg(&sc->cand_n) < kCandMax) {  // no atomics once full
      const uint32_t k = atomicAdd(&sc->cand_n, 1u);
      if (k < kCandMax) {
        sc->cand_tile[k] = tile;
        sc->cand_steps[k] = st;
      }
    }
  };
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(work, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t < nh * kHeavyItems) {
      const uint32_t ht = t / kHeavyItems, j0 = (t % kHeavyItems) * kHeavyRays;
      const uint32_t mask = (0xffffffffu >> (32u - kHeavyRays)) << j0;
      const uint32_t xy = sc->heavy[ht];
      const uint32_t x0 = xy & 0xffffu, y0 = xy >> 16;
      // a tile of the previous frame's grid that is not one of this grid's: skipped
      const uint32_t gx = (x0 - g.x0) / g.wtw, gy = (y0 - g.y0) / g.wth;
      if (x0 < g.x0 || y0 < g.y0 || (x0 - g.x0) % g.wtw || (y0 - g.y0) % g.wth || gx >= g.nx ||
          gy * g.nx + gx >= g.n)
        continue;
      const uint32_t steps0 = cn.steps;
      float acc[3];
      tr::tile_partials<KMAX, PREC, COUNT, SHADOW>(fa, x0, y0, g.wtw, rect, mask, acc, cn,
                                                   overflow);
      if ((mask >> lane) & 1u) {
        float* a = sc->acc + (size_t)(ht * 32u + lane) * 3;
        a[0] = acc[0];
        a[1] = acc[1];
        a[2] = acc[2];
        sc->ray_steps[ht * 32u + lane] = cn.steps - steps0;
      }
      __syncwarp();
      uint32_t last = 0;
      if (lane == j0) {
        __threadfence();
        last = atomicAdd(&sc->done[ht], 1u) == kHeavyItems - 1u;
      }
      last = __shfl_sync(0xffffffffu, last, j0);
      if (last) {  // every ray of the tile is done: composite its pixels
        __threadfence();
        const float* a = sc->acc + (size_t)(ht * 32u + lane) * 3;
        acc[0] = __ldcg(a);
        acc[1] = __ldcg(a + 1);
        acc[2] = __ldcg(a + 2);
        uint32_t st = __ldcg(sc->ray_steps + ht * 32u + lane);
#pragma unroll
        for (int o = 16; o; o >>= 1) st = max(st, __shfl_xor_sync(0xffffffffu, st, o));
        tr::tile_write(fa, x0, y0, g.wtw, rect, acc, rgb);
        note(gy * g.nx + gx, st);
      }
      continue;
    }
    t -= nh * kHeavyItems;
    if (t >= g.n) break;
    const uint32_t x0 = g.x0 + (t % g.nx) * g.wtw, y0 = g.y0 + (t / g.nx) * g.wth;
    if (nh) {  // traced ray by ray above
      const uint32_t xy = x0 | (y0 << 16);
      const bool mine = (lane < nh && sc->heavy[lane] == xy) ||
                        (lane + 32u < nh && sc->heavy[lane + 32u] == xy);
      if (__any_sync(0xffffffffu, mine)) continue;
    }
    const uint32_t steps0 = cn.steps;
    uint64_t t0 = 0;
    uint32_t nodes0 = 0, tests0 = 0;
    if (COUNT && fa.tile_log) {
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      nodes0 = cn.nodes;
      tests0 = cn.tests;
    }
    tr::render_warp_tile<KMAX, PREC, COUNT, SHADOW>(fa, x0, y0, g.wtw, rect, rgb, cn, overflow);
    if (sc) {
      uint32_t st = cn.steps - steps0;
#pragma unroll
      for (int o = 16; o; o >>= 1) st = max(st, __shfl_xor_sync(0xffffffffu, st, o));
      note(t, st);
    }
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
  if (sc && lane == 0 && wmax) atomicMax(&sc->max_steps, wmax);
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
  // the counting kernel keeps the plain hand-out order (its tile log is indexed by it)
  FrameArgs f = fa;
  if (count) f.sched = nullptr;
  f.frame_warps = (uint32_t)frame_grid<KMAX, PREC, false, SHADOW>() * (kBlock / 32);
  k_scene_rect<<<1, kRectThreads, 0, st>>>(f, rect, work);
  HR_LAUNCHED(ctx);
  if (count) {
    const int g = (int)std::min<uint32_t>(tiles, frame_grid<KMAX, PREC, true, SHADOW>());
    k_frame<KMAX, PREC, true, SHADOW><<<g, kBlock, 0, st>>>(f, rect, work, rgb);
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
