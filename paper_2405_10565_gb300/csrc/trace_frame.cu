// Frame kernel: one 128-thread block per 16 x 8 pixel tile, one pixel per
// thread, all of the pixel's samples in that thread (hot path of hr_render).
#include "trace_core.cuh"

namespace hr {
namespace {

template <int KMAX, int PREC, bool COUNT>
__global__ void __launch_bounds__(kBlock)
    k_frame(const FrameArgs fa, float* __restrict__ rgb) {
  __shared__ float4 s_rect;
  tr::scene_rect(fa, &s_rect);
  tr::Counts cn{0, 0, 0, 0, 0, 0};
  bool overflow = false;
  tr::render_tile<KMAX, PREC, COUNT>(fa, blockIdx.x, s_rect, rgb, cn, overflow);
  if (COUNT) tr::flush_counts(fa, cn);
  if (overflow) atomicAdd(fa.overflow, 1u);
}

template <int KMAX, int PREC>
hr_status launch_k(hr_ctx* ctx, const FrameArgs& fa, bool count, float* rgb, cudaStream_t st) {
  const uint32_t tiles = tiles_for(fa.cam.W, fa.cam.H, fa.spp);
  if (count)
    k_frame<KMAX, PREC, true><<<tiles, kBlock, 0, st>>>(fa, rgb);
  else
    k_frame<KMAX, PREC, false><<<tiles, kBlock, 0, st>>>(fa, rgb);
  HR_LAUNCHED(ctx);
  return HR_OK;
}

template <int PREC>
hr_status launch_p(hr_ctx* ctx, const FrameArgs& fa, bool count, float* rgb, cudaStream_t st) {
  switch (kmax_for(fa.k)) {
    case 1: return launch_k<1, PREC>(ctx, fa, count, rgb, st);
    case 2: return launch_k<2, PREC>(ctx, fa, count, rgb, st);
    case 4: return launch_k<4, PREC>(ctx, fa, count, rgb, st);
    default: return launch_k<8, PREC>(ctx, fa, count, rgb, st);
  }
}

}  // namespace

int kmax_for(uint32_t k) { return k <= 1 ? 1 : (k <= 2 ? 2 : (k <= 4 ? 4 : 8)); }

hr_status launch_frame(hr_ctx* ctx, const FrameArgs& fa, int precision, bool count,
                       float* rgb_dev, cudaStream_t st) {
  if (fa.cam.W <= 0 || fa.cam.H <= 0) return HR_OK;
  return precision == HR_PREC_FP16 ? launch_p<HR_PREC_FP16>(ctx, fa, count, rgb_dev, st)
                                   : launch_p<HR_PREC_FP32>(ctx, fa, count, rgb_dev, st);
}

LaunchCam to_launch_cam(const hr_camera& c) {
  LaunchCam l;
  l.kind = c.kind;
  l.W = (int)c.width;
  l.H = (int)c.height;
  l.pix = c.pix_scale;
  l.eye = make_float3(c.eye[0], c.eye[1], c.eye[2]);
  l.right = make_float3(c.right[0], c.right[1], c.right[2]);
  l.up = make_float3(c.up[0], c.up[1], c.up[2]);
  l.fwd = make_float3(c.fwd[0], c.fwd[1], c.fwd[2]);
  return l;
}

LaunchLights to_launch_lights(const hr_render_desc& d) {
  LaunchLights L{};
  L.n = (int)d.n_lights;
  for (uint32_t i = 0; i < d.n_lights && i < HR_MAX_LIGHTS; ++i) {
    const hr_light& s = d.lights[i];
    float x = s.xyz[0], y = s.xyz[1], z = s.xyz[2];
    if (s.type == 0.f) {  // directional: unit vector toward the light
      const float n = sqrtf(x * x + y * y + z * z);
      if (n > 0.f) x /= n, y /= n, z /= n;
    }
    L.xyzw[i] = make_float4(x, y, z, s.type);
    L.rgb[i] = make_float4(s.rgb[0], s.rgb[1], s.rgb[2], 0.f);
  }
  return L;
}

}  // namespace hr
