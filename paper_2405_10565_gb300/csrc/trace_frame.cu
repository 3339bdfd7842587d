// Frame kernel (hot path of hr_render): persistent warps, one sample per
// lane; this unit instantiates it without shadow rays (trace_frame_shadow.cu
// with them) and holds the host-side camera and light conversions.
#include "trace_frame.cuh"

namespace hr {

int kmax_for(uint32_t k) { return k <= 1 ? 1 : (k <= 2 ? 2 : (k <= 4 ? 4 : 8)); }

hr_status launch_frame(hr_ctx* ctx, const FrameArgs& fa, int precision, bool count,
                       float* rgb_dev, cudaStream_t st) {
  if (fa.flags & HR_FLAG_SHADOWS) return launch_frame_shadow(ctx, fa, precision, count, rgb_dev, st);
  return launch_frame_t<false>(ctx, fa, precision, count, rgb_dev, st);
}

LaunchCam to_launch_cam(const hr_camera& c) {
  LaunchCam l;
  l.kind = c.kind;
  l.W = (int)c.width;
  l.H = (int)c.height;
  l.pix = c.pix_scale;
  const double ip = 1.0 / (double)c.pix_scale;
  l.ipix_hi = (float)ip;
  l.ipix_lo = (float)(ip - (double)l.ipix_hi);
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
