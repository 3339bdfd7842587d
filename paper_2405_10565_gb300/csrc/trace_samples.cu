// Sample-list kernel (hr_render_samples): one thread per listed sample, the
// same per-sample device code as the frame kernel; returns radiance and the
// global id of the nearest hit.
#include "trace_core.cuh"

namespace hr {
namespace {

template <int KMAX, int PREC, bool SHADOW>
__global__ void __launch_bounds__(128)
    k_samples(const FrameArgs fa, const uint32_t* __restrict__ sids, uint32_t m,
              float* __restrict__ rad, int32_t* __restrict__ hit) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  tr::Counts cn{0, 0, 0, 0, 0, 0, 0, 0};
  float v[3];
  int32_t ids[KMAX];
  bool ok;
  tr::render_sample<KMAX, PREC, false, SHADOW>(fa, sids[i], v, ids, ok, cn);
  rad[3 * (size_t)i] = v[0];
  rad[3 * (size_t)i + 1] = v[1];
  rad[3 * (size_t)i + 2] = v[2];
#pragma unroll
  for (int j = 0; j < KMAX; ++j)
    if (j < (int)fa.k) hit[(size_t)fa.k * i + j] = ids[j];
  if (!ok) atomicAdd(fa.overflow, 1u);
}

template <int PREC, bool SHADOW>
hr_status launch_p(hr_ctx* ctx, const FrameArgs& fa, const uint32_t* sids, uint32_t m,
                   float* rad, int32_t* hit, cudaStream_t st) {
  const uint32_t g = (m + 127) / 128;
  switch (kmax_for(fa.k)) {
    case 1: k_samples<1, PREC, SHADOW><<<g, 128, 0, st>>>(fa, sids, m, rad, hit); break;
    case 2: k_samples<2, PREC, SHADOW><<<g, 128, 0, st>>>(fa, sids, m, rad, hit); break;
    case 4: k_samples<4, PREC, SHADOW><<<g, 128, 0, st>>>(fa, sids, m, rad, hit); break;
    default: k_samples<8, PREC, SHADOW><<<g, 128, 0, st>>>(fa, sids, m, rad, hit); break;
  }
  HR_LAUNCHED(ctx);
  return HR_OK;
}

// The bilinear IM(theta, beta) lookup of the shading code at listed points
// (test export).
template <int PREC>
__global__ void k_im_lookup(const Tables tb, const float* __restrict__ theta,
                            const float* __restrict__ beta, uint32_t m, float* __restrict__ out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = tr::im_lookup<PREC>(tb, theta[i], beta[i]);
}

template <bool SHADOW>
hr_status launch_t(hr_ctx* ctx, const FrameArgs& fa, int precision, const uint32_t* sids,
                   uint32_t m, float* rad, int32_t* hit, cudaStream_t st) {
  return precision == HR_PREC_FP16 ? launch_p<HR_PREC_FP16, SHADOW>(ctx, fa, sids, m, rad, hit, st)
                                   : launch_p<HR_PREC_FP32, SHADOW>(ctx, fa, sids, m, rad, hit, st);
}

}  // namespace

hr_status launch_im_lookup(hr_ctx* ctx, int precision, const float* theta, const float* beta,
                           uint32_t m, float* out, cudaStream_t st) {
  if (m == 0) return HR_OK;
  const uint32_t g = (m + 127) / 128;
  if (precision == HR_PREC_FP16)
    k_im_lookup<HR_PREC_FP16><<<g, 128, 0, st>>>(ctx_tables(ctx), theta, beta, m, out);
  else
    k_im_lookup<HR_PREC_FP32><<<g, 128, 0, st>>>(ctx_tables(ctx), theta, beta, m, out);
  HR_LAUNCHED(ctx);
  return HR_OK;
}

hr_status launch_samples(hr_ctx* ctx, const FrameArgs& fa, int precision, const uint32_t* sids,
                         uint32_t m, float* rad_dev, int32_t* hit_dev, cudaStream_t st) {
  if (m == 0) return HR_OK;
  return (fa.flags & HR_FLAG_SHADOWS) ? launch_t<true>(ctx, fa, precision, sids, m, rad_dev, hit_dev, st)
                                      : launch_t<false>(ctx, fa, precision, sids, m, rad_dev, hit_dev, st);
}

}  // namespace hr
