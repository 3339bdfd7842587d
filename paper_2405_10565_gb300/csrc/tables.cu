// Scattering lookup table, baked on the device once per context.
//
// IM(theta; beta) is the longitudinal factor of a lobe's directional albedo:
// the integral over theta_o in [-pi/2, pi/2] of G(beta, (theta + theta_o)/2)
// cos^2(theta_o), G the Gaussian with standard deviation beta (Section 3.2),
// cos^2 the measure of the rendering equation (Section 3).  The forward and
// backward attenuations a_F, a_B and the forward spread of the aggregated
// model (Eq. 6-13) are A_p * IM_p * (azimuthal mass of N_p in the half) summed
// over the lobes, so one table over (theta, beta) serves every material.
//
// Each cell is a composite Simpson sum over 512 intervals in FP32 with a
// compensated (Neumaier) running sum.  The narrowest lobe (beta = 0.04) is a
// Gaussian of standard deviation 0.08 in theta_o, about 13 intervals wide, so
// Simpson's truncation error is far below FP32 resolution; the compensated sum
// keeps the 513 terms' rounding at the level of one FP32 rounding of the
// result (1.4e-7 absolute in an FP32 emulation against an FP64 Gauss-Legendre
// integral).  Stored as FP32 and as FP16 (the FP16 table form).
#include "common.cuh"

namespace hr {
namespace {

constexpr int kSimpson = 512;

__global__ void k_bake_im(float* im32, __half* im16) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kImNT * kImNB) return;
  const int ib = idx / kImNT, it = idx % kImNT;
  const float beta = kImBetaLo + (kImBetaHi - kImBetaLo) * (float)ib / (float)(kImNB - 1);
  const float theta = (0.5f * kPi) * (float)it / (float)(kImNT - 1);
  const float h = kPi / (float)kSimpson;
  const float norm = kInvSqrt2Pi / beta;
  const float k2 = 0.5f / (beta * beta);
  float s = 0.f, comp = 0.f;
  for (int i = 0; i <= kSimpson; ++i) {
    // nodes centred on 0, so the grid is symmetric and exact near the middle
    const float to = (float)(i - kSimpson / 2) * h;
    const float x = 0.5f * (theta + to);
    const float c = cosf(to);
    const float w = (i == 0 || i == kSimpson) ? 1.f : ((i & 1) ? 4.f : 2.f);
    const float term = w * (norm * expf(-x * x * k2) * c * c);
    const float t = s + term;
    comp += fabsf(s) >= fabsf(term) ? (s - t) + term : (term - t) + s;
    s = t;
  }
  const float v = (s + comp) * (h / 3.f);
  im32[idx] = v;
  im16[idx] = __float2half_rn(v);
}

}  // namespace

hr_status bake_tables(hr_ctx* ctx, float** im32, __half** im16) {
  cudaStream_t st = ctx_stream(ctx);
  HR_TRY(dalloc(ctx, (void**)im32, sizeof(float) * kImNT * kImNB, "IM table"));
  HR_TRY(dalloc(ctx, (void**)im16, sizeof(__half) * kImNT * kImNB, "IM table fp16"));
  const int n = kImNT * kImNB;
  k_bake_im<<<(n + 127) / 128, 128, 0, st>>>(*im32, *im16);
  HR_LAUNCHED(ctx);
  return HR_OK;
}

}  // namespace hr
