// Scattering lookup tables, baked on the device once per context.
//
// IM(theta; beta) is the longitudinal factor of a lobe's directional albedo:
// the integral over theta_o in [-pi/2, pi/2] of G(beta, (theta + theta_o)/2)
// cos^2(theta_o), G the Gaussian with standard deviation beta (Section 3.2),
// cos^2 the measure of the rendering equation (Section 3).  The forward and
// backward attenuations a_F, a_B of the aggregated model (Eq. 6-13) are
// A_p * IM_p * (azimuthal mass of N_p in the half) summed over the lobes, so
// one table over (theta, beta) serves every material.  It is integrated in
// FP64 with composite Simpson on 4096 intervals and stored as FP32 and FP16.
#include "common.cuh"

namespace hr {
namespace {

constexpr int kSimpson = 4096;

__global__ void k_bake_im(float* im32, __half* im16) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kImNT * kImNB) return;
  const int ib = idx / kImNT, it = idx % kImNT;
  const double beta = kImBetaLo + (double)(kImBetaHi - kImBetaLo) * ib / (kImNB - 1);
  const double theta = 0.5 * kPiD * it / (kImNT - 1);
  const double h = kPiD / kSimpson;
  const double norm = 1.0 / (sqrt(2.0 * kPiD) * beta);
  double s = 0.0;
  for (int i = 0; i <= kSimpson; ++i) {
    const double to = -0.5 * kPiD + i * h;
    const double x = 0.5 * (theta + to);
    const double c = cos(to);
    const double f = norm * exp(-x * x / (2.0 * beta * beta)) * c * c;
    const double w = (i == 0 || i == kSimpson) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
    s += w * f;
  }
  s *= h / 3.0;
  im32[idx] = (float)s;
  im16[idx] = __double2half(s);
}

__global__ void k_bake_gauss(__half* gz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > kGzN) return;
  const double z = (double)kGzMax * i / kGzN;
  gz[i] = __double2half(exp(-0.5 * z * z));
}

}  // namespace

hr_status bake_tables(hr_ctx* ctx, float** im32, __half** im16, __half** gz16) {
  cudaStream_t st = ctx_stream(ctx);
  HR_TRY(dalloc(ctx, (void**)im32, sizeof(float) * kImNT * kImNB, "IM table"));
  HR_TRY(dalloc(ctx, (void**)im16, sizeof(__half) * kImNT * kImNB, "IM table fp16"));
  HR_TRY(dalloc(ctx, (void**)gz16, sizeof(__half) * (kGzN + 1), "Gaussian table"));
  const int n = kImNT * kImNB;
  k_bake_im<<<(n + 127) / 128, 128, 0, st>>>(*im32, *im16);
  HR_LAUNCHED(ctx);
  k_bake_gauss<<<(kGzN + 1 + 255) / 256, 256, 0, st>>>(*gz16);
  HR_LAUNCHED(ctx);
  return HR_OK;
}

}  // namespace hr
