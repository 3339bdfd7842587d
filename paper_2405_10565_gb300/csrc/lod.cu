// LoD selection (Section 5.1 step 5, Section 5.2 "Hair width calculation",
// "Dynamic LoD selection", Eq. 14).
//
// One thread per thick-hair cross-section projects the four corner points
// c +- a e1, c +- b e2 to pixels, takes the largest pairwise distance l_w and
// folds it into the per-(cluster, level) maximum with an atomicMax on the
// float's bit pattern (widths are >= 0 or +inf, whose bit patterns order like
// the values).  A second kernel applies the initial rule or Eq. (14).  Every
// floating-point operation is an explicit round-to-nearest FP32 intrinsic in a
// fixed order, so the widths (and hence the integer levels) do not depend on
// compiler contraction.
#include "common.cuh"

namespace hr {
namespace {

struct CamF {
  int kind;
  float pix, near_plane;
  float eye[3], right[3], up[3], fwd[3];
};

__device__ __forceinline__ float axis_dot(float rx, float ry, float rz, const float* a) {
  return __fadd_rn(__fadd_rn(__fmul_rn(rx, a[0]), __fmul_rn(ry, a[1])), __fmul_rn(rz, a[2]));
}

// pixel-plane coordinates (without the image-centre offset, which cancels in
// differences) and depth of a world point
__device__ __forceinline__ void project(const CamF& c, float px, float py, float pz, float* X,
                                        float* Y, float* Z) {
  const float rx = __fsub_rn(px, c.eye[0]), ry = __fsub_rn(py, c.eye[1]),
              rz = __fsub_rn(pz, c.eye[2]);
  const float xc = axis_dot(rx, ry, rz, c.right);
  const float yc = axis_dot(rx, ry, rz, c.up);
  const float zc = axis_dot(rx, ry, rz, c.fwd);
  if (c.kind == 1) {
    *X = __fmul_rn(__fdiv_rn(xc, zc), c.pix);
    *Y = __fmul_rn(__fdiv_rn(yc, zc), c.pix);
  } else {
    *X = __fmul_rn(xc, c.pix);
    *Y = __fmul_rn(yc, c.pix);
  }
  *Z = zc;
}

struct Levels {
  uint32_t n_levels;
  uint32_t off[16];
};

__global__ void k_widths(const float4* __restrict__ xsec, uint32_t E, uint32_t S, Levels lv,
                         CamF cam, uint32_t* wmax /* [C][n_levels] float bits */) {
  const uint64_t idx0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = idx0 < (uint64_t)E * (S + 1);
  const uint64_t idx = valid ? idx0 : 0;  // every lane stays for the warp reduction
  const uint32_t e = (uint32_t)(idx / (S + 1));
  uint32_t k = 0;
  while (k + 1 < lv.n_levels && e >= lv.off[k + 1]) ++k;
  const uint32_t cluster = (e - lv.off[k]) >> (2 * k);
  const float4 c = xsec[idx * 3], q1 = xsec[idx * 3 + 1], q2 = xsec[idx * 3 + 2];
  const float a = c.w, b = q1.w;
  const float ae[3] = {__fmul_rn(a, q1.x), __fmul_rn(a, q1.y), __fmul_rn(a, q1.z)};
  const float be[3] = {__fmul_rn(b, q2.x), __fmul_rn(b, q2.y), __fmul_rn(b, q2.z)};
  const float cc[3] = {c.x, c.y, c.z};
  float X[4], Y[4], Z[4];
  float p[3];
  for (int i = 0; i < 3; ++i) p[i] = __fadd_rn(cc[i], ae[i]);
  project(cam, p[0], p[1], p[2], &X[0], &Y[0], &Z[0]);
  for (int i = 0; i < 3; ++i) p[i] = __fsub_rn(cc[i], ae[i]);
  project(cam, p[0], p[1], p[2], &X[1], &Y[1], &Z[1]);
  for (int i = 0; i < 3; ++i) p[i] = __fadd_rn(cc[i], be[i]);
  project(cam, p[0], p[1], p[2], &X[2], &Y[2], &Z[2]);
  for (int i = 0; i < 3; ++i) p[i] = __fsub_rn(cc[i], be[i]);
  project(cam, p[0], p[1], p[2], &X[3], &Y[3], &Z[3]);
  float w = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = i + 1; j < 4; ++j) {
      const float dx = __fsub_rn(X[i], X[j]), dy = __fsub_rn(Y[i], Y[j]);
      const float d = __fsqrt_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)));
      w = fmaxf(w, d);
    }
  if (cam.kind == 1) {
    bool behind = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) behind |= !(Z[i] > cam.near_plane);
    if (behind) w = __int_as_float(0x7f800000);  // +inf
  }
  if (w != w) w = __int_as_float(0x7f800000);  // NaN (degenerate) counts as too wide
  // lanes of one (cluster, level) take their maximum first: one atomic each
  // an empty thick hair (a cluster of fewer than 4^k strands) has a = 0 and no width
  const bool live = valid && a > 0.f;
  const uint32_t slot = live ? cluster * lv.n_levels + k : 0xffffffffu;
  const uint32_t peers = __match_any_sync(0xffffffffu, slot);
  const uint32_t wm = __reduce_max_sync(peers, live ? __float_as_uint(w) : 0u);
  if (live && (threadIdx.x & 31) == (uint32_t)(__ffs(peers) - 1)) atomicMax(&wmax[slot], wm);
}

// Deferred selection with a hysteresis band (mode 2): a cluster refines only
// once its width exceeds eps by 10% and coarsens only once the coarser level
// is 10% under eps, so that widths that hover at eps under small motion keep
// their level and the BVH can be refit instead of rebuilt.
constexpr float kLodRefine = 1.1f;
constexpr float kLodCoarsen = 0.9f;

__global__ void k_rule(const uint32_t* __restrict__ wmax, uint32_t C, uint32_t L, float eps,
                       int mode, int bias, const uint8_t* __restrict__ prev, uint8_t* out) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const uint32_t* w = wmax + (size_t)c * L;
  int lvl;
  if (mode == 0) {
    // coarsest to finest: the first level whose maximum width is below eps
    lvl = (int)L;
    for (uint32_t l = 0; l < L; ++l)
      if (__uint_as_float(w[l]) < eps) {
        lvl = (int)l;
        break;
      }
  } else {
    // Eq. (14), cases in order; w_cur- = +inf at level 0; the strand level
    // only coarsens.  Mode 2 refines above eps (1 + h) and coarsens at or
    // below eps (1 - h), h = 0.1 (both products rounded to FP32 once).
    const float refine = mode == 2 ? __fmul_rn(eps, kLodRefine) : eps;
    const float coarsen = mode == 2 ? __fmul_rn(eps, kLodCoarsen) : eps;
    lvl = min((int)prev[c], (int)L);
    const float wcur = lvl < (int)L ? __uint_as_float(w[lvl]) : -__int_as_float(0x7f800000);
    const float wminus = lvl > 0 ? __uint_as_float(w[lvl - 1]) : __int_as_float(0x7f800000);
    if (lvl < (int)L && wcur > refine)
      lvl += 1;
    else if (wminus <= coarsen)
      lvl -= 1;
  }
  lvl = max(0, lvl - bias);
  out[c] = (uint8_t)lvl;
}

CamF make_cam(const hr_camera& c) {
  CamF f;
  f.kind = c.kind;
  f.pix = c.pix_scale;
  f.near_plane = c.near_plane;
  for (int i = 0; i < 3; ++i) {
    f.eye[i] = c.eye[i];
    f.right[i] = c.right[i];
    f.up[i] = c.up[i];
    f.fwd[i] = c.fwd[i];
  }
  return f;
}

hr_status compute_wmax(hr_ctx* ctx, hr_asset* a, const hr_camera* cam, uint32_t** wmax_out,
                       cudaStream_t st) {
  const uint32_t L = a->n_levels;
  uint32_t* wmax = nullptr;
  HR_TRY(scratch(ctx, 21, (size_t)a->C * L * 4, (void**)&wmax));
  HR_CUDA(ctx, cudaMemsetAsync(wmax, 0, (size_t)a->C * L * 4, st));
  Levels lv{};
  lv.n_levels = L;
  for (uint32_t k = 0; k <= L && k < 16; ++k) lv.off[k] = a->eth_offset[k];
  const uint64_t n = (uint64_t)a->E * (a->S + 1);
  if (n)
    k_widths<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a->xsec, a->E, a->S, lv,
                                                         make_cam(*cam), wmax);
  HR_LAUNCHED(ctx);
  *wmax_out = wmax;
  return HR_OK;
}

}  // namespace

hr_status lod_widths(hr_ctx* ctx, hr_asset* a, const hr_camera* cam, float* wcl_dev,
                     cudaStream_t st) {
  uint32_t* wmax = nullptr;
  HR_TRY(compute_wmax(ctx, a, cam, &wmax, st));
  HR_CUDA(ctx, cudaMemcpyAsync(wcl_dev, wmax, (size_t)a->C * a->n_levels * 4,
                               cudaMemcpyDeviceToDevice, st));
  return HR_OK;
}

hr_status lod_select(hr_ctx* ctx, hr_asset* a, const hr_camera* cam, float eps, int mode,
                     int bias, const uint8_t* prev_dev, uint8_t* out_dev, cudaStream_t st) {
  uint32_t* wmax = nullptr;
  HR_TRY(compute_wmax(ctx, a, cam, &wmax, st));
  k_rule<<<(a->C + 255) / 256, 256, 0, st>>>(wmax, a->C, a->n_levels, eps, mode, bias, prev_dev,
                                             out_dev);
  HR_LAUNCHED(ctx);
  return HR_OK;
}

}  // namespace hr
