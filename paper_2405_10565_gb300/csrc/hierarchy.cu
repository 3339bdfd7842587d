// Hair hierarchy (Section 5.1 steps 2-3) and primitive records.
//
//  * Strand segment records: every segment (s, k) of every strand becomes an
//    elliptic cylinder (Section 4 "elliptical cross-section"): semi-axes
//    a = r (1 - e^2)^-1/4, b = r (1 - e^2)^1/4 (area of the circle of radius r),
//    major axis e1 = cos(psi) b1 + sin(psi) b2 in the Duff et al. 2017 basis of
//    the segment direction.
//  * Clusters: deterministic Morton buckets of the strand roots (rank r of the
//    (code, id) order joins cluster floor(r C / N)), split 4^k ways at level k.
//  * Thick hairs: per cross-section k, mean centre, mean unit tangent, PCA of
//    the members' k-th points, the axis closest to the tangent dropped, e1 the
//    remaining axis with the larger eigenvalue, and semi-axes covering every
//    member (Section 5.1 step 3 "Cross-section fitting").  The centring sums,
//    the covariance and the eigenvector residual are double-word FP32 (the
//    FP64 rate of GB300 is 1/64 of its FP32 rate); near-degenerate sections
//    take a full FP64 eigen-solve.
//
// A primitive record is the affine map from world space to the cylinder's
// unit frame: rows (e1/a, -c0.e1/a), (e2/b, -c0.e2/b), (t/L, -c0.t/L); a ray
// hits the open cylinder where u^2 + v^2 = 1 with w in [0, 1].  Records are
// built in FP32 with compensated offsets (below); no FP64 outside the fit's
// near-degenerate path.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "dword.cuh"

namespace hr {
namespace {

struct d3 {
  double x, y, z;
};
__device__ __forceinline__ d3 mk(double x, double y, double z) { return {x, y, z}; }
__device__ __forceinline__ d3 operator-(d3 a, d3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ d3 operator*(d3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ d3 cross(d3 a, d3 b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ d3 ld3(float4 v) { return mk(v.x, v.y, v.z); }

// Double-word FP32 sum hi + lo: hi is the running rounded sum, lo collects
// every rounding error (Ogita, Rump and Oishi 2005, "Accurate sum and dot
// product", algorithm Sum2).  Over n terms the error is about n^2 2^-48 of
// the sum of magnitudes.
struct ffsum {
  float hi, lo;
};
__device__ __forceinline__ void ff_add(ffsum& s, float x, float x_lo) {
  float e;
  s.hi = two_sum(s.hi, x, e);
  s.lo = __fadd_rn(s.lo, __fadd_rn(e, x_lo));
}
// a[j] for j in {0, 1, 2} by selects (no local-memory indexing)
__device__ __forceinline__ float pick3(const float a[3], int j) {
  return j == 0 ? a[0] : (j == 1 ? a[1] : a[2]);
}

// Renormalise so |lo| <= ulp(hi) / 2 (keeps lo's own rounding small).
__device__ __forceinline__ void ff_renorm(ffsum& s) {
  float e;
  s.hi = two_sum(s.hi, s.lo, e);
  s.lo = e;
}
__device__ __forceinline__ double ff_value(const ffsum& s) { return (double)s.hi + (double)s.lo; }
__device__ __forceinline__ df df_of(const ffsum& s) {
  float e;
  const float h = two_sum(s.hi, s.lo, e);
  return {h, e};
}

// s += (xh + xl) (yh + yl), with the exact product xh yh (the FMA form of
// Dekker's TwoProduct) and the cross terms; xl yl (2^-48 relative) dropped.
__device__ __forceinline__ void ff_add_prod(ffsum& s, float xh, float xl, float yh, float yl) {
  const float p = __fmul_rn(xh, yh);
  const float pe = fmaf(xh, yh, -p);
  const float c = fmaf(xh, yl, __fmul_rn(xl, yh));
  ff_add(s, p, __fadd_rn(pe, c));
}

// Compensated dot product of FP32 3-vectors (Ogita, Rump and Oishi, Dot2):
// as accurate as if computed in twice the working precision, then rounded.
__device__ __forceinline__ float dot_comp(float3 a, float3 b) {
  ffsum s{0.f, 0.f};
  ff_add_prod(s, a.x, 0.f, b.x, 0.f);
  ff_add_prod(s, a.y, 0.f, b.y, 0.f);
  ff_add_prod(s, a.z, 0.f, b.z, 0.f);
  return __fadd_rn(s.hi, s.lo);
}

__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 mul3(float3 a, float s) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dotf(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 crossf(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// World -> unit elliptic cylinder rows and a conservative AABB of the
// segment c0 -> c1 with semi-axis a along e1 (unit, normal to the axis) and b
// along e2 = t x e1.  FP32 throughout: every row is within a few ulps of the
// correctly rounded value, and each offset is the compensated dot product of
// the stored row with c0, so the stored cylinder passes through c0 to within
// the offset's own rounding.
__device__ void write_prim(float4* xf, float4* box, float3 c0, float3 c1, float3 e1, float a, float b) {
  const float3 ax = sub3(c1, c0);
  const float L2 = dotf(ax, ax);
  if (!(L2 > 0.f)) {
    xf[0] = xf[1] = xf[2] = make_float4(0.f, 0.f, 0.f, 0.f);
    box[0] = make_float4(c0.x, c0.y, c0.z, 0.f);
    box[1] = box[0];
    return;
  }
  const float3 t = mul3(ax, 1.0f / sqrtf(L2));
  const float3 e2 = crossf(t, e1);
  const float ia = 1.0f / a, ib = 1.0f / b;
  const float3 r0 = mul3(e1, ia), r1 = mul3(e2, ib), r2 = mul3(ax, 1.0f / L2);
  xf[0] = make_float4(r0.x, r0.y, r0.z, -dot_comp(r0, c0));
  xf[1] = make_float4(r1.x, r1.y, r1.z, -dot_comp(r1, c0));
  xf[2] = make_float4(r2.x, r2.y, r2.z, -dot_comp(r2, c0));
  // half extents of the elliptic disc per axis, grown by 2e-6 relative (the
  // FP32 terms carry a few ulps); the corners are rounded outward
  const float ga = 1.000002f;
  const float hx = sqrtf(fmaf(a * e1.x, a * e1.x, (b * e2.x) * (b * e2.x))) * ga;
  const float hy = sqrtf(fmaf(a * e1.y, a * e1.y, (b * e2.y) * (b * e2.y))) * ga;
  const float hz = sqrtf(fmaf(a * e1.z, a * e1.z, (b * e2.z) * (b * e2.z))) * ga;
  box[0] = make_float4(__fsub_rd(fminf(c0.x, c1.x), hx), __fsub_rd(fminf(c0.y, c1.y), hy),
                       __fsub_rd(fminf(c0.z, c1.z), hz), 0.f);
  box[1] = make_float4(__fadd_ru(fmaxf(c0.x, c1.x), hx), __fadd_ru(fmaxf(c0.y, c1.y), hy),
                       __fadd_ru(fmaxf(c0.z, c1.z), hz), 0.f);
}

// Orthonormal basis around a unit vector (Duff, Burgess, Christensen, Hery,
// Kensler, Liani, Villemin 2017, "Building an orthonormal basis, revisited").
__device__ void duff_basis(d3 n, d3* b1, d3* b2) {
  const double sign = copysign(1.0, n.z);
  const double a = -1.0 / (sign + n.z);
  const double b = n.x * n.y * a;
  *b1 = mk(1.0 + sign * n.x * n.x * a, sign * b, -sign * n.x);
  *b2 = mk(b, sign + n.y * n.y * a, -n.y);
}
__device__ void duff_basis_f(float3 n, float3* b1, float3* b2) {
  const float sign = copysignf(1.0f, n.z);
  const float a = -1.0f / (sign + n.z);
  const float b = n.x * n.y * a;
  *b1 = make_float3(1.0f + sign * n.x * n.x * a, sign * b, -sign * n.x);
  *b2 = make_float3(b, sign + n.y * n.y * a, -n.y);
}

// Per strand: cos(psi), sin(psi) and the semi-axes a, b of its cross-section
// (equal area to the circle of radius r), so the segment kernel does no
// transcendental per segment.
__global__ void k_strand_shape(const float4* __restrict__ verts, const float2* __restrict__ shape,
                               uint32_t N, uint32_t S, float4* out) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const float r = verts[(size_t)s * (S + 1)].w;
  const float2 sh = shape[s];
  float sp, cp;
  sincosf(sh.y, &sp, &cp);
  const float q = sqrtf(sqrtf(fmaf(-sh.x, sh.x, 1.0f)));
  out[s] = make_float4(cp, sp, r / q, r * q);
}

__global__ void k_strand_prims(const float4* __restrict__ verts, const float4* __restrict__ sh4,
                               uint32_t N, uint32_t S, float4* xf, float4* box, float4* aux) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (uint64_t)N * S) return;
  const uint32_t s = (uint32_t)(idx / S), k = (uint32_t)(idx % S);
  const float4* P = verts + (size_t)s * (S + 1);
  const float4 v0 = __ldg(P + k), v1 = __ldg(P + k + 1);
  const float3 p0 = make_float3(v0.x, v0.y, v0.z), p1 = make_float3(v1.x, v1.y, v1.z);
  const float r = __ldg(&P[0].w);
  const float4 sh = __ldg(sh4 + s);
  const float3 ax = sub3(p1, p0);
  const float L2 = dotf(ax, ax);
  float3 e1 = make_float3(1.f, 0.f, 0.f);
  if (L2 > 0.f) {
    float3 b1, b2;
    duff_basis_f(mul3(ax, 1.0f / sqrtf(L2)), &b1, &b2);
    e1 = make_float3(fmaf(b1.x, sh.x, b2.x * sh.y), fmaf(b1.y, sh.x, b2.y * sh.y),
                     fmaf(b1.z, sh.x, b2.z * sh.y));
  }
  write_prim(xf + idx * 3, box + idx * 2, p0, p1, e1, sh.z, sh.w);
  aux[idx] = make_float4(__uint_as_float(s), 0.f, r, sh.z * sh.w);
}

// New strand positions in one pass: each block reads the vertices of
// `per_block` whole strands once, from device memory or from page-locked host
// memory mapped into the device's address space (so the transfer and the
// record build overlap), keeps them in shared memory, writes the asset's
// device copy, and builds every segment record of its strands exactly as
// k_strand_shape and k_strand_prims do.
__global__ void k_strand_update(const float4* __restrict__ src, float4* __restrict__ verts,
                                const float2* __restrict__ shape, uint32_t N, uint32_t S,
                                uint32_t per_block, float4* xf, float4* box, float4* aux) {
  extern __shared__ float4 sv[];  // per_block * (S + 1) vertices, then per_block shapes
  const uint32_t s0 = blockIdx.x * per_block;
  const uint32_t ns = min(per_block, N - s0);
  const uint32_t nv = ns * (S + 1);
  const size_t v0 = (size_t)s0 * (S + 1);
  for (uint32_t i = threadIdx.x; i < nv; i += blockDim.x) {
    const float4 v = src[v0 + i];
    sv[i] = v;
    verts[v0 + i] = v;
  }
  float4* ssh = sv + (size_t)per_block * (S + 1);
  __syncthreads();
  if (threadIdx.x < ns) {
    const float r = sv[threadIdx.x * (S + 1)].w;
    const float2 sh = shape[s0 + threadIdx.x];
    float sp, cp;
    sincosf(sh.y, &sp, &cp);
    const float q = sqrtf(sqrtf(fmaf(-sh.x, sh.x, 1.0f)));
    ssh[threadIdx.x] = make_float4(cp, sp, r / q, r * q);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < ns * S; i += blockDim.x) {
    const uint32_t ls = i / S, k = i % S;
    const float4* P = sv + ls * (S + 1);
    const float4 va = P[k], vb = P[k + 1];
    const float3 p0 = make_float3(va.x, va.y, va.z), p1 = make_float3(vb.x, vb.y, vb.z);
    const float r = P[0].w;
    const float4 sh = ssh[ls];
    const float3 ax = sub3(p1, p0);
    const float L2 = dotf(ax, ax);
    float3 e1 = make_float3(1.f, 0.f, 0.f);
    if (L2 > 0.f) {
      float3 b1, b2;
      duff_basis_f(mul3(ax, 1.0f / sqrtf(L2)), &b1, &b2);
      e1 = make_float3(fmaf(b1.x, sh.x, b2.x * sh.y), fmaf(b1.y, sh.x, b2.y * sh.y),
                       fmaf(b1.z, sh.x, b2.z * sh.y));
    }
    const size_t idx = (size_t)(s0 + ls) * S + k;
    write_prim(xf + idx * 3, box + idx * 2, p0, p1, e1, sh.z, sh.w);
    aux[idx] = make_float4(__uint_as_float(s0 + ls), 0.f, r, sh.z * sh.w);
  }
}

// ------------------------------------------------------------ Morton clusters


// bounds[0..2] = min (ordered bits), bounds[3..5] = max
__global__ void k_root_bounds(const float4* __restrict__ verts, uint32_t N, uint32_t S,
                              uint32_t* bounds) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0, 0, 0};
  if (s < N) {
    const float4 p = verts[(size_t)s * (S + 1)];
    const float c[3] = {p.x, p.y, p.z};
    for (int i = 0; i < 3; ++i) lo[i] = hi[i] = ordered_bits(c[i]);
  }
  for (int i = 0; i < 3; ++i) {
    for (int o = 16; o; o >>= 1) {
      lo[i] = min(lo[i], __shfl_xor_sync(0xffffffffu, lo[i], o));
      hi[i] = max(hi[i], __shfl_xor_sync(0xffffffffu, hi[i], o));
    }
  }
  // then across the block's warps: six atomics per block
  __shared__ uint32_t s_b[8][6];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
    for (int i = 0; i < 3; ++i) {
      s_b[wid][i] = lo[i];
      s_b[wid][3 + i] = hi[i];
    }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int i = threadIdx.x;
    uint32_t v = s_b[0][i];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = i < 3 ? min(v, s_b[w][i]) : max(v, s_b[w][i]);
    if (i < 3) atomicMin(&bounds[i], v); else atomicMax(&bounds[i], v);
  }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  // bits 0..9 of v to bits 0, 3, 6, ..., 27
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Root quantisation q = min(1023, floor((p - lo) * (1024 / e))) in the roots'
// bounding cube (lo its low corner, e the largest extent), every operation
// rounded to FP32 in this order; code = x bits at 3i+2, y at 3i+1, z at 3i.
__global__ void k_root_morton(const float4* __restrict__ verts, uint32_t N, uint32_t S,
                              const uint32_t* __restrict__ bounds, uint32_t* keys,
                              uint32_t* vals) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const float4 p = verts[(size_t)s * (S + 1)];
  const float c[3] = {p.x, p.y, p.z};
  float ext = 0.f;
  for (int i = 0; i < 3; ++i)
    ext = fmaxf(ext, __fsub_rn(from_ordered(bounds[3 + i]), from_ordered(bounds[i])));
  const float scale = ext > 0.f ? __fdiv_rn(1024.0f, ext) : 0.f;
  uint32_t q[3];
  for (int i = 0; i < 3; ++i) {
    const float lo = from_ordered(bounds[i]);
    const float v = __fmul_rn(__fsub_rn(c[i], lo), scale);
    const int qi = (int)floorf(v);
    q[i] = (uint32_t)min(1023, max(0, qi));
  }
  keys[s] = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
  vals[s] = s;
}

__global__ void k_assign_clusters(const uint32_t* __restrict__ order, uint32_t N, uint32_t C,
                                  uint32_t* cluster_of) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  cluster_of[order[r]] = (uint32_t)(((uint64_t)r * C) / N);
}

__global__ void k_cluster_first(uint32_t N, uint32_t C, uint32_t* first) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > C) return;
  first[c] = (uint32_t)(((uint64_t)c * N + C - 1) / C);  // ceil(c N / C)
}

// *flag |= x != y over n words
__global__ void k_words_differ(const uint32_t* __restrict__ x, const uint32_t* __restrict__ y,
                               uint32_t n, uint32_t* flag) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && x[i] != y[i]) *flag = 1u;
}

// cluster_of of the strands of cluster c (ranks cl_first[c] .. cl_first[c+1]-1)
__global__ void k_cluster_of_from_first(const uint32_t* __restrict__ order,
                                        const uint32_t* __restrict__ cl_first,
                                        uint32_t* cluster_of) {
  const uint32_t c = blockIdx.x;
  for (uint32_t r = cl_first[c] + threadIdx.x; r < cl_first[c + 1]; r += blockDim.x)
    cluster_of[order[r]] = c;
}

struct LevelInfo {
  uint32_t n_levels;
  uint32_t off[16];  // first thick-hair index of each level; off[n_levels] = E
};

// Member rank range of thick hair e: level k, cluster c, sub-bucket j; the
// members are the ranks i-in-cluster with floor(i 4^k / m) == j.
__device__ __forceinline__ void eth_members(const LevelInfo& li, const uint32_t* cl_first,
                                            uint32_t e, uint32_t* first, uint32_t* count,
                                            uint32_t* cluster, uint32_t* level) {
  uint32_t k = 0;
  while (k + 1 < li.n_levels && e >= li.off[k + 1]) ++k;
  const uint32_t sub_n = 1u << (2 * k);
  const uint32_t loc = e - li.off[k];
  const uint32_t c = loc / sub_n, j = loc % sub_n;
  const uint64_t m = cl_first[c + 1] - cl_first[c];
  const uint64_t lo = ((uint64_t)j * m + sub_n - 1) / sub_n;
  const uint64_t hi = ((uint64_t)(j + 1) * m + sub_n - 1) / sub_n;
  *first = cl_first[c] + (uint32_t)lo;
  *count = (uint32_t)(hi - lo);
  *cluster = c;
  *level = k;
}

// ------------------------------------------------------------ ellipse fit

// Cyclic Jacobi sweeps on a symmetric 3x3 matrix, accumulating the rotations
// into V (which must hold an orthonormal basis on entry).  On return A's
// diagonal holds the eigenvalues and V's columns the vectors.  T is float
// (a cheap first guess) or double (the refinement that sets the accuracy).
template <typename T>
__device__ void jacobi_sweeps(T A[3][3], T V[3][3], int max_sweeps, T rel_tol) {
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    const T off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const T diag = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= rel_tol * diag || off == T(0)) break;
    for (int p = 0; p < 2; ++p) {
      for (int q = p + 1; q < 3; ++q) {
        const T apq = A[p][q];
        if (apq == T(0)) continue;
        const T th = (A[q][q] - A[p][p]) / (T(2) * apq);
        const T t = (th >= T(0) ? T(1) : T(-1)) / (fabs(th) + sqrt(th * th + T(1)));
        const T c = T(1) / sqrt(t * t + T(1)), s = t * c;
        // A <- J^T A J with J the rotation in the (p, q) plane
        for (int k = 0; k < 3; ++k) {
          const T akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {
          const T apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          const T vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
    }
  }
}

// 1/g for a double g whose magnitude lies in [1e-30, 1e30]: the FP32
// reciprocal refined by one Newton-Raphson step r (2 - g r) in FP64, which
// squares its relative error (~6e-8 -> ~4e-15).
__device__ __forceinline__ double recip_nr(double g) {
  const double r = (double)(1.0f / (float)g);
  return r * fma(-g, r, 2.0);
}
// 1/sqrt(x) for x in [1e-30, 1e30]: the FP32 estimate refined by one Newton
// step y (3 - x y^2) / 2 in FP64 (relative error ~1.5 d^2 for an estimate
// error d of a few 1e-7).
__device__ __forceinline__ double rsqrt_nr(double x) {
  const double y = (double)rsqrtf((float)x);
  return y * fma(-0.5 * x * y, y, 1.5);
}
// Normalise a vector whose length is already 1 to about 1e-6 (the columns of
// an FP32 rotation): 1/sqrt(1 + h) = 1 - h/2 + 3h^2/8 - ..., whose first
// omitted term is below 0.32 |h|^3 (< 4e-19 here); otherwise an exact division.
__device__ __forceinline__ d3 normalize_near_unit(d3 v) {
  const double h = dot(v, v) - 1.0;
  if (fabs(h) < 1e-6) return v * fma(h, fma(0.375, h, -0.5), 1.0);
  return v * (1.0 / sqrt(h + 1.0));
}

// FP64 refinement of an FP32 eigenbasis Vf of the symmetric 3x3 covariance C
// (used where the eigenvalues are too close for the FP32 basis): the basis is
// re-orthonormalised in FP64, C is rotated into it in FP64, and a first-order
// FP64 correction of the basis (or, for nearly equal eigenvalues, FP64 Jacobi
// sweeps) finishes the job.  On return A's diagonal holds the eigenvalues and
// V's columns the vectors.
__device__ void eigen3_refine(const double C[3][3], const float Vf[3][3], double A[3][3],
                              double V[3][3]) {
  // FP64 Gram-Schmidt of the FP32 basis
  const d3 v0 = normalize_near_unit(mk(Vf[0][0], Vf[1][0], Vf[2][0]));
  d3 v1 = mk(Vf[0][1], Vf[1][1], Vf[2][1]);
  v1 = normalize_near_unit(v1 - v0 * dot(v1, v0));
  const d3 v2 = cross(v0, v1);
  const d3 cols[3] = {v0, v1, v2};
  for (int j = 0; j < 3; ++j) {
    V[0][j] = cols[j].x;
    V[1][j] = cols[j].y;
    V[2][j] = cols[j].z;
  }
  // A = V^T C V (symmetric: the upper triangle is computed and mirrored)
  d3 CV[3];
  for (int j = 0; j < 3; ++j)
    CV[j] = mk(C[0][0] * cols[j].x + C[0][1] * cols[j].y + C[0][2] * cols[j].z,
               C[1][0] * cols[j].x + C[1][1] * cols[j].y + C[1][2] * cols[j].z,
               C[2][0] * cols[j].x + C[2][1] * cols[j].y + C[2][2] * cols[j].z);
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) A[i][j] = A[j][i] = dot(cols[i], CV[j]);
  // With well-separated diagonal entries the first-order correction
  // v_i += sum_j A_ji / (A_ii - A_jj) v_j leaves an error of (off / gap)^2;
  // otherwise finish with FP64 Jacobi sweeps.
  const double d0 = A[0][0], d1 = A[1][1], d2 = A[2][2];
  const double g01 = d0 - d1, g02 = d0 - d2, g12 = d1 - d2;
  const double scale = fmax(fabs(d0), fmax(fabs(d1), fabs(d2)));
  const double off = fmax(fabs(A[0][1]), fmax(fabs(A[0][2]), fabs(A[1][2])));
  const double gap = fmin(fabs(g01), fmin(fabs(g02), fabs(g12)));
  if (scale > 1e-27 && scale < 1e27 && gap > 1e-3 * scale && off < 1e-5 * gap) {
    const double c01 = A[0][1] * recip_nr(g01), c02 = A[0][2] * recip_nr(g02),
                 c12 = A[1][2] * recip_nr(g12);
    double W[3][3];
    for (int r = 0; r < 3; ++r) {
      W[r][0] = V[r][0] + c01 * V[r][1] + c02 * V[r][2];
      W[r][1] = V[r][1] - c01 * V[r][0] + c12 * V[r][2];
      W[r][2] = V[r][2] - c02 * V[r][0] - c12 * V[r][1];
    }
    for (int r = 0; r < 3; ++r)
      for (int j = 0; j < 3; ++j) V[r][j] = W[r][j];
    A[0][1] = A[1][0] = A[0][2] = A[2][0] = A[1][2] = A[2][1] = 0.0;
  } else {
    // stop at an off-diagonal of ~3e-14 relative: the axes are then exact to
    // far below the FP32 records they end up in
    jacobi_sweeps<double>(A, V, 16, 1e-27);
  }
}

// e1 of a cross-section from the FP64 eigen-decomposition (the careful path:
// nearly equal eigenvalues, a near tie for the dropped axis, a covariance out
// of FP32 range).  The eigenvector most aligned with the tangent t is
// dropped and e1 is the remaining one with the larger eigenvalue; when the
// two kept eigenvalues are equal, e1 points to the member farthest from the
// centre in the plane normal to t (first in rank order), else along the Duff
// basis vector b1 of t.
__device__ d3 major_axis_fp64(const double C[3][3], const float Vf[3][3], const d3 t,
                              const d3 ctr, const float4* __restrict__ verts, uint32_t S,
                              uint32_t k, const uint32_t* __restrict__ order, uint32_t first,
                              uint32_t cnt) {
  double A[3][3], V[3][3];
  eigen3_refine(C, Vf, A, V);
  // ascending eigenvalues (stable for ties)
  int ord[3] = {0, 1, 2};
  for (int i = 1; i < 3; ++i)
    for (int j = i; j > 0 && A[ord[j]][ord[j]] < A[ord[j - 1]][ord[j - 1]]; --j) {
      const int tmp = ord[j];
      ord[j] = ord[j - 1];
      ord[j - 1] = tmp;
    }
  int drop = 0;
  double best = -1.0;
  for (int i = 0; i < 3; ++i) {
    const int col = ord[i];
    const double dd = fabs(V[0][col] * t.x + V[1][col] * t.y + V[2][col] * t.z);
    if (dd > best) {
      best = dd;
      drop = i;
    }
  }
  const int keep = ord[drop == 2 ? 1 : 2], keep0 = ord[drop == 0 ? 1 : 0];
  d3 e1 = mk(V[0][keep], V[1][keep], V[2][keep]);
  const double lmax = A[ord[2]][ord[2]];
  if (A[keep][keep] - A[keep0][keep0] <= 1e-9 * lmax || !(lmax > 0.0)) {
    double best_d2 = 0.0;
    d3 far = mk(0, 0, 0);
    for (uint32_t i = 0; i < cnt; ++i) {
      const d3 q = ld3(verts[(size_t)order[first + i] * (S + 1) + k]) - ctr;
      const d3 qp = q - t * dot(q, t);
      const double d2 = dot(qp, qp);
      if (d2 > best_d2) {
        best_d2 = d2;
        far = qp;
      }
    }
    if (best_d2 > 0.0) {
      e1 = far * (1.0 / sqrt(best_d2));
    } else {
      d3 b1, b2;
      duff_basis(t, &b1, &b2);
      e1 = b1;
    }
  }
  return e1;
}

// One thread per (thick hair, cross-section).  Writes the FP32 cross-section
// record (c, a) (e1, b) (e2, 0) that the LoD widths and the thick-hair
// segments are built from.
//  * Centring sums: the members' offsets d = p - p0 from the first member are
//    exact FP32 pairs (TwoSum) and their first and second moments double-word
//    FP32 sums (exact products, every rounding error kept, renormalised every
//    64 members): within ~2^-48 of exact, like FP64 sums, at a fraction of
//    their cost.
//  * Mean and covariance: double-word FP32 (about 2^-44 relative).
//    Eigenbasis: cyclic Jacobi in FP32 on the trace-normalised covariance;
//    the kept axis e1 is then corrected to first order from its double-word
//    residual r = C v - (v.Cv) v, which is where the conditioning needs more
//    than FP32 (the residual is a small difference of large terms).  The
//    FP32 basis is off by e ~ 3e-7 / gap and the correction
//    leaves ~e^2, so it is taken while every gap between e1's eigenvalue and
//    the others is at least 1e-2 of the largest (e^2 < 1e-9);
//    closer eigenvalues, a near tie for the dropped axis and covariances out
//    of FP32 range take the full FP64 solve above.
//  * Unit tangents (which only pick the dropped axis and orient e1, e2) and
//    the member projections for the semi-axes: FP32.
// 64 registers (8 blocks of 128 per SM): more warps in flight hide the FP64
// pipe's latency better than the spills of the rare full-FP64 path cost.
__global__ void __launch_bounds__(128, 8) k_fit_cross_sections(const float4* __restrict__ verts, uint32_t S,
                                     const uint32_t* __restrict__ order,
                                     const uint32_t* __restrict__ cl_first, LevelInfo li,
                                     uint32_t E, float4* xsec) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (uint64_t)E * (S + 1)) return;
  const uint32_t e = (uint32_t)(idx / (S + 1)), k = (uint32_t)(idx % (S + 1));
  uint32_t first, cnt, c, lv;
  eth_members(li, cl_first, e, &first, &cnt, &c, &lv);
  if (cnt == 0) {  // an empty thick hair (a cluster of fewer than 4^k strands): a = b = 0
    float4* o = xsec + idx * 3;
    o[0] = o[1] = o[2] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const uint32_t k0 = k > 0 ? k - 1 : 0, k1 = k < S ? k + 1 : S;
  const float4 q0 = __ldg(verts + (size_t)__ldg(order + first) * (S + 1) + k);
  const float p0x = q0.x, p0y = q0.y, p0z = q0.z;
  // pass 1: sums of the offsets from the first member and of the unit tangents
  ffsum fx{0.f, 0.f}, fy{0.f, 0.f}, fz{0.f, 0.f};
  ffsum fxx{0.f, 0.f}, fxy{0.f, 0.f}, fxz{0.f, 0.f}, fyy{0.f, 0.f}, fyz{0.f, 0.f}, fzz{0.f, 0.f};
  float tx = 0.f, ty = 0.f, tz = 0.f;
  for (uint32_t i = 0; i < cnt; ++i) {
    const float4* P = verts + (size_t)__ldg(order + first + i) * (S + 1);
    const float4 pk = __ldg(P + k), pa = __ldg(P + k0), pb = __ldg(P + k1);
    float dxl, dyl, dzl;
    const float dx = two_sum(pk.x, -p0x, dxl), dy = two_sum(pk.y, -p0y, dyl),
                dz = two_sum(pk.z, -p0z, dzl);
    ff_add(fx, dx, dxl);
    ff_add(fy, dy, dyl);
    ff_add(fz, dz, dzl);
    ff_add_prod(fxx, dx, dxl, dx, dxl);
    ff_add_prod(fxy, dx, dxl, dy, dyl);
    ff_add_prod(fxz, dx, dxl, dz, dzl);
    ff_add_prod(fyy, dy, dyl, dy, dyl);
    ff_add_prod(fyz, dy, dyl, dz, dzl);
    ff_add_prod(fzz, dz, dzl, dz, dzl);
    const float gx = pb.x - pa.x, gy = pb.y - pa.y, gz = pb.z - pa.z;
    const float ig = rsqrtf(gx * gx + gy * gy + gz * gz);
    tx += gx * ig;
    ty += gy * ig;
    tz += gz * ig;
    if ((i & 63u) == 63u) {
      ff_renorm(fx); ff_renorm(fy); ff_renorm(fz);
      ff_renorm(fxx); ff_renorm(fxy); ff_renorm(fxz);
      ff_renorm(fyy); ff_renorm(fyz); ff_renorm(fzz);
    }
  }
  // mean offset and covariance in double-word FP32
  const float fn = (float)cnt, rn = 1.0f / fn;
  const df inv_n = {rn, fmaf(-fn, rn, 1.0f) * rn};
  const df mx = df_mul(df_of(fx), inv_n), my = df_mul(df_of(fy), inv_n), mz = df_mul(df_of(fz), inv_n);
  const df m3[3] = {mx, my, mz};
  const df s3[3][3] = {{df_of(fxx), df_of(fxy), df_of(fxz)},
                       {df_of(fxy), df_of(fyy), df_of(fyz)},
                       {df_of(fxz), df_of(fyz), df_of(fzz)}};
  df C[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      C[i][j] = df_sub(df_mul(s3[i][j], inv_n), df_mul(m3[i], m3[j]));
      C[j][i] = C[i][j];
    }
  const float itn = rsqrtf(tx * tx + ty * ty + tz * tz);
  const float tfx = tx * itn, tfy = ty * itn, tfz = tz * itn;
  // FP32 Jacobi on the trace-normalised covariance
  const float tr = df_float(C[0][0]) + df_float(C[1][1]) + df_float(C[2][2]);
  const bool seed = tr > 1e-30f && tr < 1e30f;
  const float inv_tr = seed ? 1.0f / tr : 0.f;
  float Af[3][3], Vf[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Af[i][j] = df_float(C[i][j]) * inv_tr;
      Vf[i][j] = (i == j) ? 1.f : 0.f;
    }
  if (seed) jacobi_sweeps<float>(Af, Vf, 10, 1e-13f);
  // FP32 choice of the dropped and kept axes (as in the FP64 path); columns
  // are picked with selects so the basis stays in registers
  const float lam3[3] = {Af[0][0], Af[1][1], Af[2][2]};
  int o0 = 0, o1 = 1, o2 = 2;  // ascending eigenvalue order (stable)
  if (pick3(lam3, o1) < pick3(lam3, o0)) { const int tt = o0; o0 = o1; o1 = tt; }
  if (pick3(lam3, o2) < pick3(lam3, o1)) { const int tt = o1; o1 = o2; o2 = tt; }
  if (pick3(lam3, o1) < pick3(lam3, o0)) { const int tt = o0; o0 = o1; o1 = tt; }
  float dd3[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) dd3[j] = fabsf(Vf[0][j] * tfx + Vf[1][j] * tfy + Vf[2][j] * tfz);
  const float da = pick3(dd3, o0), db = pick3(dd3, o1), dc = pick3(dd3, o2);
  int drop = 0;
  float best = da, second = -1.f;
  if (db > best) { second = best; best = db; drop = 1; } else { second = db; }
  if (dc > best) { second = best; best = dc; drop = 2; } else if (dc > second) { second = dc; }
  const int keep = drop == 2 ? o1 : o2, keep0 = drop == 0 ? o1 : o0;
  const int dcol = drop == 0 ? o0 : (drop == 1 ? o1 : o2);
  const float lk = pick3(lam3, keep), lmax = pick3(lam3, o2);
  const float ga = lk - pick3(lam3, keep0), gb = lk - pick3(lam3, dcol);
  float e1x, e1y, e1z;
  if (seed && lmax > 0.f && fminf(ga, fabsf(gb)) >= 1e-2f * lmax && best - second > 1e-4f) {
    // double-word residual of the FP32 vector v, then
    // v += sum_j (v_j . r) / (l_k - l_j) v_j
    const float vx = pick3(Vf[0], keep), vy = pick3(Vf[1], keep), vz = pick3(Vf[2], keep);
    const float ax = pick3(Vf[0], keep0), ay = pick3(Vf[1], keep0), az = pick3(Vf[2], keep0);
    const float bx = pick3(Vf[0], dcol), by = pick3(Vf[1], dcol), bz = pick3(Vf[2], dcol);
    df w[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      w[i] = df_add(df_add(df_mul(C[i][0], vx), df_mul(C[i][1], vy)), df_mul(C[i][2], vz));
    const df lam = df_add(df_add(df_mul(w[0], vx), df_mul(w[1], vy)), df_mul(w[2], vz));
    const float rx = df_float(df_sub(w[0], df_mul(lam, vx))) * inv_tr;
    const float ry = df_float(df_sub(w[1], df_mul(lam, vy))) * inv_tr;
    const float rz = df_float(df_sub(w[2], df_mul(lam, vz))) * inv_tr;
    const float ca = (ax * rx + ay * ry + az * rz) / ga;
    const float cb = (bx * rx + by * ry + bz * rz) / gb;
    e1x = vx + ca * ax + cb * bx;
    e1y = vy + ca * ay + cb * by;
    e1z = vz + ca * az + cb * bz;
  } else {
    double Cd[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Cd[i][j] = df_double(C[i][j]);
    const d3 ctr = mk(p0x + df_double(mx), p0y + df_double(my), p0z + df_double(mz));
    const d3 e1 = major_axis_fp64(Cd, Vf, mk(tfx, tfy, tfz), ctr, verts, S, k, order, first, cnt);
    e1x = (float)e1.x;
    e1y = (float)e1.y;
    e1z = (float)e1.z;
  }
  // e1 made normal to t and unit, e2 = t x e1
  {
    const float d = e1x * tfx + e1y * tfy + e1z * tfz;
    e1x -= d * tfx;
    e1y -= d * tfy;
    e1z -= d * tfz;
    const float in1 = 1.0f / sqrtf(e1x * e1x + e1y * e1y + e1z * e1z);
    e1x *= in1;
    e1y *= in1;
    e1z *= in1;
  }
  const float e2x = tfy * e1z - tfz * e1y, e2y = tfz * e1x - tfx * e1z, e2z = tfx * e1y - tfy * e1x;
  // pass 2: semi-axes; pass 3: the coverage scale (one square root).  A
  // member's offset from the centre is (p - p0) - (c - p0): the first
  // difference is rounded once in FP32 (exact when the two floats are within
  // a factor of two), the second term is the mean shift rounded once, so
  // the projections run in FP32 (the results are stored as FP32 anyway).
  const float mfx = df_float(mx), mfy = df_float(my), mfz = df_float(mz);
  float af = 0.f, bf = 0.f;
  for (uint32_t i = 0; i < cnt; ++i) {
    const float4* P = verts + (size_t)__ldg(order + first + i) * (S + 1);
    const float4 pk = __ldg(P + k);
    const float qx = (pk.x - p0x) - mfx, qy = (pk.y - p0y) - mfy, qz = (pk.z - p0z) - mfz;
    const float r = __ldg(&P[0].w);  // the strand's radius (root vertex)
    af = fmaxf(af, fabsf(fmaf(qx, e1x, fmaf(qy, e1y, qz * e1z))) + r);
    bf = fmaxf(bf, fabsf(fmaf(qx, e2x, fmaf(qy, e2y, qz * e2z))) + r);
  }
  const float ia = 1.0f / af, ib = 1.0f / bf;
  float s2 = 0.f;
  for (uint32_t i = 0; i < cnt; ++i) {
    const float4 pk = __ldg(verts + (size_t)__ldg(order + first + i) * (S + 1) + k);
    const float qx = (pk.x - p0x) - mfx, qy = (pk.y - p0y) - mfy, qz = (pk.z - p0z) - mfz;
    const float u = fmaf(qx, e1x, fmaf(qy, e1y, qz * e1z)) * ia;
    const float v = fmaf(qx, e2x, fmaf(qy, e2y, qz * e2z)) * ib;
    s2 = fmaxf(s2, fmaf(u, u, v * v));
  }
  float a = af, b = bf;
  if (s2 > 1.f) {
    const float sc = sqrtf(s2);
    a = af * sc;
    b = bf * sc;
  }
  float4* o = xsec + idx * 3;
  // centre p0 + mean offset, rounded once from double-word FP32
  const df cx = df_add({p0x, 0.f}, mx), cy = df_add({p0y, 0.f}, my), cz = df_add({p0z, 0.f}, mz);
  o[0] = make_float4(df_float(cx), df_float(cy), df_float(cz), a);
  o[1] = make_float4(e1x, e1y, e1z, b);
  o[2] = make_float4(e2x, e2y, e2z, 0.f);
}

// Mean member material and radius of every thick hair (double-word FP32
// sums, so the mean is the correctly rounded one to within an ulp).
__global__ void k_eth_material(const float4* __restrict__ verts, uint32_t N, uint32_t S,
                               const uint32_t* __restrict__ order,
                               const uint32_t* __restrict__ cl_first, LevelInfo li, uint32_t E,
                               float* mat, float* eth_r) {
  // one thread per (thick hair, material float); the last float is the radius
  constexpr uint32_t F = HR_MAT_FLOATS + 1;
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (uint64_t)E * F) return;
  const uint32_t e = (uint32_t)(idx / F), j = (uint32_t)(idx % F);
  uint32_t first, cnt, c, lv;
  eth_members(li, cl_first, e, &first, &cnt, &c, &lv);
  ffsum acc{0.f, 0.f};
  for (uint32_t i = 0; i < cnt; ++i) {
    const uint32_t s = __ldg(order + first + i);
    ff_add(acc, j < HR_MAT_FLOATS ? mat[(size_t)s * HR_MAT_FLOATS + j] : __ldg(&verts[(size_t)s * (S + 1)].w),
           0.f);
  }
  const float mean = cnt ? __fadd_rn(acc.hi, acc.lo) / (float)cnt : 0.f;
  if (j < HR_MAT_FLOATS)
    mat[(size_t)(N + e) * HR_MAT_FLOATS + j] = mean;
  else
    eth_r[e] = mean;
}

// Thick-hair segment (e, k): axis c_k -> c_{k+1}, e1 = e1_k made orthogonal to
// the axis, semi-axes the larger of the two cross-sections'.
__global__ void k_eth_prims(const float4* __restrict__ xsec, uint32_t N, uint32_t S, uint32_t E,
                            const uint32_t* __restrict__ cl_first, LevelInfo li,
                            const float* __restrict__ eth_r, float4* xf, float4* box,
                            float4* aux) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (uint64_t)E * S) return;
  const uint32_t e = (uint32_t)(idx / S), k = (uint32_t)(idx % S);
  const float4* x0 = xsec + ((size_t)e * (S + 1) + k) * 3;
  const float4 q0 = __ldg(x0), q1 = __ldg(x0 + 1), r0 = __ldg(x0 + 3), r1 = __ldg(x0 + 4);
  const float3 c0 = make_float3(q0.x, q0.y, q0.z), c1 = make_float3(r0.x, r0.y, r0.z);
  const float3 ax = sub3(c1, c0);
  const float L2 = dotf(ax, ax);
  float3 e1 = make_float3(q1.x, q1.y, q1.z);
  if (L2 > 0.f) {
    const float3 t = mul3(ax, 1.0f / sqrtf(L2));
    e1 = sub3(e1, mul3(t, dotf(e1, t)));
    e1 = mul3(e1, 1.0f / sqrtf(dotf(e1, e1)));
  }
  const float a = fmaxf(q0.w, r0.w), b = fmaxf(q1.w, r1.w);
  const uint64_t p = (uint64_t)N * S + idx;
  uint32_t first, cnt, c, lv;
  eth_members(li, cl_first, e, &first, &cnt, &c, &lv);
  if (cnt == 0) {  // empty thick hair: never active; records left inert
    xf[p * 3] = xf[p * 3 + 1] = xf[p * 3 + 2] = make_float4(0.f, 0.f, 0.f, 0.f);
    box[p * 2] = box[p * 2 + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
    aux[p] = make_float4(__uint_as_float(N + e), 0.f, 0.f, 0.f);
    return;
  }
  write_prim(xf + p * 3, box + p * 2, c0, c1, e1, a, b);
  aux[p] = make_float4(__uint_as_float(N + e), (float)cnt, eth_r[e], a * b);
}

// Scene bounds over all primitive boxes (ordered-bit atomics).
__global__ void k_prim_bounds(const float4* __restrict__ box, uint64_t n, uint32_t* bounds) {
  uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0, 0, 0};
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const float4 l = box[2 * i], h = box[2 * i + 1];
    lo[0] = min(lo[0], ordered_bits(l.x));
    lo[1] = min(lo[1], ordered_bits(l.y));
    lo[2] = min(lo[2], ordered_bits(l.z));
    hi[0] = max(hi[0], ordered_bits(h.x));
    hi[1] = max(hi[1], ordered_bits(h.y));
    hi[2] = max(hi[2], ordered_bits(h.z));
  }
  for (int i = 0; i < 3; ++i) {
    for (int o = 16; o; o >>= 1) {
      lo[i] = min(lo[i], __shfl_xor_sync(0xffffffffu, lo[i], o));
      hi[i] = max(hi[i], __shfl_xor_sync(0xffffffffu, hi[i], o));
    }
  }
  if ((threadIdx.x & 31) == 0)
    for (int i = 0; i < 3; ++i) {
      atomicMin(&bounds[i], lo[i]);
      atomicMax(&bounds[3 + i], hi[i]);
    }
}

__global__ void k_init_bounds(uint32_t* bounds) {
  if (threadIdx.x < 3) bounds[threadIdx.x] = 0xffffffffu;
  else if (threadIdx.x < 6) bounds[threadIdx.x] = 0u;
}

// Bounds of the first n primitive boxes into a->d_bounds (ordered float
// bits: lo xyz, hi xyz), on the stream; nothing is read back.
hr_status scene_bounds(hr_ctx* ctx, hr_asset* a, uint64_t n, cudaStream_t st = nullptr) {
  if (!st) st = ctx_stream(ctx);
  k_init_bounds<<<1, 32, 0, st>>>(a->d_bounds);
  HR_LAUNCHED(ctx);
  const int blocks = (int)std::min<uint64_t>((n + 255) / 256, 152 * 8);
  k_prim_bounds<<<std::max(1, blocks), 256, 0, st>>>(a->prim_box, n, a->d_bounds);
  HR_LAUNCHED(ctx);
  return HR_OK;
}

}  // namespace

hr_status build_strand_prims(hr_ctx* ctx, hr_asset* a) {
  const uint64_t n = (uint64_t)a->N * a->S;
  a->n_prims_total = (uint32_t)n;
  HR_TRY(dalloc(ctx, (void**)&a->prim_xf, n * 3 * sizeof(float4), "strand records"));
  HR_TRY(dalloc(ctx, (void**)&a->prim_box, n * 2 * sizeof(float4), "strand boxes"));
  HR_TRY(dalloc(ctx, (void**)&a->prim_aux, n * sizeof(float4), "strand aux"));
  HR_TRY(dalloc(ctx, (void**)&a->d_bounds, 8 * sizeof(uint32_t), "scene bounds"));
  a->bytes += n * 6 * sizeof(float4);
  return refresh_strand_prims(ctx, a);
}

// Strand segment records and scene bounds from the current vertices, into
// the asset's existing arrays (the first N * S records).
hr_status update_strands(hr_ctx* ctx, hr_asset* a, const float4* src_dev, cudaStream_t st) {
  if (!st) st = ctx_stream(ctx);
  const uint32_t S1 = a->S + 1;
  const uint32_t per_block = std::min<uint32_t>(256u, kUpdateMaxVerts / S1);
  const size_t smem = ((size_t)per_block * S1 + per_block) * sizeof(float4);
  const uint32_t blocks = (a->N + per_block - 1) / per_block;
  k_strand_update<<<blocks, 256, smem, st>>>(src_dev, a->verts, a->shape, a->N, a->S, per_block,
                                             a->prim_xf, a->prim_box, a->prim_aux);
  HR_LAUNCHED(ctx);
  return scene_bounds(ctx, a, (uint64_t)a->N * a->S, st);
}

hr_status refresh_strand_prims(hr_ctx* ctx, hr_asset* a) {
  cudaStream_t st = ctx_stream(ctx);
  const uint64_t n = (uint64_t)a->N * a->S;
  float4* sh4 = nullptr;
  HR_TRY(scratch(ctx, 6, (size_t)a->N * sizeof(float4), (void**)&sh4));
  k_strand_shape<<<(a->N + 255) / 256, 256, 0, st>>>(a->verts, a->shape, a->N, a->S, sh4);
  HR_LAUNCHED(ctx);
  k_strand_prims<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a->verts, sh4, a->N, a->S,
                                                             a->prim_xf, a->prim_box,
                                                             a->prim_aux);
  HR_LAUNCHED(ctx);
  return scene_bounds(ctx, a, n);
}

namespace {

// Level offsets of a hierarchy of C clusters over N strands and its arrays
// (reused when the shape is unchanged, as for a new frame of the same hair).
hr_status hierarchy_setup(hr_ctx* ctx, hr_asset* a, uint32_t C, uint32_t max_levels,
                          LevelInfo& li, uint64_t& E_out, uint64_t& total_out) {
  const uint32_t N = a->N, S = a->S;
  // level count: 1 + max k with 4^k <= floor(N/C)/2, capped
  const uint32_t per = N / C;
  uint32_t L = 0;
  if (per >= 2) {
    uint32_t k = 0;
    while ((1ull << (2 * (k + 1))) <= per / 2) ++k;
    L = k + 1;
    if (max_levels > 0 && L > max_levels) L = max_levels;
  }
  if (L > 8) L = 8;
  li = LevelInfo{};
  li.n_levels = L;
  uint64_t E = 0;
  for (uint32_t k = 0; k < L; ++k) {
    li.off[k] = (uint32_t)E;
    E += (uint64_t)C << (2 * k);
  }
  li.off[L] = (uint32_t)E;
  const uint64_t total = (uint64_t)N * S + E * S;
  if (total >= (1ull << 30) || E >= (1ull << 28))
    return set_error(ctx, HR_EINVAL, "hierarchy too large for 30-bit primitive ids");

  // A hierarchy of the same shape (a new frame of the same hair) reuses the
  // arrays, and keeps the LoD selection as the previous frame's (Eq. 14);
  // another shape frees and reallocates them.
  const bool same_shape = a->order && a->C == C && a->n_levels == L && a->E == (uint32_t)E &&
                          (E == 0 || a->xsec);
  a->bvh.valid = 0;
  if (!same_shape) {
    if (a->order) dfree(ctx, a->order, (size_t)N * 4), a->order = nullptr;
    if (a->cluster_of) dfree(ctx, a->cluster_of, (size_t)N * 4), a->cluster_of = nullptr;
    if (a->cl_first) dfree(ctx, a->cl_first, (size_t)(a->C + 1) * 4), a->cl_first = nullptr;
    if (a->xsec) dfree(ctx, a->xsec, (size_t)a->E * (S + 1) * 3 * sizeof(float4)), a->xsec = nullptr;
    if (a->xsec_other)
      dfree(ctx, a->xsec_other, (size_t)a->E * (S + 1) * 3 * sizeof(float4)), a->xsec_other = nullptr;
    if (a->lod) dfree(ctx, a->lod, a->C), a->lod = nullptr;
    a->lod_valid = 0;
    HR_TRY(dalloc(ctx, (void**)&a->order, (size_t)N * 4, "order"));
    HR_TRY(dalloc(ctx, (void**)&a->cluster_of, (size_t)N * 4, "cluster_of"));
    HR_TRY(dalloc(ctx, (void**)&a->cl_first, (size_t)(C + 1) * 4, "cluster first"));
    HR_TRY(dalloc(ctx, (void**)&a->lod, C, "lod"));
  }
  a->C = C;
  a->n_levels = L;
  a->E = (uint32_t)E;
  for (uint32_t k = 0; k <= L && k < 16; ++k) a->eth_offset[k] = li.off[k];
  E_out = E;
  total_out = total;
  return HR_OK;
}

// Thick-hair materials, fits and segment records of the hierarchy whose
// order and cluster starts are set, growing the material and primitive arrays.

// The fit runs on st_fit (the side stream of a pipelined frame, or the main
// stream); the thick-hair materials and records, which the frame in flight
// reads, on the main stream after it.
hr_status hierarchy_finish(hr_ctx* ctx, hr_asset* a, const LevelInfo& li, uint64_t E,
                           uint64_t total, cudaEvent_t fit_begin, cudaEvent_t fit_end,
                           cudaStream_t st_fit = nullptr) {
  cudaStream_t st = ctx_stream(ctx);
  cudaStream_t sf = st_fit ? st_fit : st;
  const uint32_t N = a->N, S = a->S;
  // grow the material table to strands + thick hairs
  if (a->mat_cap < (size_t)N + E) {
    float* m2 = nullptr;
    HR_TRY(dalloc(ctx, (void**)&m2, (size_t)(N + E) * HR_MAT_FLOATS * 4, "materials"));
    HR_CUDA(ctx, cudaMemcpyAsync(m2, a->mat, (size_t)N * HR_MAT_FLOATS * 4,
                                 cudaMemcpyDeviceToDevice, st));
    HR_CUDA(ctx, cudaStreamSynchronize(st));
    dfree(ctx, a->mat, a->mat_cap * HR_MAT_FLOATS * 4);
    a->mat = m2;
    a->mat_cap = (size_t)N + E;
  }

  // grow the primitive arrays to strands + thick hairs (strand part copied)
  const uint64_t ns = (uint64_t)N * S;
  if (a->n_prims_total != total) {
    float4 *xf = nullptr, *bx = nullptr, *ax = nullptr;
    HR_TRY(dalloc(ctx, (void**)&xf, total * 3 * sizeof(float4), "records"));
    HR_TRY(dalloc(ctx, (void**)&bx, total * 2 * sizeof(float4), "boxes"));
    HR_TRY(dalloc(ctx, (void**)&ax, total * sizeof(float4), "aux"));
    HR_CUDA(ctx, cudaMemcpyAsync(xf, a->prim_xf, ns * 3 * sizeof(float4), cudaMemcpyDeviceToDevice, st));
    HR_CUDA(ctx, cudaMemcpyAsync(bx, a->prim_box, ns * 2 * sizeof(float4), cudaMemcpyDeviceToDevice, st));
    HR_CUDA(ctx, cudaMemcpyAsync(ax, a->prim_aux, ns * sizeof(float4), cudaMemcpyDeviceToDevice, st));
    HR_CUDA(ctx, cudaStreamSynchronize(st));
    const uint64_t old = a->n_prims_total;
    dfree(ctx, a->prim_xf, old * 3 * sizeof(float4));
    dfree(ctx, a->prim_box, old * 2 * sizeof(float4));
    dfree(ctx, a->prim_aux, old * sizeof(float4));
    a->prim_xf = xf;
    a->prim_box = bx;
    a->prim_aux = ax;
    a->n_prims_total = (uint32_t)total;
  }
  // The scene bounds (for the BVH's Morton codes) are those of the strand
  // segments' boxes, taken when the asset was created: a thick-hair segment's
  // box centre is the mean of member vertices, so it lies inside them.
  if (E == 0) {
    if (sf != st) {
      HR_CUDA(ctx, cudaEventRecord(ctx_fit_event(ctx), sf));
      HR_CUDA(ctx, cudaStreamWaitEvent(st, ctx_fit_event(ctx), 0));
    }
    return HR_OK;
  }

  // K2: cross-section fits (FP64 covariance and eigenvectors), materials and
  // thick-hair segment records
  if (!a->xsec)
    HR_TRY(dalloc(ctx, (void**)&a->xsec, (size_t)E * (S + 1) * 3 * sizeof(float4), "cross-sections"));
  float* eth_r = nullptr;
  HR_TRY(scratch(ctx, 5, (size_t)E * sizeof(float), (void**)&eth_r));
  const uint64_t nx = E * (S + 1);
  if (fit_begin) HR_CUDA(ctx, cudaEventRecord(fit_begin, sf));
  k_fit_cross_sections<<<(unsigned)((nx + 127) / 128), 128, 0, sf>>>(a->verts, S, a->order,
                                                                    a->cl_first, li, (uint32_t)E,
                                                                    a->xsec);
  HR_LAUNCHED(ctx);
  if (fit_end) HR_CUDA(ctx, cudaEventRecord(fit_end, sf));
  if (sf != st) {
    HR_CUDA(ctx, cudaEventRecord(ctx_fit_event(ctx), sf));
    HR_CUDA(ctx, cudaStreamWaitEvent(st, ctx_fit_event(ctx), 0));
  }
  k_eth_material<<<(unsigned)((E * (HR_MAT_FLOATS + 1) + 127) / 128), 128, 0, st>>>(a->verts, N, S, a->order,
                                                             a->cl_first, li, (uint32_t)E,
                                                             a->mat, eth_r);
  HR_LAUNCHED(ctx);
  const uint64_t ne = E * S;
  k_eth_prims<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(a->xsec, N, S, (uint32_t)E,
                                                           a->cl_first, li, eth_r, a->prim_xf,
                                                           a->prim_box, a->prim_aux);
  HR_LAUNCHED(ctx);
  return HR_OK;
}

}  // namespace

hr_status build_hierarchy(hr_ctx* ctx, hr_asset* a, uint32_t C, uint32_t max_levels,
                          cudaEvent_t fit_begin, cudaEvent_t fit_end, cudaStream_t st_fit) {
  // K1 and the fit on st_fit when the caller pipelines frames (see hierarchy_finish)
  cudaStream_t st = st_fit ? st_fit : ctx_stream(ctx);
  const uint32_t N = a->N, S = a->S;
  LevelInfo li{};
  uint64_t E = 0, total = 0;
  HR_TRY(hierarchy_setup(ctx, a, C, max_levels, li, E, total));
  drop_guides(ctx, a);  // a Morton hierarchy replaces a guide-driven one
  // K1: Morton order of the roots
  uint32_t *bounds, *keys, *vals, *k2, *v2;
  HR_TRY(scratch(ctx, 0, 64, (void**)&bounds));
  HR_TRY(scratch(ctx, 1, (size_t)N * 4, (void**)&keys));
  HR_TRY(scratch(ctx, 2, (size_t)N * 4, (void**)&k2));
  HR_TRY(scratch(ctx, 3, (size_t)N * 4, (void**)&v2));
  HR_TRY(scratch(ctx, 4, (size_t)N * 4, (void**)&vals));
  k_init_bounds<<<1, 32, 0, st>>>(bounds);
  HR_LAUNCHED(ctx);
  k_root_bounds<<<(N + 255) / 256, 256, 0, st>>>(a->verts, N, S, bounds);
  HR_LAUNCHED(ctx);
  k_root_morton<<<(N + 255) / 256, 256, 0, st>>>(a->verts, N, S, bounds, keys, vals);
  HR_LAUNCHED(ctx);
  HR_TRY(radix_sort_pairs(ctx, keys, vals, k2, v2, N, 30, st));
  // a new strand order (moved roots) changes the clusters: no refit of a BVH
  // built before it
  k_words_differ<<<(N + 255) / 256, 256, 0, st>>>(vals, a->order, N, a->d_bounds + kHierChanged);
  HR_LAUNCHED(ctx);
  HR_CUDA(ctx, cudaMemcpyAsync(a->order, vals, (size_t)N * 4, cudaMemcpyDeviceToDevice, st));
  k_assign_clusters<<<(N + 255) / 256, 256, 0, st>>>(a->order, N, C, a->cluster_of);
  HR_LAUNCHED(ctx);
  k_cluster_first<<<(C + 1 + 255) / 256, 256, 0, st>>>(N, C, a->cl_first);
  HR_LAUNCHED(ctx);

  return hierarchy_finish(ctx, a, li, E, total, fit_begin, fit_end, st_fit);
}

hr_status rebuild_eth_records(hr_ctx* ctx, hr_asset* a) {
  cudaStream_t st = ctx_stream(ctx);
  const uint32_t N = a->N, S = a->S, E = a->E;
  if (E == 0) return HR_OK;
  LevelInfo li{};
  li.n_levels = a->n_levels;
  for (uint32_t k = 0; k <= a->n_levels && k < 16; ++k) li.off[k] = a->eth_offset[k];
  float* eth_r = nullptr;
  HR_TRY(scratch(ctx, 5, (size_t)E * sizeof(float), (void**)&eth_r));
  k_eth_material<<<(unsigned)(((uint64_t)E * (HR_MAT_FLOATS + 1) + 127) / 128), 128, 0, st>>>(
      a->verts, N, S, a->order, a->cl_first, li, E, a->mat, eth_r);
  HR_LAUNCHED(ctx);
  k_eth_prims<<<(unsigned)(((uint64_t)E * S + 255) / 256), 256, 0, st>>>(
      a->xsec, N, S, E, a->cl_first, li, eth_r, a->prim_xf, a->prim_box, a->prim_aux);
  HR_LAUNCHED(ctx);
  return HR_OK;
}

hr_status root_morton_order(hr_ctx* ctx, hr_asset* a, uint32_t* codes, uint32_t* order,
                            cudaStream_t st) {
  const uint32_t N = a->N, S = a->S;
  uint32_t *bounds, *k2, *v2;
  HR_TRY(scratch(ctx, 0, 64, (void**)&bounds));
  HR_TRY(scratch(ctx, 2, (size_t)N * 4, (void**)&k2));
  HR_TRY(scratch(ctx, 3, (size_t)N * 4, (void**)&v2));
  k_init_bounds<<<1, 32, 0, st>>>(bounds);
  HR_LAUNCHED(ctx);
  k_root_bounds<<<(N + 255) / 256, 256, 0, st>>>(a->verts, N, S, bounds);
  HR_LAUNCHED(ctx);
  k_root_morton<<<(N + 255) / 256, 256, 0, st>>>(a->verts, N, S, bounds, codes, order);
  HR_LAUNCHED(ctx);
  return radix_sort_pairs(ctx, codes, order, k2, v2, N, 30, st);
}

hr_status build_hierarchy_from(hr_ctx* ctx, hr_asset* a, uint32_t C, uint32_t max_levels,
                               const uint32_t* order_dev, const uint32_t* cl_first_dev) {
  cudaStream_t st = ctx_stream(ctx);
  const uint32_t N = a->N;
  LevelInfo li{};
  uint64_t E = 0, total = 0;
  HR_TRY(hierarchy_setup(ctx, a, C, max_levels, li, E, total));
  HR_CUDA(ctx, cudaMemsetAsync(a->d_bounds + kHierChanged, 0xff, 4, st));  // a new hierarchy
  HR_CUDA(ctx, cudaMemcpyAsync(a->order, order_dev, (size_t)N * 4, cudaMemcpyDeviceToDevice, st));
  HR_CUDA(ctx, cudaMemcpyAsync(a->cl_first, cl_first_dev, (size_t)(C + 1) * 4,
                               cudaMemcpyDeviceToDevice, st));
  k_cluster_of_from_first<<<C, 256, 0, st>>>(a->order, a->cl_first, a->cluster_of);
  HR_LAUNCHED(ctx);
  return hierarchy_finish(ctx, a, li, E, total, nullptr, nullptr);
}

// Morton clustering of strand roots on caller-provided scratch (no
// allocation): bounds (6 words), keys / key / value temporaries (n words
// each), digit counts (ceil(n / 2048) * 256 words), scan sums (<= 1024 words).
cudaError_t morton_clusters_with(const float4* verts, uint32_t N, uint32_t S, uint32_t C,
                                 uint32_t* order, uint32_t* cluster_of, uint32_t* bounds,
                                 uint32_t* keys, uint32_t* keys_tmp, uint32_t* vals_tmp,
                                 uint32_t* counts, uint32_t* sums, cudaStream_t st) {
  k_init_bounds<<<1, 32, 0, st>>>(bounds);
  k_root_bounds<<<(N + 255) / 256, 256, 0, st>>>(verts, N, S, bounds);
  k_root_morton<<<(N + 255) / 256, 256, 0, st>>>(verts, N, S, bounds, keys, order);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = radix_sort_pairs_with(keys, order, keys_tmp, vals_tmp, N, 30, counts, sums, st);
  if (e != cudaSuccess) return e;
  k_assign_clusters<<<(N + 255) / 256, 256, 0, st>>>(order, N, C, cluster_of);
  return cudaGetLastError();
}

}  // namespace hr

