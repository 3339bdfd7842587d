// Device code of the hot path: camera rays, BVH traversal, ray versus
// elliptic-cylinder tests, k-buffer, scattering models and compositing.
//
//  * Camera: sample sid = pixel * spp + s; sub-pixel position from SplitMix64
//    outputs 2 sid and 2 sid + 1 of the frame seed (top 24 bits each).
//  * Traversal: stack-based over the binary LBVH whose nodes hold both
//    children's boxes (one 64-byte node fetch tests two boxes); nearer child
//    first.  The search interval shrinks to the K-th nearest hit and to the
//    nearest opaque (strand) hit: nothing behind an opaque hit can contribute.
//  * Intersection: the record maps the ray into the cylinder's unit frame;
//    the quadratic is solved about the point of closest approach and the root
//    kept is the nearest one with w in [0, 1] (open cylinder).
//  * Shading: f_single (Eq. 1) for strands, f_ours (Eq. 5-13) for thick
//    hairs, per light; forward/backward single-fibre albedos from the
//    longitudinal-integral table.
//  * Compositing: front to back over the k-buffer sorted by (t, id).
#pragma once

#include "common.cuh"
#include "dword.cuh"

namespace hr {
namespace tr {

#define kInf __int_as_float(0x7f800000)
constexpr int kStack = 64;

__device__ __forceinline__ uint64_t splitmix_out(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float clampf(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }

// ------------------------------------------------------------------ geometry

// ------------------------------------------------------------------ precision
//
// The hit decisions are taken in FP32 wherever FP32 rounding cannot change
// them, and precisely otherwise.
//  * Every camera ray is built in double-word FP32 (the oracle's FP64
//    construction to about 2^-44) and re-based at its entry into the scene's
//    bounding box: the FP32 ray (o', d) starts next to the hair, and depths
//    are kept relative to that origin.  FP32 rounding then
//    moves a hit by ~2^-24 of the scene's size instead of ~2^-24 of the
//    camera distance.
//  * intersect32 bounds the rounding of its affine rows and of the roots.  A
//    test within that bound of the cylinder's outline or of an end of the
//    segment, a hit whose depth bound could reorder it against another hit or
//    the search cut, or whose bound is wide, is decided by refine: the
//    double-word ray re-based near the hit relative to the segment's start
//    point, and the quadratic solved about that point.  Kept FP32 hits whose
//    order against a precise one their bounds leave open are refined too.
// Far cameras and thin fibres (4K views of 1e-3 strands ten units away)
// otherwise turn up FP32 rounding errors of a few 1e-7 in position, enough
// to swap two strands at nearly equal depth or drop a hit at the very edge of
// a fibre.

constexpr int kMiss = 0, kHit = 1, kBorder = 2;
constexpr float kEps32 = 5.9604645e-8f;   // FP32 unit roundoff, 2^-24
constexpr float kBoundK = 6.f;            // rounding steps per affine row, with margin
// Relative depth (of the absolute depth) that widens the box cull, and above
// which an FP32 depth bound sends the hit to refine.
constexpr float kTieRel = 1.52587890625e-05f;  // 2^-16

struct RayKey {  // what rebuilds the ray precisely: the sample id and the re-basing offset
  uint64_t sid;
  float s_off;  // o' = o + s_off v, v the unnormalised direction (|v| >= 1)
};

// Ray against the open elliptic cylinder of one record, in FP32, with a
// bound on the rounding of each decision.  kMiss when the ray misses by more
// than the bound; kBorder when the rounding could change the outcome; else
// kHit with the nearest root t in (0, tmax] (axial coordinate in [0, 1]),
// and its error bound terr.
// M = |o.x| + |o.y| + |o.z| of the ray.
__device__ __forceinline__ int intersect32(const float4* __restrict__ xf, const float3 o,
                                           const float3 d, const float M, const float tmax,
                                           float& t_hit, float& terr) {
  const float4 r0 = __ldg(xf), r1 = __ldg(xf + 1), r2 = __ldg(xf + 2);
  const float u0 = fmaf(r0.x, o.x, fmaf(r0.y, o.y, fmaf(r0.z, o.z, r0.w)));
  const float v0 = fmaf(r1.x, o.x, fmaf(r1.y, o.y, fmaf(r1.z, o.z, r1.w)));
  const float du = fmaf(r0.x, d.x, fmaf(r0.y, d.y, r0.z * d.z));
  const float dv = fmaf(r1.x, d.x, fmaf(r1.y, d.y, r1.z * d.z));
  const float A = fmaf(du, du, dv * dv);
  if (!(A > 0.f)) return kMiss;
  const float inv = 1.0f / A;
  const float tc = -fmaf(u0, du, v0 * dv) * inv;
  const float uc = fmaf(tc, du, u0), vc = fmaf(tc, dv, v0);
  const float h2 = fmaf(uc, uc, vc * vc);
  // rounding bound of (uc, vc): the rows' intermediate terms reach |r| (|o| + |tc|)
  const float mag = M + fabsf(tc);
  const float eu = kBoundK * kEps32 *
                   fmaf(fabsf(r0.x) + fabsf(r0.y) + fabsf(r0.z), mag, fabsf(r0.w));
  const float ev = kBoundK * kEps32 *
                   fmaf(fabsf(r1.x) + fabsf(r1.y) + fabsf(r1.z), mag, fabsf(r1.w));
  const float e = eu + ev;
  const float dh = e * (2.f + e);
  if (h2 > 1.f + dh) return kMiss;
  bool border = h2 >= 1.f - dh;  // near the outline
  const float g = fmaxf(1.f - h2, 0.f);
  const float half = sqrtf(g * inv);
  const float tm = tc - half, tp = tc + half;
  // depth bound: the (u, v) error over |(du, dv)|, the root's slope (near
  // the outline at most sqrt(dh / A)), and the rounding of t itself
  const float magt = mag + half;
  const float eroot = border ? sqrtf(dh * inv) : dh * half * (0.5f / g);
  terr = fmaf(e, sqrtf(inv), fmaf(4.f * kEps32, magt, eroot));
  if (tp + terr <= 0.f || tm - terr > tmax) return kMiss;
  const float w0 = fmaf(r2.x, o.x, fmaf(r2.y, o.y, fmaf(r2.z, o.z, r2.w)));
  const float dw = fmaf(r2.x, d.x, fmaf(r2.y, d.y, r2.z * d.z));
  // axial coordinate of each root, and its error bound (the row's rounding
  // and the root's depth error times the axial rate)
  const float ew = fmaf(kBoundK * kEps32,
                        fmaf(fabsf(r2.x) + fabsf(r2.y) + fabsf(r2.z), magt, fabsf(r2.w)),
                        fabsf(dw) * terr);
  const float wm = fmaf(tm, dw, w0), wp = fmaf(tp, dw, w0);
  // each root: certainly in range, possibly in range, or certainly not
  const bool m_in = tm > terr && wm >= ew && wm <= 1.f - ew;
  const bool m_may = tm > -terr && wm >= -ew && wm <= 1.f + ew;
  const bool p_in = tp > terr && wp >= ew && wp <= 1.f - ew;
  const bool p_may = tp > -terr && wp >= -ew && wp <= 1.f + ew;
  float t;
  if (m_in) {
    t = tm;
  } else if (m_may) {
    t = fmaxf(tm, 0.f);
    border = true;
  } else if (p_in) {
    t = tp;
  } else if (p_may) {
    t = fmaxf(tp, 0.f);
    border = true;
  } else {
    return kMiss;
  }
  if (t - terr > tmax) return kMiss;
  t_hit = t;
  return border ? kBorder : kHit;
}

// Camera ray of a sample in double-word FP32, the oracle's construction to
// about 2^-44: sub-pixel offset from the top 24 bits of SplitMix64 outputs
// 2 sid and 2 sid + 1, image-plane offset ((x + jx) - W / 2,
// H / 2 - (y + jy)) / pix (exact pairs times the double-word 1 / pix);
// perspective
// rays leave the eye along v = (fwd + sx right) + sy up, orthographic ones
// leave (eye + sx right) + sy up along fwd.  v is left unnormalised: the
// ray's point at parameter s is o + s v.
struct PreciseRay {
  df o[3], v[3];
};
static __device__ void camera_ray_dw(const LaunchCam& c, uint64_t seed, uint32_t spp, uint64_t sid,
                                     PreciseRay& r) {
  const float jx = (float)(uint32_t)(splitmix_out(seed, 2 * sid) >> 40) * (1.0f / 16777216.0f);
  const float jy = (float)(uint32_t)(splitmix_out(seed, 2 * sid + 1) >> 40) * (1.0f / 16777216.0f);
  uint32_t px, py;
  if (sid < (1ull << 32)) {
    const uint32_t pixel = (uint32_t)sid / spp;
    px = pixel % (uint32_t)c.W;
    py = pixel / (uint32_t)c.W;
  } else {
    const uint64_t pixel = sid / spp;
    px = (uint32_t)(pixel % (uint64_t)c.W);
    py = (uint32_t)(pixel / (uint64_t)c.W);
  }
  const float x = (float)px, y = (float)py;
  float ex, ey;
  const float ax = two_sum(__fsub_rn(x, 0.5f * (float)c.W), jx, ex);
  const float ay = two_sum(__fsub_rn(0.5f * (float)c.H, y), -jy, ey);
  const df ipix{c.ipix_hi, c.ipix_lo};
  const df sx = df_mul(df{ax, ex}, ipix), sy = df_mul(df{ay, ey}, ipix);
  const float E[3] = {c.eye.x, c.eye.y, c.eye.z}, R[3] = {c.right.x, c.right.y, c.right.z};
  const float U[3] = {c.up.x, c.up.y, c.up.z}, F[3] = {c.fwd.x, c.fwd.y, c.fwd.z};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const df w = df_add(df_add(df_mul(sx, R[i]), c.kind == 1 ? F[i] : E[i]), df_mul(sy, U[i]));
    if (c.kind == 1) {
      r.o[i] = df{E[i], 0.f};
      r.v[i] = w;
    } else {
      r.o[i] = w;
      r.v[i] = df{F[i], 0.f};
    }
  }
}

// |v|^2 of a double-word vector and its square root in double-word (one
// Newton correction from the exact FMA residual).
__device__ __forceinline__ df df_norm2(const df v[3]) {
  return df_add(df_add(df_mul(v[0], v[0]), df_mul(v[1], v[1])), df_mul(v[2], v[2]));
}
__device__ __forceinline__ df df_sqrt(df a) {
  const float r = __fsqrt_rn(a.hi);
  return df_fast(r, __fdiv_rn(__fadd_rn(fmaf(-r, r, a.hi), a.lo), 2.f * r));
}

// The FP32 ray of a sample: the direction normalised in FP32 (correctly
// rounded steps, so |d| = 1 within a few ulps), and the origin moved to a
// little before the ray's entry into the scene's bounding box (the root
// node's two boxes), o' = o + s_off v, formed in double-word before rounding.
// Hits are at depth t' past o' along d; no primitive lies before the entry,
// so t' > 0 for every hit.
__device__ __forceinline__ void primary_ray(const FrameArgs& fa, uint64_t sid, float3& o,
                                            float3& d, RayKey& rk) {
  PreciseRay ry;
  camera_ray_dw(fa.cam, fa.seed, fa.spp, sid, ry);
  const float vx = ry.v[0].hi, vy = ry.v[1].hi, vz = ry.v[2].hi;
  const float il = __frcp_rn(__fsqrt_rn(fmaf(vx, vx, fmaf(vy, vy, __fmul_rn(vz, vz)))));
  d = f3(__fmul_rn(vx, il), __fmul_rn(vy, il), __fmul_rn(vz, il));
  float s_off = 0.f;
  if (fa.n_prims >= 2) {
    const float4 n0 = __ldg(fa.nodes), n1 = __ldg(fa.nodes + 1), n2 = __ldg(fa.nodes + 2);
    const float3 oo = f3(ry.o[0].hi, ry.o[1].hi, ry.o[2].hi);
    const float3 inv = f3(1.0f / (fabsf(d.x) > 1e-12f ? d.x : copysignf(1e-12f, d.x)),
                          1.0f / (fabsf(d.y) > 1e-12f ? d.y : copysignf(1e-12f, d.y)),
                          1.0f / (fabsf(d.z) > 1e-12f ? d.z : copysignf(1e-12f, d.z)));
    const float lx = (fminf(n0.x, n1.x) - oo.x) * inv.x, hx = (fmaxf(n0.y, n1.y) - oo.x) * inv.x;
    const float ly = (fminf(n0.z, n1.z) - oo.y) * inv.y, hy = (fmaxf(n0.w, n1.w) - oo.y) * inv.y;
    const float lz = (fminf(n2.x, n2.z) - oo.z) * inv.z, hz = (fmaxf(n2.y, n2.w) - oo.z) * inv.z;
    const float t0 = fmaxf(fmaxf(fminf(lx, hx), fminf(ly, hy)), fminf(lz, hz));
    const float t1 = fminf(fminf(fmaxf(lx, hx), fmaxf(ly, hy)), fmaxf(lz, hz));
    // 2^-10 before the FP32 entry: far more than the slab test's rounding
    if (t0 > 0.f && t0 <= t1) s_off = t0 * (1.f - 9.765625e-4f) * il;
  }
  rk = RayKey{sid, s_off};
  o = f3(df_float(df_add(ry.o[0], df_mul(ry.v[0], s_off))),
         df_float(df_add(ry.o[1], df_mul(ry.v[1], s_off))),
         df_float(df_add(ry.o[2], df_mul(ry.v[2], s_off))));
}

// The precise decision of one test, for hits the FP32 test cannot order or
// classify.  The ray is built in double-word FP32 and re-based at its point
// s0 v (s0 from the FP32 depth estimate) relative to the segment's start
// point c0 (a strand vertex or a thick-hair cross-section centre): that point
// lies within about a segment length of c0, so rounding it to FP32 costs
// ~2^-24 of a segment length instead of ~2^-24 of the camera distance.  The
// cylinder (the record's FP32 linear rows, through c0) is then solved about
// it in FP32: the nearest root of o + s v with s > 0 and axial coordinate in
// [0, 1].  t_est and the result are depths past the re-based origin
// o' = o + s_off v; the result is a normalised pair t' = t_hi + t_lo.  About 300 FP32 operations, against ~200 FP64 operations (1/64 of
// the FP32 rate on this GPU) for the same test in FP64.
static __device__ __noinline__ bool refine(const FrameArgs& fa, const RayKey& rk, uint32_t id,
                                           float t_est, float& t_hi, float& t_lo) {
  PreciseRay ry;
  camera_ray_dw(fa.cam, fa.seed, fa.spp, rk.sid, ry);
  const float4* xf = fa.prim_xf + 3 * (size_t)id;
  const float4 r0 = __ldg(xf), r1 = __ldg(xf + 1), r2 = __ldg(xf + 2);
  const uint32_t S = fa.S, NS = fa.N * fa.S;
  float4 c0;
  if (id < NS)
    c0 = __ldg(fa.verts + (size_t)(id / S) * (S + 1) + id % S);
  else
    c0 = __ldg(fa.xsec + ((size_t)((id - NS) / S) * (S + 1) + (id - NS) % S) * 3);
  const float vx = ry.v[0].hi, vy = ry.v[1].hi, vz = ry.v[2].hi;
  const df L = df_sqrt(df_norm2(ry.v));  // depth along the unit direction = s |v|
  // re-base at o + (s_off + s0) v, s0 the FP32 depth estimate past o' in units of v
  const float s0 = t_est / L.hi;
  float sb;
  const float sa = two_sum(rk.s_off, s0, sb);
  const df sp0{sa, sb};
  const float C0[3] = {c0.x, c0.y, c0.z};
  float p[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) p[i] = df_float(df_add(df_add(ry.o[i], -C0[i]), df_mul(ry.v[i], sp0)));
  const float u0 = fmaf(r0.x, p[0], fmaf(r0.y, p[1], __fmul_rn(r0.z, p[2])));
  const float v0 = fmaf(r1.x, p[0], fmaf(r1.y, p[1], __fmul_rn(r1.z, p[2])));
  const float w0 = fmaf(r2.x, p[0], fmaf(r2.y, p[1], __fmul_rn(r2.z, p[2])));
  const float du = fmaf(r0.x, vx, fmaf(r0.y, vy, __fmul_rn(r0.z, vz)));
  const float dv = fmaf(r1.x, vx, fmaf(r1.y, vy, __fmul_rn(r1.z, vz)));
  const float dw = fmaf(r2.x, vx, fmaf(r2.y, vy, __fmul_rn(r2.z, vz)));
  const float A = fmaf(du, du, __fmul_rn(dv, dv));
  if (!(A > 0.f)) return false;
  const float inv = 1.0f / A;
  const float sc = __fmul_rn(-fmaf(u0, du, __fmul_rn(v0, dv)), inv);
  const float uc = fmaf(sc, du, u0), vc = fmaf(sc, dv, v0);
  const float h2 = fmaf(uc, uc, __fmul_rn(vc, vc));
  if (h2 > 1.f) return false;
  const float half = sqrtf(__fmul_rn(__fsub_rn(1.f, h2), inv));
  const float sm = __fsub_rn(sc, half), sp = __fadd_rn(sc, half);
  const float wm = fmaf(sm, dw, w0), wp = fmaf(sp, dw, w0);
  float s;
  // in front of the eye: s_off + s0 + s > 0 (s_off is 0 unless the eye is
  // outside the scene box, and then every root is far in front of it)
  if (__fadd_rn(sa, sm) > 0.f && wm >= 0.f && wm <= 1.f)
    s = sm;
  else if (__fadd_rn(sa, sp) > 0.f && wp >= 0.f && wp <= 1.f)
    s = sp;
  else
    return false;
  float e;
  const float th = two_sum(s0, s, e);
  const df t = df_mul(df_fast(th, e), L);
  t_hi = t.hi;
  t_lo = t.lo;
  return true;
}

// The K nearest hits: depth and entry word.  The entry word holds the
// global primitive id (which also addresses the primitive's records; a thick
// hair's chord is recomputed from them when it is shaded) and two flags:
// kExact when the depth was decided precisely (t + tr is then a normalised
// double-word depth) and kOpaque for a strand hit.  An FP32 entry has tr = 0.
// Entries order by (t, tr, id).
constexpr uint32_t kIdMask = 0x3fffffffu, kOpaque = 0x40000000u, kExact = 0x80000000u;
constexpr uint32_t kNoEntry = kIdMask;  // an empty slot (t = inf)
template <int KMAX>
struct KBuf {
  float t[KMAX];
  float tr[KMAX];
  uint32_t id[KMAX];
};

template <int KMAX>
__device__ __forceinline__ void kbuf_init(KBuf<KMAX>& kb) {
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    kb.t[j] = kInf;
    kb.tr[j] = 0.f;
    kb.id[j] = kNoEntry;
  }
}

__device__ __forceinline__ bool key_less(float t, float tr, uint32_t id, float t2, float tr2,
                                         uint32_t id2) {
  return t < t2 || (t == t2 && (tr < tr2 || (tr == tr2 && (id & kIdMask) < (id2 & kIdMask))));
}

// Insert keeping the k nearest by (t, tr, id): the candidate bubbles through
// the sorted slots and whatever falls off the end is dropped.
template <int KMAX>
__device__ __forceinline__ void kbuf_insert(KBuf<KMAX>& kb, const uint32_t k, float t, float tr,
                                            uint32_t id) {
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    if (j < (int)k && key_less(t, tr, id, kb.t[j], kb.tr[j], kb.id[j])) {
      float a = kb.t[j]; kb.t[j] = t; t = a;
      float r = kb.tr[j]; kb.tr[j] = tr; tr = r;
      uint32_t b = kb.id[j]; kb.id[j] = id; id = b;
    }
  }
}

// The search cut: the depth of the k-th entry, or of the first opaque entry
// when it comes earlier (nothing behind an opaque hit is composited).
template <int KMAX>
__device__ __forceinline__ float kbuf_cut(const KBuf<KMAX>& kb, const uint32_t k) {
  float r = kInf;
#pragma unroll
  for (int j = KMAX - 1; j >= 0; --j)
    if (j < (int)k && (j == (int)k - 1 || (kb.id[j] & kOpaque))) r = kb.t[j];
  return r;
}

struct Counts {
  uint32_t nodes, tests, sshade, eshade, hits, rays, precise_tests, precise_entries;
  uint32_t steps;  // node visits plus primitive tests, counted in every kernel (tile schedule)
};

// Test primitive `id` (a leaf names its global primitive id) and keep it in
// the k-buffer when it is among the K nearest before the nearest opaque
// (strand) hit.  An FP32 hit is kept as it is when its depth bound terr is
// narrow, it is not near the outline or an end, and neither the cut nor any
// entry lies within terr + errmax of it, errmax being the widest bound of the
// FP32 entries kept so far: the FP32 entries are then pairwise further apart
// than the sum of their bounds, so their FP32 order is their true order.
// Otherwise the hit is decided precisely, and so is every FP32 entry within
// errmax of its precise depth (the only entries whose order against it the
// FP32 depths leave open).
template <int KMAX, bool COUNT>
__device__ __forceinline__ void leaf_test(const FrameArgs& fa, const RayKey& rk, uint32_t id,
                                          const float3 o, const float3 d, const float M,
                                          KBuf<KMAX>& kb, float& tcut, float& errmax, Counts& cn) {
  float th, terr;
  ++cn.steps;
  if (COUNT) ++cn.tests;
  const int r =
      intersect32(fa.prim_xf + 3 * (size_t)id, o, d, M, tcut + errmax, th, terr);
  if (r == kMiss) return;
  const float slack = terr + errmax;
  bool need = r == kBorder || terr > kTieRel * (rk.s_off + th) || th >= tcut - slack;
  if (!need) {
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < (int)fa.k && fabsf(th - kb.t[j]) <= slack) need = true;
  }
  uint32_t word = id | (__ldg(&fa.prim_aux[id].y) == 0.f ? kOpaque : 0u);
  float tr = 0.f;
  if (need) {
    if (COUNT) ++cn.precise_tests;
    float tl;
    if (!refine(fa, rk, id, th, th, tl)) return;
    tr = tl;
    word |= kExact;
    bool moved = false;
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
      if (j < (int)fa.k && kb.t[j] < kInf && !(kb.id[j] & kExact) &&
          fabsf(th - kb.t[j]) <= errmax) {
        float h, l;
        if (COUNT) ++cn.precise_entries;
        if (refine(fa, rk, kb.id[j] & kIdMask, kb.t[j], h, l)) {
          kb.t[j] = h;
          kb.tr[j] = l;
          kb.id[j] |= kExact;
        } else {  // not expected for an FP32 hit inside its bounds; dropped if it happens
          kb.t[j] = kInf;
          kb.tr[j] = 0.f;
          kb.id[j] = kNoEntry;
        }
        moved = true;
      }
    }
    if (moved) {  // refined depths moved by at most errmax: restore the order
#pragma unroll
      for (int i = 0; i + 1 < KMAX; ++i)
#pragma unroll
        for (int j = 0; j + 1 < KMAX - i; ++j)
          if (key_less(kb.t[j + 1], kb.tr[j + 1], kb.id[j + 1], kb.t[j], kb.tr[j], kb.id[j])) {
            float a = kb.t[j]; kb.t[j] = kb.t[j + 1]; kb.t[j + 1] = a;
            float q = kb.tr[j]; kb.tr[j] = kb.tr[j + 1]; kb.tr[j + 1] = q;
            uint32_t b = kb.id[j]; kb.id[j] = kb.id[j + 1]; kb.id[j + 1] = b;
          }
    }
  } else {
    errmax = fmaxf(errmax, terr);
  }
  kbuf_insert<KMAX>(kb, fa.k, th, tr, word);
  tcut = kbuf_cut<KMAX>(kb, fa.k);
}

// K nearest hits of one ray.  Returns false when the traversal stack overflowed
// (the far subtree was dropped; counted by the caller, never expected).
// Boxes are culled against the cut widened by the FP32 hits' depth bound and
// by 2 kTieRel of the absolute depth, so that no hit the precise ordering
// would keep is lost to FP32 rounding of the slab tests.
template <int KMAX, bool COUNT>
__device__ __forceinline__ bool traverse(const FrameArgs& fa, const RayKey& rk, const float3 o,
                                         const float3 d, KBuf<KMAX>& kb, Counts& cn) {
  kbuf_init<KMAX>(kb);
  if (fa.n_prims == 0) return true;
  float tcut = kInf, errmax = 0.f;
  const float M = fabsf(o.x) + fabsf(o.y) + fabsf(o.z);
  if (fa.n_prims == 1) {
    leaf_test<KMAX, COUNT>(fa, rk, __ldg(fa.leaf_id), o, d, M, kb, tcut, errmax, cn);
    return true;
  }
  // a zero direction component would turn the slab products into inf - inf;
  // keep its sign and floor its magnitude so every slab value stays ordered
  const float3 inv = f3(1.0f / (fabsf(d.x) > 1e-12f ? d.x : copysignf(1e-12f, d.x)),
                        1.0f / (fabsf(d.y) > 1e-12f ? d.y : copysignf(1e-12f, d.y)),
                        1.0f / (fabsf(d.z) > 1e-12f ? d.z : copysignf(1e-12f, d.z)));
  const float3 ooi = f3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
  int stack[kStack];
  int sp = 0;
  int node = 0;
  bool ok = true;
  for (;;) {
    if (node >= 0) {
      const float4* nd = fa.nodes + 4 * (size_t)node;
      const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
      ++cn.steps;
      if (COUNT) ++cn.nodes;
      const float tb = fmaf(tcut + errmax, 1.f + 2.f * kTieRel, 2.f * kTieRel * rk.s_off);
      // child 0
      float lx = fmaf(n0.x, inv.x, -ooi.x), hx = fmaf(n0.y, inv.x, -ooi.x);
      float ly = fmaf(n0.z, inv.y, -ooi.y), hy = fmaf(n0.w, inv.y, -ooi.y);
      float lz = fmaf(n2.x, inv.z, -ooi.z), hz = fmaf(n2.y, inv.z, -ooi.z);
      const float a0 = fmaxf(fmaxf(fminf(lx, hx), fminf(ly, hy)), fmaxf(fminf(lz, hz), 0.f));
      const float b0 = fminf(fminf(fmaxf(lx, hx), fmaxf(ly, hy)), fminf(fmaxf(lz, hz), tb));
      // child 1
      lx = fmaf(n1.x, inv.x, -ooi.x); hx = fmaf(n1.y, inv.x, -ooi.x);
      ly = fmaf(n1.z, inv.y, -ooi.y); hy = fmaf(n1.w, inv.y, -ooi.y);
      lz = fmaf(n2.z, inv.z, -ooi.z); hz = fmaf(n2.w, inv.z, -ooi.z);
      const float a1 = fmaxf(fmaxf(fminf(lx, hx), fminf(ly, hy)), fmaxf(fminf(lz, hz), 0.f));
      const float b1 = fminf(fminf(fmaxf(lx, hx), fmaxf(ly, hy)), fminf(fmaxf(lz, hz), tb));
      const bool h0 = a0 <= b0, h1 = a1 <= b1;
      const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
      if (h0 && h1) {
        const bool first0 = a0 <= a1;
        const int nearc = first0 ? c0 : c1, farc = first0 ? c1 : c0;
        if (sp < kStack)
          stack[sp++] = farc;
        else
          ok = false;
        node = nearc;
        continue;
      }
      if (h0 || h1) {
        node = h0 ? c0 : c1;
        continue;
      }
    } else {
      leaf_test<KMAX, COUNT>(fa, rk, (uint32_t)(~node), o, d, M, kb, tcut, errmax, cn);
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
  return ok;
}

// Slab reciprocals of a ray: a zero direction component would turn the slab
// products into inf - inf, so its sign is kept and its magnitude floored.
__device__ __forceinline__ void ray_slabs(const float3 o, const float3 d, float3& inv,
                                          float3& ooi) {
  inv = f3(1.0f / (fabsf(d.x) > 1e-12f ? d.x : copysignf(1e-12f, d.x)),
           1.0f / (fabsf(d.y) > 1e-12f ? d.y : copysignf(1e-12f, d.y)),
           1.0f / (fabsf(d.z) > 1e-12f ? d.z : copysignf(1e-12f, d.z)));
  ooi = f3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
}

// ------------------------------------------------------------------ scattering

struct Mat {
  float A[3][3];  // [R, TT, D][rgb]
  float bR, bT, gT;
};

__device__ __forceinline__ void load_mat(const float* __restrict__ m, Mat& o) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(m));
  const float4 b = __ldg(reinterpret_cast<const float4*>(m) + 1);
  const float4 c = __ldg(reinterpret_cast<const float4*>(m) + 2);
  o.A[0][0] = a.x; o.A[0][1] = a.y; o.A[0][2] = a.z;
  o.A[1][0] = a.w; o.A[1][1] = b.x; o.A[1][2] = b.y;
  o.A[2][0] = b.z; o.A[2][1] = b.w; o.A[2][2] = c.x;
  o.bR = c.y; o.bT = c.z; o.gT = c.w;
}

// Gaussian G(beta, x) = exp(-x^2 / 2 beta^2) / (sqrt(2 pi) beta), Section 3.2,
// evaluated with the hardware exponential in both table precisions (a table
// gather costs more than the exponential it replaces).
__device__ __forceinline__ float gauss(float beta, float x) {
  const float ib = 1.0f / beta;
  const float z = x * ib;
  return __expf(-0.5f * z * z) * (kInvSqrt2Pi * ib);
}

// Longitudinal albedo factor IM(theta, beta), bilinear in the baked table.
template <int PREC>
__device__ __forceinline__ float im_lookup(const Tables& tb, float theta, float beta) {
  const float ft = clampf(theta * ((kImNT - 1) / (0.5f * kPi)), 0.f, (float)(kImNT - 1));
  const float fb = clampf((beta - kImBetaLo) * ((kImNB - 1) / (kImBetaHi - kImBetaLo)), 0.f,
                          (float)(kImNB - 1));
  const int it = min((int)ft, kImNT - 2), ib = min((int)fb, kImNB - 2);
  const float wt = ft - (float)it, wb = fb - (float)ib;
  float v00, v01, v10, v11;
  const int i0 = ib * kImNT + it;
  if (PREC == HR_PREC_FP32) {
    v00 = __ldg(tb.im32 + i0);
    v01 = __ldg(tb.im32 + i0 + 1);
    v10 = __ldg(tb.im32 + i0 + kImNT);
    v11 = __ldg(tb.im32 + i0 + kImNT + 1);
  } else {
    v00 = __half2float(tb.im16[i0]);
    v01 = __half2float(tb.im16[i0 + 1]);
    v10 = __half2float(tb.im16[i0 + kImNT]);
    v11 = __half2float(tb.im16[i0 + kImNT + 1]);
  }
  const float a = fmaf(wt, v01 - v00, v00), b = fmaf(wt, v11 - v10, v10);
  return fmaf(wb, b - a, a);
}

constexpr float kInv2Pi = 0.15915494309189535f;
constexpr float kInvPi = 0.3183098861837907f;
constexpr float kInv2Pi2 = 0.05066059182116889f;  // 1 / (2 pi^2)

// Single-fibre BCSDF, Eq. (1).  sg2: the spread variance gathered on the
// light's path (0 without shadow rays), added to every lobe's variance.  With
// trt (HR_FLAG_TRT, Marschner's R / TT / TRT fibre) the third lobe is
// A_TRT G(2 beta_R, theta_h) / 2 pi instead of the diffuse A_D / 2 pi^2.
template <int PREC>
__device__ __forceinline__ void f_single(const Tables& tb, const Mat& m, float th_i, float th_o,
                                         float cphi, float sg2, bool trt, float out[3]) {
  const float th_h = 0.5f * (th_i + th_o);
  const float phi = acosf(clampf(cphi, -1.f, 1.f));
  const bool wide = sg2 > 0.f;
  const float bR = wide ? sqrtf(fmaf(m.bR, m.bR, sg2)) : m.bR;
  const float bT = wide ? sqrtf(fmaf(m.bT, m.bT, sg2)) : m.bT;
  const float gT = wide ? sqrtf(fmaf(m.gT, m.gT, sg2)) : m.gT;
  const float mR = gauss(bR, th_h) * kInv2Pi;
  const float mT = gauss(bT, th_h) * gauss(gT, phi - kPi);
  const float m3 = trt ? gauss(sqrtf(fmaf(4.f * m.bR, m.bR, sg2)), th_h) * kInv2Pi : kInv2Pi2;
#pragma unroll
  for (int c = 0; c < 3; ++c)
    out[c] = fmaf(m.A[0][c], mR, fmaf(m.A[1][c], mT, m.A[2][c] * m3));
}

// Per-hit constants of the aggregated model.
struct EthHit {
  float rho, n_view, nF, nB;
};

// Aggregated BCSDF of a thick hair, Eq. (5)-(13); readings as in the oracle:
// a_F, a_B at incidence |theta_d| / 2; variances add; n = 1 toward the back
// hemisphere (cos phi > 0); A_1+ summed in closed form for real n; B^ variance
// the attenuation-weighted mean of the path variances; S only for cos phi > 0
// with P_n floored at 0.
template <int PREC>
__device__ __forceinline__ void f_ours(const Tables& tb, const Mat& m, const EthHit& eh,
                                       float th_i, float th_o, float cphi, uint32_t flags,
                                       float sg2, float out[3]) {
  const float th_h = 0.5f * (th_i + th_o);
  const float ta = 0.5f * fabsf(th_i - th_o);
  const float phi = acosf(clampf(cphi, -1.f, 1.f));
  const bool trt = flags & HR_FLAG_TRT;
  const float imR = im_lookup<PREC>(tb, ta, m.bR);
  const float imT = im_lookup<PREC>(tb, ta, m.bT);
  // third lobe: diffuse (a quarter of A_D per half) or TRT (half of
  // A_TRT IM(2 beta_R) per half, its width weighted into the forward spread)
  const float im3 = trt ? 0.5f * im_lookup<PREC>(tb, ta, 2.f * m.bR) : 0.25f;
  float aF[3], aB[3];
  float wR = 0.f, wT = 0.f, w3 = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float r = m.A[0][c] * imR * 0.5f;
    const float tt = m.A[1][c] * imT;
    const float third = m.A[2][c] * im3;
    aF[c] = r + tt * eh.nF + third;
    aB[c] = r + tt * eh.nB + third;
    wR += r;
    wT += tt * eh.nF;
    w3 += third;
  }
  const float bR2 = m.bR * m.bR, bT2 = m.bT * m.bT;
  const float s2 = trt ? (wR * bR2 + wT * bT2 + w3 * 4.f * bR2) / (wR + wT + w3)
                       : (wR * bR2 + wT * bT2) / (wR + wT);
  const bool back = cphi > 0.f;
  const float n = back ? 1.f : eh.n_view;
  const float nm1 = n - 1.f;
  const float mR = gauss(sqrtf(fmaf(nm1, s2, bR2) + sg2), th_h) * kInv2Pi;
  const float mT = gauss(sqrtf(fmaf(nm1, s2, bT2) + sg2), th_h) *
                   gauss(sqrtf(fmaf(nm1, s2, m.gT * m.gT) + sg2), phi - kPi);
  const float m3 = trt ? gauss(sqrtf(fmaf(nm1, s2, 4.f * bR2) + sg2), th_h) * kInv2Pi : kInv2Pi2;
  float lob[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float att = nm1 > 0.f ? exp2f(nm1 * __log2f(aF[c])) : 1.f;
    lob[c] = att * fmaf(m.A[0][c], mR, fmaf(m.A[1][c], mT, m.A[2][c] * m3));
  }
  if (back) {
    float A1[3], A3[3], A1p[3];
    float w1 = 0.f, w3 = 0.f, w1p = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float f = fminf(aF[c], 1.f - 1e-6f);
      const float f2 = f * f, g = 1.f - f2, ig = 1.f / g;
      const float b = aB[c];
      A1[c] = b * f2 * ig;
      A3[c] = b * b * b * f2 * ig * ig * ig;
      A1p[c] = 0.6f * b * f * (1.f - exp2f(2.f * eh.n_view * __log2f(f))) * ig;
      w1 += A1[c];
      w3 += A3[c];
      w1p += A1p[c];
    }
    const float vB = (w1 * (bR2 + 2.f * s2) + w3 * (3.f * bR2 + 2.f * s2) +
                      w1p * (bR2 + (eh.n_view + 1.f) * s2)) / (w1 + w3 + w1p);
    const float mB = gauss(sqrtf(vB + sg2), th_h) * kInvPi;
#pragma unroll
    for (int c = 0; c < 3; ++c) lob[c] = fmaf(A1p[c] + A1[c] + A3[c], mB, lob[c]);
    if (!(flags & HR_FLAG_NO_S)) {
      const float Ps = (1.f - eh.rho) * (1.f - cphi);
      const float Pm = 0.2f * (1.f - eh.rho);
      const float Pn = fmaxf(0.f, 1.f - Pm - Ps);
#pragma unroll
      for (int c = 0; c < 3; ++c) lob[c] *= fmaf(Ps, aF[c], Pn);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) out[c] = lob[c];
}

// Forward albedo a_F (rgb) and forward spread variance of a fibre for light
// at incidence |theta| (the a_F reading of the aggregated model).
template <int PREC>
__device__ __forceinline__ void forward_albedo(const Tables& tb, const Mat& m, float theta_abs,
                                               bool trt, float aF[3], float& s2) {
  const float imR = im_lookup<PREC>(tb, theta_abs, m.bR);
  const float imT = im_lookup<PREC>(tb, theta_abs, m.bT);
  const float im3 = trt ? 0.5f * im_lookup<PREC>(tb, theta_abs, 2.f * m.bR) : 0.25f;
  const float nF = erff(kPi / (2.f * 1.41421356f * m.gT));
  float wR = 0.f, wT = 0.f, w3 = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float r = m.A[0][c] * imR * 0.5f;
    const float tt = m.A[1][c] * imT * nF;
    const float third = m.A[2][c] * im3;
    aF[c] = r + tt + third;
    wR += r;
    wT += tt;
    w3 += third;
  }
  const float bR2 = m.bR * m.bR;
  s2 = trt ? (wR * bR2 + wT * m.bT * m.bT + w3 * 4.f * bR2) / (wR + wT + w3)
           : (wR * bR2 + wT * m.bT * m.bT) / (wR + wT);
}

// The ray's interval inside one record's finite cylinder, clipped to
// (tmin, tmax): the hair a shadow ray crosses, or the chord of a primary hit.
// Returns false when empty.
__device__ __forceinline__ bool leaf_span(const float4* __restrict__ xf, const float3 o,
                                          const float3 d, const float tmin, const float tmax,
                                          float& lo, float& hi) {
  const float4 r0 = __ldg(xf), r1 = __ldg(xf + 1), r2 = __ldg(xf + 2);
  const float u0 = fmaf(r0.x, o.x, fmaf(r0.y, o.y, fmaf(r0.z, o.z, r0.w)));
  const float v0 = fmaf(r1.x, o.x, fmaf(r1.y, o.y, fmaf(r1.z, o.z, r1.w)));
  const float du = fmaf(r0.x, d.x, fmaf(r0.y, d.y, r0.z * d.z));
  const float dv = fmaf(r1.x, d.x, fmaf(r1.y, d.y, r1.z * d.z));
  const float A = fmaf(du, du, dv * dv);
  if (!(A > 0.f)) return false;
  const float inv = 1.0f / A;
  const float tc = -fmaf(u0, du, v0 * dv) * inv;
  const float uc = fmaf(tc, du, u0), vc = fmaf(tc, dv, v0);
  const float h2 = fmaf(uc, uc, vc * vc);
  if (h2 > 1.f) return false;
  const float half = sqrtf((1.f - h2) * inv);
  lo = tc - half;
  hi = tc + half;
  const float w0 = fmaf(r2.x, o.x, fmaf(r2.y, o.y, fmaf(r2.z, o.z, r2.w)));
  const float dw = fmaf(r2.x, d.x, fmaf(r2.y, d.y, r2.z * d.z));
  if (dw != 0.f) {
    const float idw = 1.0f / dw;
    const float ta = -w0 * idw, tb = (1.f - w0) * idw;
    lo = fmaxf(lo, fminf(ta, tb));
    hi = fminf(hi, fmaxf(ta, tb));
  } else if (w0 < 0.f || w0 > 1.f) {
    return false;
  }
  lo = fmaxf(lo, tmin);
  hi = fminf(hi, tmax);
  return hi > lo;
}

// Transmittance of the light path of dual scattering (readings as in the
// oracle): the shadow ray from x along wi up to tmax crosses hairs; every
// primitive of the shading hair itself (material row self_mat) is skipped; a
// strand segment counts one hair, a thick-hair segment rho l sqrt(n_tot /
// (pi a b)) for its chord l; each hair multiplies T by its forward albedo at
// incidence |asin(wi . t)| and adds its forward spread variance; T = d_F prod
// a_F^n (d_F = 0.7) once a hair is crossed.  The walk visits every box on the
// path (all crossings count) and stops early once T < 1e-7 in every channel,
// where the light's contribution is below FP32 resolution of the pixel.
constexpr float kDF = 0.7f;
template <int PREC, bool COUNT>
__device__ __forceinline__ void shadow_path(const FrameArgs& fa, const float3 x, const float3 wi,
                                            const float tmax, const uint32_t self_mat, float T[3],
                                            float& sg2, bool& ok, Counts& cn) {
  T[0] = T[1] = T[2] = 1.f;
  sg2 = 0.f;
  if (fa.n_prims == 0) return;
  float3 inv, ooi;
  ray_slabs(x, wi, inv, ooi);
  int stack[kStack];
  int sp = 0;
  int node = fa.n_prims == 1 ? ~(int)__ldg(fa.leaf_id) : 0;
  bool crossed = false;
  for (;;) {
    if (node >= 0) {
      const float4* nd = fa.nodes + 4 * (size_t)node;
      const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
      if (COUNT) ++cn.nodes;
      float lx = fmaf(n0.x, inv.x, -ooi.x), hx = fmaf(n0.y, inv.x, -ooi.x);
      float ly = fmaf(n0.z, inv.y, -ooi.y), hy = fmaf(n0.w, inv.y, -ooi.y);
      float lz = fmaf(n2.x, inv.z, -ooi.z), hz = fmaf(n2.y, inv.z, -ooi.z);
      const float a0 = fmaxf(fmaxf(fminf(lx, hx), fminf(ly, hy)), fmaxf(fminf(lz, hz), 0.f));
      const float b0 = fminf(fminf(fmaxf(lx, hx), fmaxf(ly, hy)), fminf(fmaxf(lz, hz), tmax));
      lx = fmaf(n1.x, inv.x, -ooi.x); hx = fmaf(n1.y, inv.x, -ooi.x);
      ly = fmaf(n1.z, inv.y, -ooi.y); hy = fmaf(n1.w, inv.y, -ooi.y);
      lz = fmaf(n2.z, inv.z, -ooi.z); hz = fmaf(n2.w, inv.z, -ooi.z);
      const float a1 = fmaxf(fmaxf(fminf(lx, hx), fminf(ly, hy)), fmaxf(fminf(lz, hz), 0.f));
      const float b1 = fminf(fminf(fmaxf(lx, hx), fmaxf(ly, hy)), fminf(fmaxf(lz, hz), tmax));
      const bool h0 = a0 <= b0, h1 = a1 <= b1;
      const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
      if (h0 && h1) {
        if (sp < kStack)
          stack[sp++] = c1;
        else
          ok = false;
        node = c0;
        continue;
      }
      if (h0 || h1) {
        node = h0 ? c0 : c1;
        continue;
      }
    } else {
      const uint32_t id = (uint32_t)(~node);
      const float4 aux = __ldg(fa.prim_aux + id);
      float lo, hi;
      if (COUNT) ++cn.tests;
      if (__float_as_uint(aux.x) != self_mat &&
          leaf_span(fa.prim_xf + 3 * (size_t)id, x, wi, 0.f, tmax, lo, hi)) {
        const float4 r2 = __ldg(fa.prim_xf + 3 * (size_t)id + 2);
        const float si = clampf(dot3(wi, f3(r2.x, r2.y, r2.z)) *
                                    rsqrtf(r2.x * r2.x + r2.y * r2.y + r2.z * r2.z),
                                -1.f, 1.f);
        Mat m;
        load_mat(fa.mat + (size_t)__float_as_uint(aux.x) * HR_MAT_FLOATS, m);
        float aF[3], s2;
        forward_albedo<PREC>(fa.tables, m, fabsf(asinf(si)), (fa.flags & HR_FLAG_TRT) != 0, aF, s2);
        if (aux.y > 0.f) {  // thick hair: its hair number over the chord
          const float ntot = aux.y, r = aux.z, ab = aux.w;
          const float rho = fminf(1.f, ntot * r * r / ab);
          const float n = rho * (hi - lo) * sqrtf(ntot / (kPi * ab));
#pragma unroll
          for (int c = 0; c < 3; ++c) T[c] *= exp2f(n * __log2f(aF[c]));
          sg2 = fmaf(n, s2, sg2);
        } else {
#pragma unroll
          for (int c = 0; c < 3; ++c) T[c] *= aF[c];
          sg2 += s2;
        }
        crossed = true;
        if (fmaxf(T[0], fmaxf(T[1], T[2])) < 1e-7f) break;
      }
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
  if (crossed) {
    T[0] *= kDF;
    T[1] *= kDF;
    T[2] *= kDF;
  }
}

// Radiance of one hit toward -d (sum over lights of T f E cos(theta_i), T and
// the spread of f from shadow_path when SHADOW (HR_FLAG_SHADOWS), else T = 1)
// and its opacity (strand 1; thick hair 1 - exp(-2 r l n_tot / (pi a b))).
// SHADOW is a template parameter so kernels without shadow rays carry none
// of their registers.
template <int PREC, bool COUNT, bool SHADOW = false>
__device__ __forceinline__ void shade_hit(const FrameArgs& fa, uint32_t id, float t,
                                          const float3 o, const float3 d, float rgb[3],
                                          float& alpha, Counts& cn) {
  const float4 aux = __ldg(fa.prim_aux + id);
  const float4 r2 = __ldg(fa.prim_xf + 3 * (size_t)id + 2);
  const float3 T = f3(r2.x, r2.y, r2.z) * rsqrtf(r2.x * r2.x + r2.y * r2.y + r2.z * r2.z);
  Mat m;
  load_mat(fa.mat + (size_t)__float_as_uint(aux.x) * HR_MAT_FLOATS, m);
  const float3 wo = d * -1.f;
  const float so = clampf(dot3(wo, T), -1.f, 1.f);
  const float th_o = asinf(so);
  const float3 wop = wo - T * so;
  const float nop = sqrtf(dot3(wop, wop));
  const float3 x = o + d * t;
  const bool eth = aux.y > 0.f && !(fa.flags & HR_FLAG_SINGLE_ON_ETH);
  EthHit eh{0.f, 1.f, 0.f, 0.f};
  alpha = 1.f;
  if (aux.y > 0.f) {
    // the chord: the ray's length inside the finite cylinder (0 when FP32
    // rounding puts a hit at the very outline outside it)
    float lo, hi;
    const float chord =
        leaf_span(fa.prim_xf + 3 * (size_t)id, o, d, -kInf, kInf, lo, hi) ? hi - lo : 0.f;
    const float ntot = aux.y, r = aux.z, ab = aux.w;
    eh.rho = fminf(1.f, ntot * r * r / ab);
    const float n_raw = eh.rho * chord * sqrtf(ntot / (kPi * ab));
    eh.n_view = fmaxf(1.f, n_raw);
    alpha = 1.f - __expf(-2.f * r * chord * ntot / (kPi * ab));
    eh.nF = erff(kPi / (2.f * 1.41421356f * m.gT));
    eh.nB = erff(kPi / (1.41421356f * m.gT)) - eh.nF;
  }
  rgb[0] = rgb[1] = rgb[2] = 0.f;
  for (int l = 0; l < fa.lights.n; ++l) {
    const float4 L = fa.lights.xyzw[l];
    float3 wi;
    float E = 1.f;
    if (L.w == 0.f) {
      wi = f3(L.x, L.y, L.z);
    } else {
      const float3 to = f3(L.x, L.y, L.z) - x;
      const float dd = dot3(to, to);
      const float id = rsqrtf(dd);
      wi = to * id;
      E = id * id;
    }
    const float si = clampf(dot3(wi, T), -1.f, 1.f);
    const float th_i = asinf(si);
    const float3 wip = wi - T * si;
    const float nip = sqrtf(dot3(wip, wip));
    const float cphi =
        (nip > 0.f && nop > 0.f) ? clampf(dot3(wip, wop) / (nip * nop), -1.f, 1.f) : 1.f;
    float Tl[3] = {1.f, 1.f, 1.f}, sg2 = 0.f;
    if (SHADOW) {
      bool sok = true;
      shadow_path<PREC, COUNT>(fa, x, wi, L.w == 0.f ? kInf : sqrtf(1.f / E),
                               __float_as_uint(aux.x), Tl, sg2, sok, cn);
      if (!sok) atomicAdd(fa.overflow, 1u);
    }
    float f[3];
    if (eth) {
      f_ours<PREC>(fa.tables, m, eh, th_i, th_o, cphi, fa.flags, sg2, f);
      if (COUNT) ++cn.eshade;
    } else {
      f_single<PREC>(fa.tables, m, th_i, th_o, cphi, sg2, (fa.flags & HR_FLAG_TRT) != 0, f);
      if (COUNT) ++cn.sshade;
    }
    const float g = E * sqrtf(fmaxf(0.f, 1.f - si * si));
    const float4 Lc = fa.lights.rgb[l];
    rgb[0] = fmaf(f[0] * Tl[0] * g, Lc.x, rgb[0]);
    rgb[1] = fmaf(f[1] * Tl[1] * g, Lc.y, rgb[1]);
    rgb[2] = fmaf(f[2] * Tl[2] * g, Lc.z, rgb[2]);
  }
}

// One sample: ray, K nearest hits, shading and front-to-back compositing.
template <int KMAX, int PREC, bool COUNT, bool SHADOW = false>
__device__ __forceinline__ void render_ray(const FrameArgs& fa, const RayKey& rk, const float3 o,
                                           const float3 d, float out[3], int32_t* ids, bool& ok,
                                           Counts& cn) {
  KBuf<KMAX> kb;
  ok = traverse<KMAX, COUNT>(fa, rk, o, d, kb, cn);
  float T = 1.f;
  out[0] = out[1] = out[2] = 0.f;
  if (ids) {  // the composited hits: none after the first opaque (strand) one
    bool past = false;
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < (int)fa.k) {
        const bool live = kb.t[j] < kInf && !past;
        ids[j] = live ? (int32_t)(kb.id[j] & kIdMask) : -1;
        if (live && (kb.id[j] & kOpaque)) past = true;
      }
  }
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    if (j < (int)fa.k && kb.t[j] < kInf && T > 0.f) {
      float rgb[3], a;
      shade_hit<PREC, COUNT, SHADOW>(fa, kb.id[j] & kIdMask, kb.t[j], o, d, rgb, a, cn);
      if (COUNT) ++cn.hits;
      const float ta = T * a;
      out[0] = fmaf(ta, rgb[0], out[0]);
      out[1] = fmaf(ta, rgb[1], out[1]);
      out[2] = fmaf(ta, rgb[2], out[2]);
      T *= 1.f - a;
    }
  }
}

template <int KMAX, int PREC, bool COUNT, bool SHADOW = false>
__device__ __forceinline__ void render_sample(const FrameArgs& fa, uint64_t sid, float out[3],
                                              int32_t* ids, bool& ok, Counts& cn) {
  RayKey rk;
  float3 o, d;
  primary_ray(fa, sid, o, d, rk);
  render_ray<KMAX, PREC, COUNT, SHADOW>(fa, rk, o, d, out, ids, ok, cn);
}

__device__ __forceinline__ void flush_counts(const FrameArgs& fa, const Counts& cn) {
  unsigned long long v[8] = {cn.nodes, cn.tests, cn.sshade, cn.eshade, cn.hits, cn.rays,
                             cn.precise_tests, cn.precise_entries};
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    unsigned long long x = v[i];
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(fa.counters + i, x);
  }
}

// Pixel-space rectangle (x0, y0, x1, y1) that contains the projection of the
// BVH root box, grown by one pixel; computed by one warp (lanes 0-7 project
// the box corners) and stored by lane 0.  A pixel whose square lies outside it
// cannot see any primitive.  The whole screen when the box reaches behind the
// eye or the BVH has fewer than two leaves.
__device__ __forceinline__ void scene_rect_warp(const FrameArgs& fa, float4* rect) {
  {
    const int lane = threadIdx.x & 31;
    float X0 = kInf, Y0 = kInf, X1 = -kInf, Y1 = -kInf;
    bool ok = fa.n_prims >= 2;
    if (ok && lane < 8) {
      const float4 n0 = __ldg(fa.nodes), n1 = __ldg(fa.nodes + 1), n2 = __ldg(fa.nodes + 2);
      const float3 p = f3((lane & 1) ? fmaxf(n0.y, n1.y) : fminf(n0.x, n1.x),
                          (lane & 2) ? fmaxf(n0.w, n1.w) : fminf(n0.z, n1.z),
                          (lane & 4) ? fmaxf(n2.y, n2.w) : fminf(n2.x, n2.z));
      const float3 r = p - fa.cam.eye;
      const float xc = dot3(r, fa.cam.right), yc = dot3(r, fa.cam.up), zc = dot3(r, fa.cam.fwd);
      float X, Y;
      if (fa.cam.kind == 1) {
        ok = zc > 1e-6f;
        X = xc / zc * fa.cam.pix;
        Y = -yc / zc * fa.cam.pix;
      } else {
        X = xc * fa.cam.pix;
        Y = -yc * fa.cam.pix;
      }
      X += 0.5f * (float)fa.cam.W;
      Y += 0.5f * (float)fa.cam.H;
      if (!(X == X) || !(Y == Y)) ok = false;
      X0 = X1 = X;
      Y0 = Y1 = Y;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      X0 = fminf(X0, __shfl_xor_sync(0xffffffffu, X0, o));
      Y0 = fminf(Y0, __shfl_xor_sync(0xffffffffu, Y0, o));
      X1 = fmaxf(X1, __shfl_xor_sync(0xffffffffu, X1, o));
      Y1 = fmaxf(Y1, __shfl_xor_sync(0xffffffffu, Y1, o));
    }
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0)
      *rect = ok ? make_float4(X0 - 1.f, Y0 - 1.f, X1 + 1.f, Y1 + 1.f)
                 : make_float4(-kInf, -kInf, kInf, kInf);
  }
}

// Warp tile: the 32 / grp pixels one warp renders (wtw x wth); a pixel's
// samples on `grp` adjacent lanes.  tile_partials traces a lane's samples and
// returns their sum in sample order, for the lanes in `lanes` (the others
// return zeros).  tile_write sums a pixel's lanes with a fixed
// XOR-shuffle tree and stores the mean.  Both are called by whole warps.
template <int KMAX, int PREC, bool COUNT, bool SHADOW = false>
__device__ __forceinline__ void tile_partials(const FrameArgs& fa, uint32_t x0, uint32_t y0,
                                              uint32_t wtw, const float4 rect, uint32_t lanes,
                                              float acc[3], Counts& cn, bool& overflow) {
  const uint32_t G = fa.grp;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t lane_g = lane & (G - 1);
  const uint32_t p = lane / G;
  const uint32_t x = x0 + p % wtw, y = y0 + p / wtw;
  const bool valid = x < (uint32_t)fa.cam.W && y < (uint32_t)fa.cam.H;
  const bool inside = valid && (float)x + 1.f >= rect.x && (float)x <= rect.z &&
                      (float)y + 1.f >= rect.y && (float)y <= rect.w && ((lanes >> lane) & 1u);
  const uint64_t pixel = (uint64_t)y * (uint32_t)fa.cam.W + x;
  acc[0] = acc[1] = acc[2] = 0.f;
  if (inside) {
    for (uint32_t s = lane_g; s < fa.spp; s += G) {
      float v[3];
      bool ok;
      RayKey rk;
      float3 o, d;
      primary_ray(fa, pixel * fa.spp + s, o, d, rk);
      render_ray<KMAX, PREC, COUNT, SHADOW>(fa, rk, o, d, v, nullptr, ok, cn);
      if (COUNT) ++cn.rays;
      overflow |= !ok;
      acc[0] += v[0];
      acc[1] += v[1];
      acc[2] += v[2];
    }
  }
}

__device__ __forceinline__ void tile_write(const FrameArgs& fa, uint32_t x0, uint32_t y0,
                                           uint32_t wtw, const float4 rect, float acc[3],
                                           float* __restrict__ rgb) {
  const uint32_t G = fa.grp;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t p = lane / G;
  const uint32_t x = x0 + p % wtw, y = y0 + p / wtw;
  const bool valid = x < (uint32_t)fa.cam.W && y < (uint32_t)fa.cam.H;
  const bool inside = valid && (float)x + 1.f >= rect.x && (float)x <= rect.z &&
                      (float)y + 1.f >= rect.y && (float)y <= rect.w;
  const uint64_t pixel = (uint64_t)y * (uint32_t)fa.cam.W + x;
  for (uint32_t o = 1; o < G; o <<= 1) {
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
    acc[1] += __shfl_xor_sync(0xffffffffu, acc[1], o);
    acc[2] += __shfl_xor_sync(0xffffffffu, acc[2], o);
  }
  if (inside && (lane & (G - 1)) == 0) {
    const float inv = 1.0f / (float)fa.spp;
    rgb[3 * pixel] = acc[0] * inv;
    rgb[3 * pixel + 1] = acc[1] * inv;
    rgb[3 * pixel + 2] = acc[2] * inv;
  }
}

template <int KMAX, int PREC, bool COUNT, bool SHADOW = false>
__device__ __forceinline__ void render_warp_tile(const FrameArgs& fa, uint32_t x0, uint32_t y0,
                                                 uint32_t wtw, const float4 rect,
                                                 float* __restrict__ rgb, Counts& cn,
                                                 bool& overflow) {
  float acc[3];
  tile_partials<KMAX, PREC, COUNT, SHADOW>(fa, x0, y0, wtw, rect, 0xffffffffu, acc, cn, overflow);
  tile_write(fa, x0, y0, wtw, rect, acc, rgb);
}

}  // namespace tr
}  // namespace hr
