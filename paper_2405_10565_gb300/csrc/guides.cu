// Guide hairs, the guide-driven hierarchy and linear skinning (Section 5.1
// steps 1, 2 and 4; Section 5.2 "Runtime").
//
//  * Guides: k-means over the strands with D(i, j) = sum_k |p^{i,k} -
//    p^{j,k}|^2 over corresponding vertices, each cluster's guide its medoid
//    (the member with the smallest sum of distances to the others).
//  * Hierarchy: every strand's three nearest guides; strands sharing the same
//    three form one cluster of the coarsest level, listed in (Morton code of
//    the root, id) order; finer levels, fits and records as for the Morton
//    hierarchy.
//  * Skinning: every strand vertex and every thick-hair cross-section centre
//    and corner (c +- a e1, c +- b e2) gets weights in the triangular prism
//    of its cluster's three guides' corresponding points, p = g0 + w1 (g1 -
//    g0) + w2 (g2 - g0) + h n (n the unit normal of the triangle; a
//    degenerate triangle keeps the offset p - g0).  A new pose of the guides
//    moves the strands and the thick hairs without a new clustering or fit.
//
// D, the centroid sums and the medoid sums are FP32 without contraction, in
// vertex order and, over members, in ascending strand id: the decisions they
// make (cluster ids, medoids, nearest guides) are reproducible and compare bit
// for bit with a plain FP32 evaluation in that order.  The prism weights are
// FP64 (once per hierarchy), the skinning FP32 (every frame).
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace hr {
namespace {

constexpr uint32_t kMaxGuides = 1024;  // three guide indices of 10 bits in one key

// One vertex's term of D: ((dx dx + dy dy) + dz dz), each operation rounded.
__device__ __forceinline__ float point_d(const float4 a, const float4 b) {
  const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ __forceinline__ float strand_d(const float4* __restrict__ A, const float4* __restrict__ B,
                                          uint32_t S1) {
  float d = 0.f;
  for (uint32_t k = 0; k < S1; ++k) d = __fadd_rn(d, point_d(__ldg(A + k), __ldg(B + k)));
  return d;
}

__global__ void k_seed(const float4* __restrict__ verts, uint32_t S1, const uint32_t* __restrict__ order,
                       uint32_t N, uint32_t G, float4* cent) {
  const uint32_t g = blockIdx.x;
  const uint32_t s = order[(uint32_t)(((uint64_t)(2 * g + 1) * N) / (2ull * G))];
  for (uint32_t k = threadIdx.x; k < S1; k += blockDim.x) {
    const float4 p = verts[(size_t)s * S1 + k];
    cent[(size_t)g * S1 + k] = make_float4(p.x, p.y, p.z, 0.f);
  }
}

// Nearest centroid of every strand (ties: the lower cluster).  Eight
// centroids at a time, each D accumulated over the vertices in order.
__global__ void k_assign(const float4* __restrict__ verts, uint32_t N, uint32_t S1,
                         const float4* __restrict__ cent, uint32_t G, uint32_t* assign) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float4* P = verts + (size_t)i * S1;
  float best = __int_as_float(0x7f800000);
  uint32_t bg = 0;
  for (uint32_t g0 = 0; g0 < G; g0 += 8) {
    float d[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (uint32_t k = 0; k < S1; ++k) {
      const float4 p = __ldg(P + k);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (g0 + j < G) d[j] = __fadd_rn(d[j], point_d(p, __ldg(cent + (size_t)(g0 + j) * S1 + k)));
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (g0 + j < G && d[j] < best) {
        best = d[j];
        bg = g0 + j;
      }
  }
  assign[i] = bg;
}

__global__ void k_count(const uint32_t* __restrict__ key, uint32_t n, uint32_t* counts) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(counts + key[i], 1u);
}

__global__ void k_iota_copy(const uint32_t* __restrict__ src, uint32_t n, uint32_t* keys,
                            uint32_t* vals) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = src[i];
  vals[i] = i;
}

// Centroid of every cluster: the members' vertices summed in ascending strand
// id (FP32), divided by the count; an empty cluster keeps its centroid.
__global__ void k_update(const float4* __restrict__ verts, uint32_t S1,
                         const uint32_t* __restrict__ start, const uint32_t* __restrict__ ids,
                         float4* cent) {
  const uint32_t g = blockIdx.x;
  const uint32_t r0 = start[g], r1 = start[g + 1];
  if (r1 == r0) return;
  const float* V = reinterpret_cast<const float*>(verts);
  float* Cg = reinterpret_cast<float*>(cent + (size_t)g * S1);
  for (uint32_t j = threadIdx.x; j < S1 * 3; j += blockDim.x) {
    const uint32_t k = j / 3, c = j % 3;
    float acc = 0.f;
    for (uint32_t r = r0; r < r1; ++r) acc = __fadd_rn(acc, __ldg(V + ((size_t)ids[r] * S1 + k) * 4 + c));
    Cg[k * 4 + c] = __fdiv_rn(acc, (float)(r1 - r0));
  }
}

// Medoid of every cluster: the member whose sum of D to the members (in
// ascending id) is least; ties to the lower strand id; -1 for an empty cluster.
__global__ void k_medoid(const float4* __restrict__ verts, uint32_t S1,
                         const uint32_t* __restrict__ start, const uint32_t* __restrict__ ids,
                         int32_t* guides) {
  const uint32_t g = blockIdx.x;
  const uint32_t r0 = start[g], r1 = start[g + 1];
  __shared__ float s_v[32];
  __shared__ uint32_t s_i[32];
  float bv = __int_as_float(0x7f800000);
  uint32_t bi = 0xffffffffu;
  for (uint32_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const uint32_t i = ids[r];
    const float4* Pi = verts + (size_t)i * S1;
    float s = 0.f;
    for (uint32_t q = r0; q < r1; ++q) s = __fadd_rn(s, strand_d(Pi, verts + (size_t)ids[q] * S1, S1));
    if (s < bv || (s == bv && i < bi)) {
      bv = s;
      bi = i;
    }
  }
  for (int o = 16; o; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const uint32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov < bv || (ov == bv && oi < bi)) {
      bv = ov;
      bi = oi;
    }
  }
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    s_v[w] = bv;
    s_i[w] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (uint32_t k = 1; k < (blockDim.x + 31) / 32; ++k)
      if (s_v[k] < bv || (s_v[k] == bv && s_i[k] < bi)) {
        bv = s_v[k];
        bi = s_i[k];
      }
    guides[g] = r1 > r0 ? (int32_t)bi : -1;
  }
}

// The three nearest guides of every strand (ties: the lower guide), as a key
// of three ascending 10-bit guide indices, for the strands in Morton order.
__global__ void k_nearest3(const float4* __restrict__ verts, uint32_t N, uint32_t S1,
                           const int32_t* __restrict__ guides, uint32_t G,
                           const uint32_t* __restrict__ morton_order, uint32_t* key) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const uint32_t i = morton_order[r];
  const float4* P = verts + (size_t)i * S1;
  const float inf = __int_as_float(0x7f800000);
  float b0 = inf, b1 = inf, b2 = inf;
  uint32_t g0 = 0, g1 = 0, g2 = 0;
  for (uint32_t g = 0; g < G; ++g) {
    const int32_t s = __ldg(guides + g);
    if (s < 0) continue;
    const float d = strand_d(P, verts + (size_t)s * S1, S1);
    if (d < b2) {
      if (d < b1) {
        b2 = b1;
        g2 = g1;
        if (d < b0) {
          b1 = b0;
          g1 = g0;
          b0 = d;
          g0 = g;
        } else {
          b1 = d;
          g1 = g;
        }
      } else {
        b2 = d;
        g2 = g;
      }
    }
  }
  // ascending guide indices
  uint32_t x = g0, y = g1, z = g2, t;
  if (x > y) t = x, x = y, y = t;
  if (y > z) t = y, y = z, z = t;
  if (x > y) t = x, x = y, y = t;
  key[r] = (x << 20) | (y << 10) | z;
}

// Cluster starts from the ranks where the sorted key changes (excl = the
// exclusive scan of those flags); the number of clusters into *C.
__global__ void k_starts(const uint32_t* __restrict__ key, const uint32_t* __restrict__ excl,
                         uint32_t N, uint32_t* cl_first, uint32_t* cl_tri, uint32_t* C) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const bool head = r == 0 || key[r] != key[r - 1];
  if (head) {
    cl_first[excl[r]] = r;
    cl_tri[excl[r]] = key[r];
  }
  if (r == N - 1) {
    const uint32_t n = excl[r] + (head ? 1u : 0u);
    cl_first[n] = N;
    *C = n;
  }
}

__global__ void k_head_flags(const uint32_t* __restrict__ key, uint32_t N, uint32_t* flags) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < N) flags[r] = (r == 0 || key[r] != key[r - 1]) ? 1u : 0u;
}

// ---------------------------------------------------------------- prism weights

struct D3 {
  double x, y, z;
};
__device__ __forceinline__ D3 d3(const float4 p) { return D3{p.x, p.y, p.z}; }
__device__ __forceinline__ D3 dsub(D3 a, D3 b) { return D3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double ddot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 dcross(D3 a, D3 b) {
  return D3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// (w1, w2, h, 0) of p in the prism of (g0, g1, g2), or (offset from g0, 1)
// for a degenerate triangle (|e1 x e2| <= 1e-6 |e1| |e2|).
__device__ float4 prism_weights(const D3 p, const D3 g0, const D3 g1, const D3 g2) {
  const D3 e1 = dsub(g1, g0), e2 = dsub(g2, g0);
  const D3 n = dcross(e1, e2);
  const double nn = sqrt(ddot(n, n));
  const double scale = sqrt(ddot(e1, e1)) * sqrt(ddot(e2, e2));
  const D3 q = dsub(p, g0);
  if (!(nn > 1e-6 * scale)) return make_float4((float)q.x, (float)q.y, (float)q.z, 1.f);
  const D3 nh{n.x / nn, n.y / nn, n.z / nn};
  const double h = ddot(q, nh);
  const D3 qp{q.x - h * nh.x, q.y - h * nh.y, q.z - h * nh.z};
  const double w1 = ddot(dcross(qp, e2), nh) / nn;
  const double w2 = ddot(dcross(e1, qp), nh) / nn;
  return make_float4((float)w1, (float)w2, (float)h, 0.f);
}

__device__ __forceinline__ void tri_of(uint32_t key, uint32_t& a, uint32_t& b, uint32_t& c) {
  a = key >> 20;
  b = (key >> 10) & 1023u;
  c = key & 1023u;
}

// Weights of every strand vertex in its cluster's guide prism.
__global__ void k_strand_weights(const float4* __restrict__ verts, uint32_t N, uint32_t S1,
                                 const uint32_t* __restrict__ cluster_of,
                                 const uint32_t* __restrict__ cl_tri,
                                 const int32_t* __restrict__ guides, float4* w) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (uint64_t)N * S1) return;
  const uint32_t i = (uint32_t)(idx / S1), k = (uint32_t)(idx % S1);
  uint32_t ga, gb, gc;
  tri_of(cl_tri[cluster_of[i]], ga, gb, gc);
  const float4* V = verts;
  w[idx] = prism_weights(d3(V[idx]), d3(V[(size_t)guides[ga] * S1 + k]),
                         d3(V[(size_t)guides[gb] * S1 + k]), d3(V[(size_t)guides[gc] * S1 + k]));
}

__device__ __forceinline__ uint32_t eth_cluster(uint32_t e, const uint32_t* off, uint32_t L) {
  uint32_t k = 0;
  while (k + 1 < L && e >= off[k + 1]) ++k;
  return (e - off[k]) >> (2 * k);
}

struct Offs {
  uint32_t n_levels;
  uint32_t off[16];
};

// Weights of every thick-hair cross-section's centre and four corners.
__global__ void k_eth_weights(const float4* __restrict__ verts, uint32_t S1,
                              const float4* __restrict__ xsec, uint32_t E, Offs lv,
                              const uint32_t* __restrict__ cl_tri,
                              const int32_t* __restrict__ guides, float4* w) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (uint64_t)E * S1) return;
  const uint32_t e = (uint32_t)(idx / S1), k = (uint32_t)(idx % S1);
  const float4 c = xsec[idx * 3], q1 = xsec[idx * 3 + 1], q2 = xsec[idx * 3 + 2];
  float4* o = w + idx * 5;
  if (!(c.w > 0.f)) {  // empty thick hair
    for (int j = 0; j < 5; ++j) o[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  uint32_t ga, gb, gc;
  tri_of(cl_tri[eth_cluster(e, lv.off, lv.n_levels)], ga, gb, gc);
  const D3 g0 = d3(verts[(size_t)guides[ga] * S1 + k]), g1 = d3(verts[(size_t)guides[gb] * S1 + k]),
           g2 = d3(verts[(size_t)guides[gc] * S1 + k]);
  const double a = c.w, b = q1.w;
  const D3 cc{c.x, c.y, c.z};
  const D3 pts[5] = {cc,
                     D3{cc.x + a * q1.x, cc.y + a * q1.y, cc.z + a * q1.z},
                     D3{cc.x - a * q1.x, cc.y - a * q1.y, cc.z - a * q1.z},
                     D3{cc.x + b * q2.x, cc.y + b * q2.y, cc.z + b * q2.z},
                     D3{cc.x - b * q2.x, cc.y - b * q2.y, cc.z - b * q2.z}};
  for (int j = 0; j < 5; ++j) o[j] = prism_weights(pts[j], g0, g1, g2);
}

// ---------------------------------------------------------------- skinning (FP32)

__device__ __forceinline__ float3 skin(const float4 w, const float4 g0, const float4 g1,
                                       const float4 g2) {
  if (w.w > 0.5f) return make_float3(g0.x + w.x, g0.y + w.y, g0.z + w.z);
  const float3 e1 = make_float3(g1.x - g0.x, g1.y - g0.y, g1.z - g0.z);
  const float3 e2 = make_float3(g2.x - g0.x, g2.y - g0.y, g2.z - g0.z);
  float3 n = make_float3(e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z,
                         e1.x * e2.y - e1.y * e2.x);
  const float nn = sqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
  const float inv = nn > 0.f ? 1.f / nn : 0.f;
  n = make_float3(n.x * inv, n.y * inv, n.z * inv);
  return make_float3(g0.x + w.x * e1.x + w.y * e2.x + w.z * n.x,
                     g0.y + w.x * e1.y + w.y * e2.y + w.z * n.y,
                     g0.z + w.x * e1.z + w.y * e2.z + w.z * n.z);
}

// New strand vertices from the guides' new vertices gv [G][S1] (radius kept).
__global__ void k_skin_strands(const float4* __restrict__ gv, uint32_t N, uint32_t S1,
                               const uint32_t* __restrict__ cluster_of,
                               const uint32_t* __restrict__ cl_tri,
                               const float4* __restrict__ w, float4* verts) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (uint64_t)N * S1) return;
  const uint32_t i = (uint32_t)(idx / S1), k = (uint32_t)(idx % S1);
  uint32_t ga, gb, gc;
  tri_of(cl_tri[cluster_of[i]], ga, gb, gc);
  const float3 p = skin(w[idx], __ldg(gv + (size_t)ga * S1 + k), __ldg(gv + (size_t)gb * S1 + k),
                        __ldg(gv + (size_t)gc * S1 + k));
  verts[idx] = make_float4(p.x, p.y, p.z, verts[idx].w);
}

// New thick-hair cross-sections from the skinned centre and corners: a and
// e1 from the corners c +- a e1, b and e2 from c +- b e2.
__global__ void k_skin_eth(const float4* __restrict__ gv, uint32_t S1, uint32_t E, Offs lv,
                           const uint32_t* __restrict__ cl_tri, const float4* __restrict__ w,
                           float4* xsec) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (uint64_t)E * S1) return;
  if (!(xsec[idx * 3].w > 0.f)) return;  // empty thick hair
  const uint32_t e = (uint32_t)(idx / S1), k = (uint32_t)(idx % S1);
  uint32_t ga, gb, gc;
  tri_of(cl_tri[eth_cluster(e, lv.off, lv.n_levels)], ga, gb, gc);
  const float4 g0 = __ldg(gv + (size_t)ga * S1 + k), g1 = __ldg(gv + (size_t)gb * S1 + k),
               g2 = __ldg(gv + (size_t)gc * S1 + k);
  float3 p[5];
  for (int j = 0; j < 5; ++j) p[j] = skin(w[idx * 5 + j], g0, g1, g2);
  const float3 u = make_float3(p[1].x - p[2].x, p[1].y - p[2].y, p[1].z - p[2].z);
  const float3 v = make_float3(p[3].x - p[4].x, p[3].y - p[4].y, p[3].z - p[4].z);
  const float lu = sqrtf(u.x * u.x + u.y * u.y + u.z * u.z);
  const float lv_ = sqrtf(v.x * v.x + v.y * v.y + v.z * v.z);
  const float iu = lu > 0.f ? 1.f / lu : 0.f, iv = lv_ > 0.f ? 1.f / lv_ : 0.f;
  xsec[idx * 3] = make_float4(p[0].x, p[0].y, p[0].z, 0.5f * lu);
  xsec[idx * 3 + 1] = make_float4(u.x * iu, u.y * iu, u.z * iu, 0.5f * lv_);
  xsec[idx * 3 + 2] = make_float4(v.x * iv, v.y * iv, v.z * iv, 0.f);
}

unsigned blocks_for(uint64_t n, unsigned b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

void drop_guides(hr_ctx* ctx, hr_asset* a) {
  const size_t S1 = a->S + 1;
  if (a->guides) dfree(ctx, a->guides, (size_t)a->G * 4);
  if (a->cl_tri) dfree(ctx, a->cl_tri, (size_t)a->guided_C * 4);
  if (a->w_strand) dfree(ctx, a->w_strand, (size_t)a->N * S1 * sizeof(float4));
  if (a->w_eth) dfree(ctx, a->w_eth, (size_t)a->guided_E * S1 * 5 * sizeof(float4));
  a->guides = nullptr;
  a->cl_tri = nullptr;
  a->w_strand = nullptr;
  a->w_eth = nullptr;
  a->G = 0;
  a->guided_C = a->guided_E = 0;
}

hr_status build_guided_hierarchy(hr_ctx* ctx, hr_asset* a, uint32_t G, uint32_t iters,
                                 uint32_t max_levels) {
  cudaStream_t st = ctx_stream(ctx);
  const uint32_t N = a->N, S1 = a->S + 1;
  if (G < 3 || G > kMaxGuides || G > N)
    return set_error(ctx, HR_EINVAL, "n_guides must be in 3..min(1024, n_strands)");
  drop_guides(ctx, a);
  // scratch: Morton order and codes, keys / values and their temporaries,
  // the assignment, counts and starts, centroids
  uint32_t *order, *codes, *kk, *vv, *k2, *v2, *assign, *start, *dC;
  float4* cent;
  HR_TRY(scratch(ctx, 52, (size_t)N * 4, (void**)&order));
  HR_TRY(scratch(ctx, 53, (size_t)N * 4, (void**)&codes));
  HR_TRY(scratch(ctx, 54, (size_t)N * 4, (void**)&kk));
  HR_TRY(scratch(ctx, 55, (size_t)N * 4, (void**)&vv));
  HR_TRY(scratch(ctx, 56, (size_t)N * 4, (void**)&k2));
  HR_TRY(scratch(ctx, 57, (size_t)N * 4, (void**)&v2));
  HR_TRY(scratch(ctx, 58, (size_t)N * 4, (void**)&assign));
  HR_TRY(scratch(ctx, 59, ((size_t)std::max(G, N) + 2) * 4, (void**)&start));
  HR_TRY(scratch(ctx, 60, (size_t)G * S1 * sizeof(float4) + 16, (void**)&cent));
  HR_TRY(scratch(ctx, 61, 16, (void**)&dC));
  int32_t* guides = nullptr;
  HR_TRY(dalloc(ctx, (void**)&guides, (size_t)G * 4, "guides"));
  a->guides = guides;
  a->G = G;
  HR_TRY(root_morton_order(ctx, a, codes, order, st));
  int bits = 1;
  while ((1u << bits) < G) ++bits;
  // the members of every cluster in ascending strand id, and the starts
  auto members = [&]() -> hr_status {
    k_iota_copy<<<blocks_for(N, 256), 256, 0, st>>>(assign, N, kk, vv);
    HR_LAUNCHED(ctx);
    HR_TRY(radix_sort_pairs(ctx, kk, vv, k2, v2, N, bits, st));
    HR_CUDA(ctx, cudaMemsetAsync(start, 0, ((size_t)G + 1) * 4, st));
    k_count<<<blocks_for(N, 256), 256, 0, st>>>(assign, N, start);
    HR_LAUNCHED(ctx);
    return scan_u32(ctx, start, G + 1, st);
  };
  k_seed<<<G, 64, 0, st>>>(a->verts, S1, order, N, G, cent);
  HR_LAUNCHED(ctx);
  for (uint32_t it = 0; it < iters; ++it) {
    k_assign<<<blocks_for(N, 128), 128, 0, st>>>(a->verts, N, S1, cent, G, assign);
    HR_LAUNCHED(ctx);
    HR_TRY(members());
    k_update<<<G, 256, 0, st>>>(a->verts, S1, start, vv, cent);
    HR_LAUNCHED(ctx);
  }
  k_assign<<<blocks_for(N, 128), 128, 0, st>>>(a->verts, N, S1, cent, G, assign);
  HR_LAUNCHED(ctx);
  HR_TRY(members());
  k_medoid<<<G, 256, 0, st>>>(a->verts, S1, start, vv, guides);
  HR_LAUNCHED(ctx);
  // at least three guides
  std::vector<int32_t> gh(G);
  HR_CUDA(ctx, cudaMemcpyAsync(gh.data(), guides, (size_t)G * 4, cudaMemcpyDeviceToHost, st));
  HR_CUDA(ctx, cudaStreamSynchronize(st));
  uint32_t n_valid = 0;
  for (int32_t g : gh) n_valid += g >= 0;
  if (n_valid < 3) return set_error(ctx, HR_EINVAL, "fewer than three non-empty guide clusters");
  // three nearest guides of every strand (Morton order), then the strands by
  // (key, Morton code, id): a stable sort of the keys of the Morton order
  k_nearest3<<<blocks_for(N, 128), 128, 0, st>>>(a->verts, N, S1, guides, G, order, kk);
  HR_LAUNCHED(ctx);
  HR_CUDA(ctx, cudaMemcpyAsync(vv, order, (size_t)N * 4, cudaMemcpyDeviceToDevice, st));
  HR_TRY(radix_sort_pairs(ctx, kk, vv, k2, v2, N, 30, st));
  // cluster starts where the key changes
  k_head_flags<<<blocks_for(N, 256), 256, 0, st>>>(kk, N, assign);
  HR_LAUNCHED(ctx);
  HR_TRY(scan_u32(ctx, assign, N, st));
  uint32_t* cl_tri_tmp = k2;  // [C <= N]
  k_starts<<<blocks_for(N, 256), 256, 0, st>>>(kk, assign, N, start, cl_tri_tmp, dC);
  HR_LAUNCHED(ctx);
  uint32_t C = 0;
  HR_CUDA(ctx, cudaMemcpyAsync(&C, dC, 4, cudaMemcpyDeviceToHost, st));
  HR_CUDA(ctx, cudaStreamSynchronize(st));
  HR_TRY(build_hierarchy_from(ctx, a, C, max_levels, vv, start));
  // the hierarchy's arrays are set: the guide state for skinning
  HR_TRY(dalloc(ctx, (void**)&a->cl_tri, (size_t)C * 4, "cluster guides"));
  a->guided_C = C;
  HR_CUDA(ctx, cudaMemcpyAsync(a->cl_tri, cl_tri_tmp, (size_t)C * 4, cudaMemcpyDeviceToDevice, st));
  HR_TRY(dalloc(ctx, (void**)&a->w_strand, (size_t)N * S1 * sizeof(float4), "strand weights"));
  k_strand_weights<<<blocks_for((uint64_t)N * S1, 128), 128, 0, st>>>(a->verts, N, S1, a->cluster_of,
                                                                      a->cl_tri, guides, a->w_strand);
  HR_LAUNCHED(ctx);
  if (a->E) {
    HR_TRY(dalloc(ctx, (void**)&a->w_eth, (size_t)a->E * S1 * 5 * sizeof(float4), "thick-hair weights"));
    a->guided_E = a->E;
    Offs lv{};
    lv.n_levels = a->n_levels;
    for (uint32_t k = 0; k <= a->n_levels && k < 16; ++k) lv.off[k] = a->eth_offset[k];
    k_eth_weights<<<blocks_for((uint64_t)a->E * S1, 128), 128, 0, st>>>(a->verts, S1, a->xsec, a->E, lv,
                                                                        a->cl_tri, guides, a->w_eth);
    HR_LAUNCHED(ctx);
  }
  return HR_OK;
}

hr_status skin_asset(hr_ctx* ctx, hr_asset* a, const float4* gv_dev) {
  cudaStream_t st = ctx_stream(ctx);
  const uint32_t N = a->N, S1 = a->S + 1;
  k_skin_strands<<<blocks_for((uint64_t)N * S1, 256), 256, 0, st>>>(gv_dev, N, S1, a->cluster_of,
                                                                   a->cl_tri, a->w_strand, a->verts);
  HR_LAUNCHED(ctx);
  HR_TRY(refresh_strand_prims(ctx, a));
  if (a->E) {
    Offs lv{};
    lv.n_levels = a->n_levels;
    for (uint32_t k = 0; k <= a->n_levels && k < 16; ++k) lv.off[k] = a->eth_offset[k];
    k_skin_eth<<<blocks_for((uint64_t)a->E * S1, 256), 256, 0, st>>>(gv_dev, S1, a->E, lv, a->cl_tri,
                                                                    a->w_eth, a->xsec);
    HR_LAUNCHED(ctx);
    HR_TRY(rebuild_eth_records(ctx, a));
  }
  a->bvh.valid = 0;
  return HR_OK;
}

}  // namespace hr
