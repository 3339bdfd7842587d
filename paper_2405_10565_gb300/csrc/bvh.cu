// Active-primitive compaction and linear BVH build.
//
// Compaction ("hair data reorganisation", Section 6 "Real-time performance"):
// a cluster at the strand level contributes every segment of its member
// strands, a cluster at level L contributes every segment of its level-L
// thick hairs.  Per-cluster counts are scanned and each cluster's block writes
// its global primitive ids.
//
// LBVH (Karras 2012, "Maximizing parallelism in the construction of BVHs,
// octrees, and k-d trees"): 21-bit Morton codes (7 bits per axis) of the
// primitive box centroids in the strand boxes' bounds, stable single-sweep
// radix sort of (code, position in the active list), one thread per internal
// node finds its key range and split from the longest common prefix (ties
// between equal codes broken by index).  Bounds go bottom-up in two kernels:
// k_gather_refit copies the leaf records into Morton order and finishes the
// nodes whose leaf range lies inside its thread block's leaves (nearly all of
// them) in barrier-separated rounds in shared memory; k_climb finishes the few
// nodes that span blocks by float atomic min / max from each climb start.
//
// Node layout (4 x float4 = 64 bytes), children's boxes stored in the parent:
//   n0 = (lo0.x, hi0.x, lo0.y, hi0.y)  n1 = (lo1.x, hi1.x, lo1.y, hi1.y)
//   n2 = (lo0.z, hi0.z, lo1.z, hi1.z)  n3 = (child0, child1, -, -) as int bits
// A child index >= 0 is an internal node, < 0 is leaf ~index.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace hr {
namespace {

// Active primitives per cluster, and the thick-hair total in counts[C + 1]
// (zeroed by the caller) for the statistics.
__global__ void k_cluster_counts(const uint8_t* __restrict__ lod, const uint32_t* __restrict__ cl_first,
                                 uint32_t C, uint32_t L, uint32_t S, uint32_t* counts) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const uint32_t l = min((uint32_t)lod[c], L);
  const uint32_t m = cl_first[c + 1] - cl_first[c];
  // a cluster of m < 4^l strands has m non-empty level-l thick hairs
  const uint32_t eths = min(1u << (2 * l), m);
  counts[c] = (l == L) ? m * S : eths * S;
  if (l < L) atomicAdd(counts + C + 1, eths * S);
}

__global__ void k_cluster_fill(const uint8_t* __restrict__ lod, const uint32_t* __restrict__ cl_first,
                               const uint32_t* __restrict__ order, const uint32_t* __restrict__ offs,
                               const uint32_t* __restrict__ eth_off, uint32_t C, uint32_t L,
                               uint32_t N, uint32_t S, uint32_t* ids) {
  const uint32_t c = blockIdx.x;
  const uint32_t l = min((uint32_t)lod[c], L);
  const uint32_t base = offs[c];
  if (l == L) {
    const uint32_t r0 = cl_first[c], m = cl_first[c + 1] - r0;
    for (uint32_t j = threadIdx.x; j < m * S; j += blockDim.x) {
      const uint32_t s = order[r0 + j / S];
      ids[base + j] = s * S + j % S;
    }
  } else {
    const uint32_t sub = 1u << (2 * l);
    const uint32_t e0 = eth_off[l] + c * sub;
    const uint32_t m = cl_first[c + 1] - cl_first[c];
    if (m >= sub) {
      for (uint32_t j = threadIdx.x; j < sub * S; j += blockDim.x)
        ids[base + j] = N * S + (e0 + j / S) * S + j % S;
    } else {
      // fewer strands than buckets: member i alone fills bucket floor(i 4^l / m)
      for (uint32_t j = threadIdx.x; j < m * S; j += blockDim.x) {
        const uint32_t b = (uint32_t)(((uint64_t)(j / S) * sub) / m);
        ids[base + j] = N * S + (e0 + b) * S + j % S;
      }
    }
  }
}

__global__ void k_iota(uint32_t* ids, uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ids[i] = i;
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Primitive centroid codes keep the top 7 bits of each axis (21 bits, three
// radix passes).  Primitives in one cell keep the order of the active list
// (clusters in root Morton order, each strand's segments in order along the
// strand), and Karras' index tie-break splits them by that order.  At the
// full-head workload this took the BVH build plus frame from 1.51 to 1.42 ms
// against 10 bits per axis; 8 bits gave 1.47, 6 bits 1.48 and 5 bits 1.91
// (the cells then hold too many primitives).
constexpr int kMortonBits = 21;

__global__ void k_prim_morton(const float4* __restrict__ box, const uint32_t* __restrict__ ids,
                              uint32_t n, const uint32_t* __restrict__ bounds, uint32_t* keys) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float3 lo, hi, inv_ext;
  lo.x = from_ordered(__ldg(bounds)), lo.y = from_ordered(__ldg(bounds + 1));
  lo.z = from_ordered(__ldg(bounds + 2)), hi.x = from_ordered(__ldg(bounds + 3));
  hi.y = from_ordered(__ldg(bounds + 4)), hi.z = from_ordered(__ldg(bounds + 5));
  inv_ext.x = hi.x > lo.x ? 1.f / (hi.x - lo.x) : 0.f;
  inv_ext.y = hi.y > lo.y ? 1.f / (hi.y - lo.y) : 0.f;
  inv_ext.z = hi.z > lo.z ? 1.f / (hi.z - lo.z) : 0.f;
  const uint32_t id = ids[i];
  const float4 l = box[2 * (size_t)id], h = box[2 * (size_t)id + 1];
  const float cx = (0.5f * (l.x + h.x) - lo.x) * inv_ext.x;
  const float cy = (0.5f * (l.y + h.y) - lo.y) * inv_ext.y;
  const float cz = (0.5f * (l.z + h.z) - lo.z) * inv_ext.z;
  const uint32_t qx = (uint32_t)min(1023.f, fmaxf(0.f, cx * 1024.f));
  const uint32_t qy = (uint32_t)min(1023.f, fmaxf(0.f, cy * 1024.f));
  const uint32_t qz = (uint32_t)min(1023.f, fmaxf(0.f, cz * 1024.f));
  keys[i] = ((spread10(qx) << 2) | (spread10(qy) << 1) | spread10(qz)) >> (30 - kMortonBits);
}

// Length of the common prefix of (key, index) at i and j; -1 outside [0, n).
__device__ __forceinline__ int delta(const uint32_t* __restrict__ keys, int n, uint32_t ki, int i,
                                     int j) {
  if ((unsigned)j >= (unsigned)n) return -1;
  const uint32_t x = ki ^ __ldg(keys + j);
  return x ? __clz(x) : 32 + __clz((uint32_t)i ^ (uint32_t)j);
}

__global__ void k_karras(const uint32_t* __restrict__ keys, int n, int4* child,
                         int* parent_int, int* parent_leaf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  const uint32_t ki = __ldg(keys + i);
  const int d = (delta(keys, n, ki, i, i + 1) - delta(keys, n, ki, i, i - 1)) >= 0 ? 1 : -1;
  const int dmin = delta(keys, n, ki, i, i - d);
  int lmax = 2;
  while (delta(keys, n, ki, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(keys, n, ki, i, i + (l + t) * d) > dmin) l += t;
  const int j = i + l * d;
  const int dnode = delta(keys, n, ki, i, j);
  int s = 0;
  for (int k = 1;; ++k) {  // t = ceil(l / 2^k)
    const int t = (l + (1 << k) - 1) >> k;
    if (delta(keys, n, ki, i, i + (s + t) * d) > dnode) s += t;
    if (t == 1) break;
  }
  const int gamma = i + s * d + min(d, 0);
  const int lo = min(i, j), hi = max(i, j);
  int c0, c1;
  if (lo == gamma) {
    c0 = ~gamma;
    parent_leaf[gamma] = i;
  } else {
    c0 = gamma;
    parent_int[gamma] = i;
  }
  if (hi == gamma + 1) {
    c1 = ~(gamma + 1);
    parent_leaf[gamma + 1] = i;
  } else {
    c1 = gamma + 1;
    parent_int[gamma + 1] = i;
  }
  child[i] = make_int4(c0, c1, lo, hi);  // children and the node's leaf range
}

// The global primitive id of every leaf (Morton order).
__global__ void k_gather(const uint32_t* __restrict__ sorted_ids, uint32_t n, uint32_t* leaf_id) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) leaf_id[i] = sorted_ids[i];
}

__device__ __forceinline__ void node_union(const float4* nodes, int c, float* b) {
  // union of an internal node's two child boxes (read through L2: written by
  // other blocks during this kernel)
  const float4 n0 = __ldcg(nodes + 4 * c), n1 = __ldcg(nodes + 4 * c + 1),
               n2 = __ldcg(nodes + 4 * c + 2);
  b[0] = fminf(n0.x, n1.x);
  b[1] = fmaxf(n0.y, n1.y);
  b[2] = fminf(n0.z, n1.z);
  b[3] = fmaxf(n0.w, n1.w);
  b[4] = fminf(n2.x, n2.z);
  b[5] = fmaxf(n2.y, n2.w);
}

__device__ __forceinline__ void lbox_read(const float4* lbox, int leaf, float* b) {
  const float4 l = __ldcg(lbox + 2 * leaf), h = __ldcg(lbox + 2 * leaf + 1);
  b[0] = l.x; b[1] = h.x; b[2] = l.y; b[3] = h.y; b[4] = l.z; b[5] = h.z;
}

// Bounds of an internal node, from two child boxes (lo.x, hi.x, lo.y, hi.y,
// lo.z, hi.z), as the node record.  The records are stored with an L2
// evict-last policy: the frame kernel that follows the build reads them, and
// keeping them in L2 over the leaf records written beside them took the
// full-head frame from 0.63 to 0.60 ms (evict-last on the leaf records as
// well was slower).
__device__ __forceinline__ void store_node(float4* nodes, int node, int4 ch, const float* c0,
                                           const float* c1) {
  float4* o = nodes + 4 * node;
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  const float4 v[4] = {make_float4(c0[0], c0[1], c0[2], c0[3]), make_float4(c1[0], c1[1], c1[2], c1[3]),
                       make_float4(c0[4], c0[5], c1[4], c1[5]),
                       make_float4(__int_as_float(ch.x), __int_as_float(ch.y), 0.f, 0.f)};
#pragma unroll
  for (int q = 0; q < 4; ++q)
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;"
                 :: "l"(o + q), "f"(v[q].x), "f"(v[q].y), "f"(v[q].z), "f"(v[q].w), "l"(pol)
                 : "memory");
}

// Float min / max as one integer atomic on the float's bits (non-negative
// floats order like signed ints; negative ones order like unsigned ints in
// reverse).  -0 must not reach them: callers pass +0.  Returns whether the
// stored value changed.
__device__ __forceinline__ bool atomic_min_f(float* a, float v) {
  if (v >= 0.f) return atomicMin(reinterpret_cast<int*>(a), __float_as_int(v)) > __float_as_int(v);
  return atomicMax(reinterpret_cast<unsigned*>(a), __float_as_uint(v)) < __float_as_uint(v);
}
__device__ __forceinline__ bool atomic_max_f(float* a, float v) {
  if (v >= 0.f) return atomicMax(reinterpret_cast<int*>(a), __float_as_int(v)) < __float_as_int(v);
  return atomicMin(reinterpret_cast<unsigned*>(a), __float_as_uint(v)) > __float_as_uint(v);
}

// Warp-aggregated append of one child (node index, or ~leaf) per lane that
// has one to the list of climb starts; every lane of the warp calls it.
__device__ __forceinline__ void append_start(bool has, int v, unsigned* count, int* list) {
  const unsigned m = __ballot_sync(0xffffffffu, has);
  if (!m) return;
  const int lane = threadIdx.x & 31, lead = __ffs(m) - 1;
  unsigned base = 0;
  if (lane == lead) base = atomicAdd(count, (unsigned)__popc(m));
  base = __shfl_sync(0xffffffffu, base, lead);
  if (has) list[base + __popc(m & ((1u << lane) - 1u))] = v;
}

// Leaf boxes and bottom-up bounds in one kernel.  Thread j of block b owns
// leaf b0 + j and internal node b0 + j (b0 = b * B).  A node record names a
// leaf child by ~(its global primitive id), so the frame kernel reads the
// primitive's records where they are (no copy into leaf order).
//  1. Gather: each thread reads its leaf's box (and id) into shared memory.
//  2. Local subtrees: node i's leaf range starts or ends at leaf i, so a node
//     whose range lies inside the block's leaves ("local") is owned by a
//     thread of the block and so are its children.  These are finished in
//     rounds separated by barriers: a node whose children are done takes
//     their boxes from shared memory, writes its record and its union.  The
//     rounds number the local subtrees' height; no fences, no atomics.
//  3. The few nodes that span blocks are left to k_climb: their owners set
//     their child boxes empty, and the owner of each local node (or leaf)
//     whose parent spans blocks publishes its box and lists it as a climb
//     start, so that no block stays resident behind a climb.
template <int B>
__global__ void __launch_bounds__(B) k_gather_refit(
    const int4* __restrict__ child, const int* __restrict__ parent_int,
    const int* __restrict__ parent_leaf, const float4* __restrict__ box,
    const uint32_t* sorted_ids, int n, float4* nodes, float4* lbox, uint32_t* leaf_id,
    unsigned* n_starts, int* starts) {
  __shared__ int4 s_child[B];
  __shared__ uint32_t s_id[B];  // global primitive id of each of the block's leaves
  __shared__ float s_lbox[B][6];  // leaf boxes (lo.x, hi.x, lo.y, hi.y, lo.z, hi.z)
  __shared__ float s_nbox[B][6];  // unions of the block's local nodes
  __shared__ unsigned char s_done[B];
  const int b0 = blockIdx.x * B;
  const int j = threadIdx.x;
  const int leaf = b0 + j, node = b0 + j;
  const bool has_node = node <= n - 2;
  int4 ch = make_int4(0, 0, -1, -1);
  if (has_node) ch = __ldg(child + node);
  s_child[j] = ch;
  s_done[j] = 0;
  const bool node_local = has_node && ch.z >= b0 && ch.w < b0 + B;
  // 1. gather
  float4 bl = make_float4(0.f, 0.f, 0.f, 0.f), bh = bl;
  int lparent = -1;
  if (leaf < n) {
    const uint32_t id = sorted_ids[leaf];
    bl = box[2 * (size_t)id];
    bh = box[2 * (size_t)id + 1];
    lparent = parent_leaf[leaf];
    leaf_id[leaf] = id;
    s_id[j] = id;
    s_lbox[j][0] = bl.x; s_lbox[j][1] = bh.x; s_lbox[j][2] = bl.y;
    s_lbox[j][3] = bh.y; s_lbox[j][4] = bl.z; s_lbox[j][5] = bh.z;
  }
  __syncthreads();
  // 2. local subtrees, one level of readiness per round
  bool pending = node_local;
  for (;;) {
    bool ready = false;
    if (pending)
      ready = (ch.x < 0 || s_done[ch.x - b0]) && (ch.y < 0 || s_done[ch.y - b0]);
    if (ready) {
      const float* p0 = ch.x < 0 ? s_lbox[~ch.x - b0] : s_nbox[ch.x - b0];
      const float* p1 = ch.y < 0 ? s_lbox[~ch.y - b0] : s_nbox[ch.y - b0];
      float c0[6], c1[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        c0[q] = p0[q];
        c1[q] = p1[q];
      }
      // a leaf child is named by its primitive id (the leaf lies in this block)
      const int4 chp = make_int4(ch.x < 0 ? ~(int)s_id[~ch.x - b0] : ch.x,
                                 ch.y < 0 ? ~(int)s_id[~ch.y - b0] : ch.y, ch.z, ch.w);
      store_node(nodes, node, chp, c0, c1);
      s_nbox[j][0] = fminf(c0[0], c1[0]);
      s_nbox[j][1] = fmaxf(c0[1], c1[1]);
      s_nbox[j][2] = fminf(c0[2], c1[2]);
      s_nbox[j][3] = fmaxf(c0[3], c1[3]);
      s_nbox[j][4] = fminf(c0[4], c1[4]);
      s_nbox[j][5] = fmaxf(c0[5], c1[5]);
    }
    const int any = __syncthreads_or(ready);  // this round's reads of s_done are over
    if (ready) {
      s_done[j] = 1;
      pending = false;
    }
    if (!any) break;
    __syncthreads();  // this round's flags are visible
  }
  // 3. nodes that span blocks: empty child boxes, widened by k_climb
  if (has_node && !node_local) {
    float4* o = nodes + 4 * (size_t)node;
    const float inf = __int_as_float(0x7f800000);
    const float4 e = make_float4(inf, -inf, inf, -inf);
    __stcg(o, e);
    __stcg(o + 1, e);
    __stcg(o + 2, e);
    const int c0 = ch.x < 0 ? ~(int)sorted_ids[~ch.x] : ch.x;
    const int c1 = ch.y < 0 ? ~(int)sorted_ids[~ch.y] : ch.y;
    __stcg(o + 3, make_float4(__int_as_float(c0), __int_as_float(c1), 0.f, 0.f));
  }
  bool start_leaf = false, start_node = false;
  if (leaf < n && lparent >= 0) {
    const bool parent_local = lparent >= b0 && lparent < b0 + B && s_child[lparent - b0].z >= b0 &&
                              s_child[lparent - b0].w < b0 + B;
    if (!parent_local) {
      __stcg(lbox + 2 * leaf, bl);
      __stcg(lbox + 2 * leaf + 1, bh);
      start_leaf = true;
    }
  }
  if (node_local && node != 0) {
    const int p = __ldg(parent_int + node);
    start_node = !(p >= b0 && p < b0 + B && s_child[p - b0].z >= b0 && s_child[p - b0].w < b0 + B);
  }
  append_start(start_leaf, ~leaf, n_starts, starts);
  append_start(start_node, node, n_starts, starts);
}

// Bounds of the nodes that span blocks.  Each climb start (a leaf or local
// node whose parent spans blocks; its record is complete) widens, with float
// atomics, its own slot in its parent, then its parent's slot in the
// grandparent, and so on to the root.  Each of the six coordinates stops at
// the first ancestor slot that it does not change: that slot already holds a
// value at least as wide from another start below it, which carries it on
// up.  No ordering between starts is needed.
__global__ void k_climb(const unsigned* __restrict__ n_starts, const int* __restrict__ starts,
                        const int4* __restrict__ child, const int* __restrict__ parent_int,
                        const int* __restrict__ parent_leaf, float4* nodes, const float4* lbox) {
  const unsigned m = *n_starts;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    int cur = __ldg(starts + i);
    float b[6];
    int p;
    if (cur < 0) {
      lbox_read(lbox, ~cur, b);
      p = __ldg(parent_leaf + ~cur);
    } else {
      node_union(nodes, cur, b);
      p = __ldg(parent_int + cur);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) b[q] = b[q] + 0.f;  // -0 -> +0
    unsigned live = 0x3fu;
    while (p >= 0) {
      const int4 ch = __ldg(child + p);
      const int up = p == 0 ? -1 : __ldg(parent_int + p);
      float* r = reinterpret_cast<float*>(nodes + 4 * (size_t)p);
      // record slots of (lo.x, hi.x, lo.y, hi.y, lo.z, hi.z) for child 0 / child 1
      const int o = ch.x == cur ? 0 : 4, oz = ch.x == cur ? 8 : 10;
      const int off[6] = {o, o + 1, o + 2, o + 3, oz, oz + 1};
#pragma unroll
      for (int q = 0; q < 6; ++q)
        if ((live >> q) & 1u) {
          const bool changed = (q & 1) ? atomic_max_f(r + off[q], b[q]) : atomic_min_f(r + off[q], b[q]);
          if (!changed) live &= ~(1u << q);
        }
      if (!live) break;
      cur = p;
      p = up;
    }
  }
}

__global__ void k_bytes_differ(const uint8_t* __restrict__ x, const uint8_t* __restrict__ y,
                               uint32_t n, uint32_t* diff) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && x[i] != y[i]) *diff = 1u;
}

// Leaf records of the primitives `ids` (in leaf order) and every node's
// bounds, over the topology in bv.
hr_status gather_refit(hr_ctx* ctx, hr_asset* a, Bvh& bv, const uint32_t* ids, cudaStream_t st) {
  const uint32_t n = bv.n;
  unsigned* n_starts = nullptr;
  float4* lbox = nullptr;
  int* starts = nullptr;  // at most one per leaf and one per internal node
  HR_TRY(scratch(ctx, 39, 16, (void**)&n_starts));
  HR_TRY(scratch(ctx, 46, (size_t)n * 2 * sizeof(float4), (void**)&lbox));
  HR_TRY(scratch(ctx, 48, (size_t)n * 2 * 4, (void**)&starts));
  HR_CUDA(ctx, cudaMemsetAsync(n_starts, 0, 4, st));
  k_gather_refit<256><<<(n + 255) / 256, 256, 0, st>>>(bv.child, bv.par_int, bv.par_leaf,
                                                       a->prim_box, ids, (int)n, bv.nodes, lbox,
                                                       bv.leaf_id, n_starts, starts);
  HR_LAUNCHED(ctx);
  static int climb_grid = 0;
  if (!climb_grid) {
    int dev = 0, sms = 1, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_climb, 256, 0) != cudaSuccess || per < 1) {
      cudaGetLastError();
      per = 1;
    }
    climb_grid = sms * per;
  }
  const unsigned grid = (unsigned)std::min<size_t>((size_t)climb_grid, ((size_t)n * 2 + 255) / 256);
  k_climb<<<grid, 256, 0, st>>>(n_starts, starts, bv.child, bv.par_int, bv.par_leaf, bv.nodes, lbox);
  HR_LAUNCHED(ctx);
  return HR_OK;
}

}  // namespace

void free_bvh(hr_ctx* ctx, Bvh& bv) {
  if (bv.cap) {
    dfree(ctx, bv.nodes, (size_t)std::max(bv.cap, 2u) * 4 * sizeof(float4));
    dfree(ctx, bv.leaf_id, (size_t)bv.cap * 4);
    dfree(ctx, bv.child, (size_t)bv.cap * sizeof(int4));
    dfree(ctx, bv.par_int, (size_t)bv.cap * 4);
    dfree(ctx, bv.par_leaf, (size_t)bv.cap * 4);
  }
  if (bv.lod_built) dfree(ctx, bv.lod_built, bv.lod_cap);
  bv = Bvh();
}

hr_status build_bvh(hr_ctx* ctx, hr_asset* a, const uint8_t* lod_dev, Bvh& bv, cudaStream_t st) {
  const uint32_t N = a->N, S = a->S;
  bv.valid = 0;
  // 1. active primitive ids
  uint32_t n = 0, n_eth = 0;
  uint32_t* ids = nullptr;
  if (a->C == 0 || a->n_levels == 0 || lod_dev == nullptr) {
    n = N * S;
    HR_TRY(scratch(ctx, 30, (size_t)n * 4, (void**)&ids));
    k_iota<<<(n + 255) / 256, 256, 0, st>>>(ids, n);
    HR_LAUNCHED(ctx);
  } else {
    const uint32_t C = a->C, L = a->n_levels;
    uint32_t* cnt = nullptr;
    HR_TRY(scratch(ctx, 31, (size_t)(C + 2) * 4, (void**)&cnt));
    HR_CUDA(ctx, cudaMemsetAsync(cnt + C, 0, 8, st));
    k_cluster_counts<<<(C + 255) / 256, 256, 0, st>>>(lod_dev, a->cl_first, C, L, S, cnt);
    HR_LAUNCHED(ctx);
    HR_TRY(scan_u32(ctx, cnt, C + 1, st));
    uint32_t tot[2] = {0, 0};  // active primitives, of which thick-hair segments
    HR_CUDA(ctx, cudaMemcpyAsync(tot, cnt + C, 8, cudaMemcpyDeviceToHost, st));
    HR_CUDA(ctx, cudaStreamSynchronize(st));
    n = tot[0];
    n_eth = tot[1];
    uint32_t* eoff = nullptr;
    HR_TRY(scratch(ctx, 32, 16 * 4, (void**)&eoff));
    HR_CUDA(ctx, cudaMemcpyAsync(eoff, a->eth_offset, 16 * 4, cudaMemcpyHostToDevice, st));
    HR_TRY(scratch(ctx, 30, (size_t)std::max(n, 1u) * 4, (void**)&ids));
    k_cluster_fill<<<C, 256, 0, st>>>(lod_dev, a->cl_first, a->order, cnt, eoff, C, L, N, S, ids);
    HR_LAUNCHED(ctx);
  }
  // 2. storage (grow only)
  if (n > bv.cap) {
    if (bv.cap) {
      HR_CUDA(ctx, cudaStreamSynchronize(st));
      free_bvh(ctx, bv);
    }
    HR_TRY(dalloc(ctx, (void**)&bv.nodes, (size_t)std::max(n, 2u) * 4 * sizeof(float4), "BVH nodes"));
    HR_TRY(dalloc(ctx, (void**)&bv.leaf_id, (size_t)n * 4, "BVH leaf ids"));
    HR_TRY(dalloc(ctx, (void**)&bv.child, (size_t)n * sizeof(int4), "BVH children"));
    HR_TRY(dalloc(ctx, (void**)&bv.par_int, (size_t)n * 4, "BVH parents"));
    HR_TRY(dalloc(ctx, (void**)&bv.par_leaf, (size_t)n * 4, "BVH leaf parents"));
    bv.cap = n;
  }
  // (after the grow: free_bvh resets every field)
  bv.n = n;
  bv.n_eth = n_eth;
  // what the topology is built for (checked by refit_bvh); the hierarchy as it is now
  HR_CUDA(ctx, cudaMemsetAsync(a->d_bounds + kHierChanged, 0, 4, st));
  bv.topo = 0;
  bv.built_C = a->C;
  bv.built_E = a->E;
  bv.built_total = a->n_prims_total;
  bv.built_with_lod = lod_dev != nullptr;
  if (lod_dev) {
    if (bv.lod_cap < a->C) {
      if (bv.lod_built) dfree(ctx, bv.lod_built, bv.lod_cap);
      bv.lod_built = nullptr;
      bv.lod_cap = 0;
      HR_TRY(dalloc(ctx, (void**)&bv.lod_built, a->C, "BVH LoD"));
      bv.lod_cap = a->C;
    }
    HR_CUDA(ctx, cudaMemcpyAsync(bv.lod_built, lod_dev, a->C, cudaMemcpyDeviceToDevice, st));
  }
  if (n == 0) {
    bv.valid = 1;
    bv.topo = 1;
    return HR_OK;
  }
  // 3. Morton codes and sort
  uint32_t *keys, *k2, *v2;
  HR_TRY(scratch(ctx, 33, (size_t)n * 4, (void**)&keys));
  HR_TRY(scratch(ctx, 34, (size_t)n * 4, (void**)&k2));
  HR_TRY(scratch(ctx, 35, (size_t)n * 4, (void**)&v2));
  k_prim_morton<<<(n + 255) / 256, 256, 0, st>>>(a->prim_box, ids, n, a->d_bounds, keys);
  HR_LAUNCHED(ctx);
  HR_TRY(radix_sort_pairs(ctx, keys, ids, k2, v2, n, kMortonBits, st, kLookbackPolls, &keys, &ids));
  if (n == 1) {
    k_gather<<<1, 32, 0, st>>>(ids, n, bv.leaf_id);
    HR_LAUNCHED(ctx);
    bv.valid = 1;
    bv.topo = 1;
    return HR_OK;
  }
  // 4. hierarchy, then leaf records and bounds in one bottom-up pass
  k_karras<<<(n - 1 + 255) / 256, 256, 0, st>>>(keys, (int)n, bv.child, bv.par_int, bv.par_leaf);
  HR_LAUNCHED(ctx);
  HR_TRY(gather_refit(ctx, a, bv, ids, st));
  bv.valid = 1;
  bv.topo = 1;
  return HR_OK;
}

hr_status refit_bvh(hr_ctx* ctx, hr_asset* a, const uint8_t* lod_dev, Bvh& bv, cudaStream_t st) {
  if (!bv.topo || bv.built_C != a->C || bv.built_E != a->E || bv.built_total != a->n_prims_total ||
      bv.built_with_lod != (lod_dev != nullptr))
    return set_error(ctx, HR_ESTATE, "refit: the BVH was built for another hierarchy");
  {
    // one read-back: the LoD selection against the build's, and whether a
    // hierarchy build changed the strand order since
    uint32_t* diff = nullptr;
    HR_TRY(scratch(ctx, 36, 8, (void**)&diff));
    HR_CUDA(ctx, cudaMemsetAsync(diff, 0, 4, st));
    if (lod_dev) {
      k_bytes_differ<<<(a->C + 255) / 256, 256, 0, st>>>(lod_dev, bv.lod_built, a->C, diff);
      HR_LAUNCHED(ctx);
    }
    HR_CUDA(ctx, cudaMemcpyAsync(diff + 1, a->d_bounds + kHierChanged, 4, cudaMemcpyDeviceToDevice, st));
    uint32_t h[2] = {0, 0};
    HR_CUDA(ctx, cudaMemcpyAsync(h, diff, 8, cudaMemcpyDeviceToHost, st));
    HR_CUDA(ctx, cudaStreamSynchronize(st));
    if (h[0]) return set_error(ctx, HR_ESTATE, "refit: the LoD selection changed since the build");
    if (h[1]) return set_error(ctx, HR_ESTATE, "refit: the strand order changed since the build");
  }
  bv.valid = 0;
  const uint32_t n = bv.n;
  // a single leaf has no node; its records are the primitive's own
  if (n > 1) HR_TRY(gather_refit(ctx, a, bv, bv.leaf_id, st));
  bv.valid = 1;
  return HR_OK;
}

}  // namespace hr
