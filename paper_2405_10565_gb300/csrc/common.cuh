// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/hairrt.h"

namespace hr {

constexpr float kPi = 3.14159265358979323846f;
constexpr double kPiD = 3.14159265358979323846;
constexpr float kInvSqrt2Pi = 0.3989422804014327f;

// Scattering lookup tables (baked once per context).
// IM(theta, beta) = integral over theta_o in [-pi/2, pi/2] of
// G(beta, (theta + theta_o)/2) cos^2(theta_o), theta in [0, pi/2],
// beta in [kImBetaLo, kImBetaHi]; row-major [beta][theta].
constexpr int kImNT = 256;
constexpr int kImNB = 64;
constexpr float kImBetaLo = 0.04f;
constexpr float kImBetaHi = 0.68f;
struct Tables {
  const float* im32;   // [kImNB][kImNT]
  const __half* im16;  // [kImNB][kImNT]
};

// One BVH over the active primitives of an asset.
struct TileSched;

struct Bvh {
  uint32_t n = 0;           // active primitives (leaves)
  uint32_t cap = 0;         // allocated leaves
  float4* nodes = nullptr;  // [(n-1) * 4]; a leaf child is ~(global primitive id)
  uint32_t* leaf_id = nullptr; // [n] global primitive id of every leaf, Morton order
  uint32_t n_eth = 0;
  int valid = 0;               // bounds and leaf records match the primitives
  // topology kept for refits: children + leaf range, parents; the LoD and
  // hierarchy shape it was built for
  int4* child = nullptr;       // [cap]
  int* par_int = nullptr;      // [cap]
  int* par_leaf = nullptr;     // [cap]
  uint8_t* lod_built = nullptr;  // [lod_cap] copy of the LoD of the build (none: all strands)
  uint32_t lod_cap = 0, built_C = 0, built_E = 0, built_total = 0;
  int built_with_lod = 0;
  int topo = 0;                // a topology exists
};

// Device scratch that grows on demand (owned by the context).
struct Scratch {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace hr

struct hr_ctx;

struct hr_asset {
  hr_ctx* ctx = nullptr;
  uint32_t N = 0, S = 0;
  float4* verts = nullptr;  // [N * (S + 1)]
  float* mat = nullptr;     // [(N + E) * 12]: strands then thick hairs
  float2* shape = nullptr;  // [N]
  size_t mat_cap = 0;       // rows allocated in mat
  // hierarchy
  uint32_t C = 0, n_levels = 0, E = 0;
  uint32_t eth_offset[16] = {0};
  uint32_t* order = nullptr;       // [N] strand ids by (code, id)
  uint32_t* cluster_of = nullptr;  // [N]
  uint32_t* cl_first = nullptr;    // [C + 1] first rank of each cluster
  float4* xsec = nullptr;          // [E * (S+1) * 3] (c,a) (e1,b) (e2,0)
  float4* xsec_other = nullptr;    // the other buffer of a pipelined hr_render_frame (or null)
  // the other vertex and record buffers of a pipelined hr_asset_update (or
  // null), sized for other_total records
  float4* verts_other = nullptr;
  float4 *xf_other = nullptr, *box_other = nullptr, *aux_other = nullptr;
  uint32_t other_total = 0;
  // all potential primitives: strand segments then thick-hair segments
  uint32_t n_prims_total = 0;
  float4* prim_xf = nullptr;   // [P_total * 3]
  float4* prim_box = nullptr;  // [P_total * 2]
  float4* prim_aux = nullptr;  // [P_total]
  uint32_t* d_bounds = nullptr;  // [8] strand boxes' bounds, ordered float bits (lo xyz, hi xyz);
                                 // word kHierChanged: the strand order changed since the last BVH build
  // LoD
  uint8_t* lod = nullptr;  // [C] current selection on the device
  int lod_valid = 0;
  hr::Bvh bvh;
  size_t bytes = 0;
  // guide-driven hierarchy and skinning (hr_build_guided_clusters)
  uint32_t G = 0;                 // k-means clusters; 0: no guides
  int32_t* guides = nullptr;      // [G] guide strand of every k-means cluster, -1 when empty
  uint32_t* cl_tri = nullptr;     // [C] the three guides of every cluster, 10 bits each
  float4* w_strand = nullptr;     // [N * (S + 1)] prism weights of the strand vertices
  float4* w_eth = nullptr;        // [E * (S + 1) * 5] of thick-hair centres and corners
  uint32_t guided_C = 0, guided_E = 0;  // shape the weights were taken for
  // frame-kernel schedule carried between frames (TileSched)
  hr::TileSched* sched = nullptr;
};

namespace hr {

// ----------------------------------------------------------------- helpers

uint64_t ctx_alloc_note(hr_ctx* ctx, int64_t delta);
hr_status set_error(hr_ctx* ctx, hr_status st, const std::string& msg);
cudaStream_t ctx_stream(hr_ctx* ctx);
// Stream and event of a pipelined hr_render_frame: the next frame's clusters
// and fit run on the side stream while the previous frame renders.
cudaStream_t ctx_side_stream(hr_ctx* ctx);
cudaEvent_t ctx_fit_event(hr_ctx* ctx);
Tables ctx_tables(hr_ctx* ctx);
// device allocation charged to the context budget
hr_status dalloc(hr_ctx* ctx, void** p, size_t bytes, const char* what);
void dfree(hr_ctx* ctx, void* p, size_t bytes);
// grow-only scratch slot `slot` of the context
hr_status scratch(hr_ctx* ctx, int slot, size_t bytes, void** p);

#define HR_CUDA(ctx, call)                                                              \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return ::hr::set_error((ctx), HR_ECUDA,                                           \
                             std::string(#call) + ": " + cudaGetErrorString(e_));       \
  } while (0)

// After every kernel launch: count it and check the launch error.
void note_launch(hr_ctx* ctx);
#define HR_LAUNCHED(ctx)          \
  do {                            \
    ::hr::note_launch(ctx);       \
    HR_CUDA(ctx, cudaGetLastError()); \
  } while (0)

#define HR_TRY(call)                 \
  do {                               \
    hr_status s_ = (call);           \
    if (s_ != HR_OK) return s_;      \
  } while (0)

// --- primitives (sort.cu)
// exclusive scan of n uint32 values in place (device); uses scratch slots 10-12
hr_status scan_u32(hr_ctx* ctx, uint32_t* data, uint32_t n, cudaStream_t st);
// stable LSD radix sort of (key, value) pairs on the low `bits` key bits,
// one kernel per 8-bit digit pass (decoupled look-back); result in
// keys/vals; tmp buffers of n entries; scratch slot 14; n < 2^30
// max_polls: reads of an unpublished earlier tile before counting instead
// (0: count at once, for tests)
constexpr int kLookbackPolls = 1 << 16;
// The sorted pairs end in (keys, vals); with keys_out and vals_out given they
// are left where the last pass wrote them (keys / vals or the temporaries)
// and those pointers name them, which saves copying back after an odd number
// of passes.
hr_status radix_sort_pairs(hr_ctx* ctx, uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp,
                           uint32_t* vals_tmp, uint32_t n, int bits, cudaStream_t st,
                           int max_polls = kLookbackPolls, uint32_t** keys_out = nullptr,
                           uint32_t** vals_out = nullptr);

// no-allocation variants on caller-provided scratch (sort.cu, hierarchy.cu)
cudaError_t scan_u32_with(uint32_t* data, uint32_t n, uint32_t* sums, cudaStream_t st);
cudaError_t radix_sort_pairs_with(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp,
                                  uint32_t* vals_tmp, uint32_t n, int bits, uint32_t* counts,
                                  uint32_t* sums, cudaStream_t st);
cudaError_t morton_clusters_with(const float4* verts, uint32_t N, uint32_t S, uint32_t C,
                                 uint32_t* order, uint32_t* cluster_of, uint32_t* bounds,
                                 uint32_t* keys, uint32_t* keys_tmp, uint32_t* vals_tmp,
                                 uint32_t* counts, uint32_t* sums, cudaStream_t st);

// --- hierarchy.cu
hr_status build_strand_prims(hr_ctx* ctx, hr_asset* a);
hr_status refresh_strand_prims(hr_ctx* ctx, hr_asset* a);
// new vertices from a device-readable source (device memory, or page-locked
// host memory mapped into the device's address space) in one fused kernel:
// device copy, strand records, Morton bounds; strands of at most
// kUpdateMaxVerts vertices
constexpr uint32_t kUpdateMaxVerts = 2048;
// on stream st (null: the context's stream)
hr_status update_strands(hr_ctx* ctx, hr_asset* a, const float4* src_dev, cudaStream_t st = nullptr);
// device address through which kernels can read p (device memory, or mapped
// page-locked host memory), or nullptr
const void* device_view(const void* p);

// Word of hr_asset::d_bounds set by a hierarchy build that changed the strand
// order (or the hierarchy) and cleared by a BVH build: a refit is then invalid.
constexpr int kHierChanged = 6;

// Float <-> unsigned with the same order (atomic min / max of floats).
__device__ __forceinline__ uint32_t ordered_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_ordered(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
// st_fit: run the clusters and the fit on this stream (the side stream of a
// pipelined hr_render_frame), the thick-hair records on the main stream after
// them; null: everything on the main stream.
hr_status build_hierarchy(hr_ctx* ctx, hr_asset* a, uint32_t C, uint32_t max_levels,
                          cudaEvent_t fit_begin = nullptr, cudaEvent_t fit_end = nullptr,
                          cudaStream_t st_fit = nullptr);
// The roots' Morton codes (sorted, into codes) and the strands in (code, id)
// order (into order), both [N] device.
hr_status root_morton_order(hr_ctx* ctx, hr_asset* a, uint32_t* codes, uint32_t* order,
                            cudaStream_t st);
// The levels, fits and records of a hierarchy given by its strand order and
// cluster starts (device, [N] and [C + 1]).
hr_status build_hierarchy_from(hr_ctx* ctx, hr_asset* a, uint32_t C, uint32_t max_levels,
                               const uint32_t* order_dev, const uint32_t* cl_first_dev);

// The thick-hair materials and segment records from the current
// cross-sections (after skinning moved them; no new fit).
hr_status rebuild_eth_records(hr_ctx* ctx, hr_asset* a);

// --- guides.cu
// Free the guide-driven state of an asset (its hierarchy is being replaced).
void drop_guides(hr_ctx* ctx, hr_asset* a);
// Guides by k-means (G clusters, `iters` update rounds), clusters of strands
// sharing their three nearest guides, the hierarchy's levels, fits and
// records, and the skinning weights of strand vertices and thick-hair
// centres and corners.
hr_status build_guided_hierarchy(hr_ctx* ctx, hr_asset* a, uint32_t G, uint32_t iters,
                                 uint32_t max_levels);
// Move the strands and thick hairs with the guides' new vertices gv_dev
// [G][S + 1] (device) by the skinning weights, and rebuild their records.
hr_status skin_asset(hr_ctx* ctx, hr_asset* a, const float4* gv_dev);

// --- lod.cu
hr_status lod_widths(hr_ctx* ctx, hr_asset* a, const hr_camera* cam, float* wcl_dev,
                     cudaStream_t st);
hr_status lod_select(hr_ctx* ctx, hr_asset* a, const hr_camera* cam, float eps, int mode,
                     int bias, const uint8_t* prev_dev, uint8_t* out_dev, cudaStream_t st);

// --- bvh.cu
// Build `out` over the active primitives of LoD `lod_dev` (nullptr: all
// strands) on stream `st`.
hr_status build_bvh(hr_ctx* ctx, hr_asset* a, const uint8_t* lod_dev, Bvh& out, cudaStream_t st);
// Refit `bv` to the asset's current primitive records, keeping its topology
// and leaf order.  HR_ESTATE unless the hierarchy shape and the LoD `lod_dev`
// (nullptr: all strands) are those bv was built for (one read-back).
hr_status refit_bvh(hr_ctx* ctx, hr_asset* a, const uint8_t* lod_dev, Bvh& bv, cudaStream_t st);
void free_bvh(hr_ctx* ctx, Bvh& b);

// --- tables.cu
hr_status bake_tables(hr_ctx* ctx, float** im32, __half** im16);

// --- trace.cu
struct LaunchCam {
  int kind, W, H;
  float pix;
  float ipix_hi, ipix_lo;  // 1 / pix as a double-word pair (host-rounded from FP64)
  float3 eye, right, up, fwd;
};
struct LaunchLights {
  int n;
  float4 xyzw[HR_MAX_LIGHTS];
  float4 rgb[HR_MAX_LIGHTS];
};
// Warp-tile schedule carried from one frame of an asset to the next.  The
// warp tiles whose slowest lane took the most traversal steps (node visits
// plus primitive tests) in the previous frame are traced first, kHeavyRays
// rays per warp: a ray that shares its warp with 31 other long rays advances
// at a fraction of the pace it keeps with few (the slowest full-head ray:
// ~550 us in its 32-ray tile, ~300 us alone), and these few tiles otherwise
// set the frame's length.  Each traced lane of such a tile stores its partial
// sums; the warp that finishes the tile's last hand-out composites its pixels
// with the same shuffle tree as a whole-warp tile, so the image does not
// depend on the schedule.  Measured on the full-head frame (FP32, 8 spp):
// 16 tiles of 4-ray hand-outs took the frame from 0.58 to 0.48 ms alone;
// 64 tiles, 1 or 2 rays per hand-out or a 60-70% threshold were no better,
// and spent more warp time.
constexpr uint32_t kHeavyMax = 16;         // heavy tiles per frame, at most
constexpr uint32_t kHeavyRelPct = 50;      // steps of a heavy tile's slowest lane, at least, in
                                           // percent of the frame's slowest tile
constexpr uint32_t kHeavyMinSteps = 16;    // and more than this
constexpr uint32_t kHeavyRays = 4;         // rays (lanes) of a heavy tile per hand-out
constexpr uint32_t kHeavyItems = 32 / kHeavyRays;
// Only frames of at most this many warp tiles per resident warp trace heavy
// tiles: with many tiles per warp the hand-out balances the work by itself
// (the close full-head view, ~160 tiles per warp, was 1.3% slower with them,
// the middle one, ~24, 1.3% faster, the far one, ~2.4, 19% faster).
constexpr uint32_t kHeavyTilesPerWarp = 64;
// The frame kernel lists the tiles whose step count reaches a threshold (half
// the previous frame's largest) as candidates, kCandMax at most, and keeps
// the frame's largest; the next frame picks its heavy tiles among them.
constexpr uint32_t kCandMax = 1024;
struct TileSched {
  uint32_t n_heavy;    // heavy tiles of the frame being rendered
  uint32_t grp;        // lanes per pixel the list was made for
  uint32_t prev_n;     // warp tiles of the previous frame (0: no previous frame)
  uint32_t prev_W, prev_H, prev_grp;
  uint32_t thresh;     // steps that make a tile of this frame a candidate
  uint32_t max_steps;  // this frame's largest tile step count (atomic max)
  float4 prev_rect;    // the previous frame's scene rectangle (its warp grid)
  uint32_t cand_n;     // candidates listed by this frame (atomic; may exceed kCandMax)
  uint32_t pad[3];
  uint32_t cand_tile[kCandMax];   // grid index of each candidate tile
  uint32_t cand_steps[kCandMax];  // and its slowest lane's steps
  uint32_t heavy[kHeavyMax];            // tile origins x0 | y0 << 16, heaviest first
  uint32_t done[kHeavyMax];             // rays finished per heavy tile
  uint32_t ray_steps[kHeavyMax * 32];   // per ray of a heavy tile
  float acc[kHeavyMax * 32 * 3];        // per-lane partial sums of a heavy tile
};

struct FrameArgs {
  const float4* nodes;     // BVH nodes; a leaf child is ~(global primitive id)
  const float4* prim_xf;   // [P_total * 3] world -> unit-cylinder rows, by global id
  const float4* prim_aux;  // [P_total] (material index bits, n_tot, r, a*b)
  const uint32_t* leaf_id; // the single leaf's id when the BVH has one leaf
  const float4* verts;     // strand vertices and thick-hair cross-sections: the
  const float4* xsec;      // segments' start points for FP64 decisions
  uint32_t N, S;           // strands, segments per strand
  const float* mat;
  uint32_t n_prims;
  Tables tables;
  LaunchCam cam;
  LaunchLights lights;
  uint32_t spp;
  uint64_t seed;
  uint32_t flags;
  uint32_t* overflow;  // device counter of stack overflows
  unsigned long long* counters;  // [6] node visits, prim tests, strand shades, eth shades,
                                 // hits, traced samples
  uint32_t k;          // k-buffer depth (<= the kernel's KMAX)
  uint32_t grp;        // lanes per pixel (power of two <= 32; samples spread over them)
  uint32_t tile_w, tile_h;  // pixels per 128-thread block: tile_w x tile_h = 128 / grp
  hr_tile_record* tile_log;  // counting kernel only: per warp tile times and counts, or null
  uint32_t tile_cap;         // records tile_log holds
  uint32_t* tile_count;      // the frame's number of warp tiles (written when tile_log is set)
  TileSched* sched;          // plain frame kernel: the heavy-tile schedule, or null
  uint32_t frame_warps;      // with sched: resident warps of the frame kernel
};

// Tile geometry of the frame and serving kernels for a given spp: each pixel
// owns `grp` adjacent lanes (the smallest power of two >= spp, at most 32),
// a 128-thread block covers 128 / grp pixels in a tile_w x tile_h rectangle.
struct TileGeom {
  uint32_t grp, tile_w, tile_h;
};
inline TileGeom tile_geom(uint32_t spp) {
  uint32_t g = 1, lg = 0;
  while (g < spp && g < 32) g <<= 1, ++lg;
  const uint32_t pixels = 128 / g;
  const uint32_t tw = 16u >> ((lg + 1) / 2);
  return TileGeom{g, tw, pixels / tw};
}
inline uint32_t tiles_for(uint32_t W, uint32_t H, uint32_t spp) {
  const TileGeom t = tile_geom(spp);
  return ((W + t.tile_w - 1) / t.tile_w) * ((H + t.tile_h - 1) / t.tile_h);
}
hr_status launch_frame(hr_ctx* ctx, const FrameArgs& fa, int precision, bool count,
                       float* rgb_dev, cudaStream_t st);
hr_status launch_frame_shadow(hr_ctx* ctx, const FrameArgs& fa, int precision, bool count,
                       float* rgb_dev, cudaStream_t st);
hr_status launch_samples(hr_ctx* ctx, const FrameArgs& fa, int precision, const uint32_t* sids,
                         uint32_t m, float* rad_dev, int32_t* hit_dev, cudaStream_t st);
// IM(theta, beta) lookups at m device points (test export of the shading code)
hr_status launch_im_lookup(hr_ctx* ctx, int precision, const float* theta, const float* beta,
                           uint32_t m, float* out, cudaStream_t st);

// Warp tiles of a frame: a warp renders wtw x wth pixels (32 / grp pixels, a
// pixel's samples on grp adjacent lanes); the tiles that overlap the projected
// scene rectangle `rect` (pixel space, from the BVH root box) form an nx-wide
// grid from pixel (x0, y0), n tiles in all.  The frame and serving kernels
// enumerate only these; every other pixel is background.
struct WarpGrid {
  uint32_t wtw, wth, x0, y0, nx, n;
};
__host__ __device__ inline WarpGrid warp_grid(const float4 rect, uint32_t W, uint32_t H,
                                              uint32_t grp) {
  WarpGrid g{1, 1, 0, 0, 0, 0};
  const uint32_t P = 32u / grp;  // pixels per warp tile
  while (g.wtw * g.wtw < P) g.wtw <<= 1;
  g.wth = P / g.wtw;
  const float fx0 = fmaxf(0.f, floorf(rect.x)), fy0 = fmaxf(0.f, floorf(rect.y));
  const float fx1 = fminf(rect.z, (float)W - 1.f), fy1 = fminf(rect.w, (float)H - 1.f);
  if (fx0 <= fx1 && fy0 <= fy1) {
    g.x0 = (uint32_t)fx0 / g.wtw * g.wtw;
    g.y0 = (uint32_t)fy0 / g.wth * g.wth;
    g.nx = ((uint32_t)fx1 - g.x0) / g.wtw + 1;
    g.n = g.nx * (((uint32_t)fy1 - g.y0) / g.wth + 1);
  }
  return g;
}

// Batched serving launch: warp tiles from several requests.
struct ServeItem {
  FrameArgs fa;
  float* rgb;       // device output of the request (cleared to background)
  float4 rect;      // the request's projected scene rectangle
  WarpGrid grid;    // its warp tiles
  uint32_t wt0;     // first warp tile (of the request's grid) in this item
  uint32_t nwt;     // warp tiles in this item
};
// Projected scene rectangle of a frame into rect_dev (one warp; device).
hr_status launch_scene_rect(hr_ctx* ctx, const FrameArgs& fa, float4* rect_dev, cudaStream_t st);
// items_dev[i] covers batch tiles [item_start_dev[i], item_start_dev[i+1]);
// every item of one launch has the same k-buffer bound and precision.
hr_status launch_serve_batch(hr_ctx* ctx, int kmax, int precision, const ServeItem* items_dev,
                             const uint32_t* item_start_dev, uint32_t n_items,
                             uint32_t total_tiles, uint32_t* work_counter_dev, int grid,
                             cudaStream_t st);
int kmax_for(uint32_t k);

LaunchCam to_launch_cam(const hr_camera& c);
LaunchLights to_launch_lights(const hr_render_desc& d);

// Threads per block of the frame and serving kernels.
constexpr int kBlock = 128;

}  // namespace hr
