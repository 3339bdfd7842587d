// C ABI of the library: contexts, device memory under an HBM budget, assets,
// and the hierarchy / LoD / BVH / render entry points.  Every computation is
// a kernel of this library; this file only validates, allocates, copies and
// launches.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "serve.h"

constexpr int kFrameCall = 1, kUpdateCall = 2;

struct hr_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint64_t budget = 0;
  std::atomic<uint64_t> used{0};
  float* im32 = nullptr;
  __half* im16 = nullptr;
  std::vector<hr::Scratch> scratch;
  std::mutex err_mu;
  std::string last_error;
  std::recursive_mutex api_mu;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t ph[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  uint32_t* d_overflow = nullptr;
  unsigned long long* d_counters = nullptr;
  std::chrono::steady_clock::time_point t0;
  hr::Server* server = nullptr;
  std::atomic<uint64_t> launches{0};
  // pipelined hr_render_frame: the side stream runs the next frame's clusters
  // and fit once ev_built (the previous frame's BVH is done) has passed
  cudaStream_t side = nullptr;
  cudaEvent_t ev_built = nullptr, ev_fit = nullptr, ev_update = nullptr;
  // the kind of the last API call, as set by it (0 any other, kFrameCall,
  // kUpdateCall a pipelined hr_asset_update) and as seen by the current call
  int call_kind = 0, prev_kind = 0;
  // frame-time ring: per hr_render_frame, events around the fit and the frame
  static constexpr int kRing = 256;
  cudaEvent_t ring[kRing][4] = {};
  uint64_t ring_n = 0;
  std::vector<uint8_t> ring_fit;  // entry i: bit 0 its fit events were recorded, bit 1 it refit the BVH
};

namespace hr {

hr_status set_error(hr_ctx* ctx, hr_status st, const std::string& msg) {
  if (ctx) {
    std::lock_guard<std::mutex> g(ctx->err_mu);
    ctx->last_error = msg;
  }
  return st;
}

cudaStream_t ctx_stream(hr_ctx* ctx) { return ctx->stream; }
cudaStream_t ctx_side_stream(hr_ctx* ctx) { return ctx->side; }
cudaEvent_t ctx_fit_event(hr_ctx* ctx) { return ctx->ev_fit; }

void note_launch(hr_ctx* ctx) { ctx->launches++; }

Tables ctx_tables(hr_ctx* ctx) { return Tables{ctx->im32, ctx->im16}; }

std::recursive_mutex& ctx_mutex(hr_ctx* ctx) { return ctx->api_mu; }

double ctx_now_ms(hr_ctx* ctx) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ctx->t0)
      .count();
}

int ctx_device(hr_ctx* ctx) { return ctx->device; }

Server** ctx_server_slot(hr_ctx* ctx) { return &ctx->server; }

uint64_t ctx_budget(hr_ctx* ctx) { return ctx->budget; }

uint32_t* ctx_overflow(hr_ctx* ctx) { return ctx->d_overflow; }

hr_status dalloc(hr_ctx* ctx, void** p, size_t bytes, const char* what) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (ctx->budget && ctx->used.load() + bytes > ctx->budget)
    return set_error(ctx, HR_ENOMEM, std::string("HBM budget exceeded allocating ") + what);
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_error(ctx, HR_ENOMEM,
                     std::string("cudaMalloc failed for ") + what + ": " + cudaGetErrorString(e));
  }
  ctx->used += bytes;
  return HR_OK;
}

void dfree(hr_ctx* ctx, void* p, size_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  cudaFree(p);
  ctx->used -= bytes;
}

hr_status scratch(hr_ctx* ctx, int slot, size_t bytes, void** p) {
  if (slot < 0 || slot >= (int)ctx->scratch.size()) return set_error(ctx, HR_EINVAL, "scratch slot");
  Scratch& s = ctx->scratch[slot];
  if (bytes > s.bytes) {
    if (s.p) {
      cudaStreamSynchronize(ctx->stream);
      dfree(ctx, s.p, s.bytes);
      s.p = nullptr;
      s.bytes = 0;
    }
    size_t want = bytes + bytes / 4 + 256;
    HR_TRY(dalloc(ctx, &s.p, want, "scratch"));
    s.bytes = want;
  }
  *p = s.p;
  return HR_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

const void* device_view(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return p;
  if (at.type == cudaMemoryTypeHost) return at.devicePointer;
  return nullptr;
}

// Copy `bytes` from a host-or-device source into a device destination.
hr_status to_device(hr_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (!bytes) return HR_OK;
  HR_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes,
                               is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                               st));
  return HR_OK;
}

FrameArgs frame_args(hr_ctx* ctx, hr_asset* a, const Bvh& bv, const hr_render_desc& d) {
  FrameArgs fa{};
  fa.nodes = bv.nodes;
  fa.prim_xf = a->prim_xf;
  fa.prim_aux = a->prim_aux;
  fa.leaf_id = bv.leaf_id;
  fa.verts = a->verts;
  fa.xsec = a->xsec;
  fa.N = a->N;
  fa.S = a->S;
  fa.mat = a->mat;
  fa.n_prims = bv.n;
  fa.tables = ctx_tables(ctx);
  fa.cam = to_launch_cam(d.camera);
  fa.lights = to_launch_lights(d);
  fa.spp = d.spp;
  fa.seed = d.seed;
  fa.flags = d.flags;
  fa.overflow = ctx->d_overflow;
  fa.counters = ctx->d_counters;
  fa.tile_log = nullptr;
  fa.tile_cap = 0;
  fa.tile_count = nullptr;
  fa.k = d.k_depth;
  const TileGeom tg = tile_geom(d.spp);
  fa.grp = tg.grp;
  fa.tile_w = tg.tile_w;
  fa.tile_h = tg.tile_h;
  return fa;
}

hr_status check_desc(hr_ctx* ctx, const hr_render_desc* d) {
  if (!d) return set_error(ctx, HR_EINVAL, "render desc is null");
  if (d->spp < 1) return set_error(ctx, HR_EINVAL, "spp must be >= 1");
  if (d->k_depth < 1 || d->k_depth > HR_MAX_K) return set_error(ctx, HR_EINVAL, "k_depth out of 1..8");
  if (d->n_lights < 1 || d->n_lights > HR_MAX_LIGHTS)
    return set_error(ctx, HR_EINVAL, "n_lights out of 1..16");
  if (d->camera.width < 1 || d->camera.height < 1 || d->camera.width > 65536 ||
      d->camera.height > 65536)
    return set_error(ctx, HR_EINVAL, "image size out of range");
  if ((uint64_t)d->camera.width * d->camera.height * d->spp >= (1ull << 40))
    return set_error(ctx, HR_EINVAL, "too many samples");
  if (d->camera.kind != 0 && d->camera.kind != 1) return set_error(ctx, HR_EINVAL, "camera kind");
  if (!(d->camera.pix_scale > 0.f)) return set_error(ctx, HR_EINVAL, "pix_scale must be > 0");
  if (d->precision != HR_PREC_FP32 && d->precision != HR_PREC_FP16)
    return set_error(ctx, HR_EINVAL, "precision");
  return HR_OK;
}

}  // namespace hr

using namespace hr;

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

#define API_ENTER(ctx)                                                   \
  if (!(ctx)) return HR_EINVAL;                                          \
  std::lock_guard<std::recursive_mutex> api_lock_((ctx)->api_mu);        \
  DeviceGuard dev_guard_((ctx)->device);                                 \
  (ctx)->prev_kind = (ctx)->call_kind;                                   \
  (ctx)->call_kind = 0

}  // namespace

extern "C" {

hr_status hr_create(hr_ctx** out, int device, uint64_t hbm_budget, void* cuda_stream) {
  if (!out) return HR_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
    cudaGetLastError();
    return HR_ECUDA;
  }
  if (device < 0 || device >= n) return HR_EINVAL;
  hr_ctx* ctx = new hr_ctx();
  ctx->device = device;
  ctx->budget = hbm_budget;
  ctx->scratch.resize(64);
  ctx->t0 = std::chrono::steady_clock::now();
  DeviceGuard g(device);
  if (cuda_stream) {
    ctx->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return HR_ECUDA;
    }
    ctx->own_stream = true;
  }
  hr_status st = HR_OK;
  if (cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess)
    st = HR_ECUDA;
  for (int i = 0; i < 6 && st == HR_OK; ++i)
    if (cudaEventCreate(&ctx->ph[i]) != cudaSuccess) st = HR_ECUDA;
  if (st == HR_OK && (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
                      cudaEventCreateWithFlags(&ctx->ev_built, cudaEventDisableTiming) != cudaSuccess ||
                      cudaEventCreateWithFlags(&ctx->ev_fit, cudaEventDisableTiming) != cudaSuccess ||
                      cudaEventCreateWithFlags(&ctx->ev_update, cudaEventDisableTiming) != cudaSuccess))
    st = HR_ECUDA;
  for (int i = 0; i < hr_ctx::kRing && st == HR_OK; ++i)
    for (int j = 0; j < 4 && st == HR_OK; ++j)
      if (cudaEventCreate(&ctx->ring[i][j]) != cudaSuccess) st = HR_ECUDA;
  ctx->ring_fit.assign(hr_ctx::kRing, 0);
  if (st == HR_OK) st = dalloc(ctx, (void**)&ctx->d_overflow, 64, "flags");
  if (st == HR_OK) st = dalloc(ctx, (void**)&ctx->d_counters, 8 * sizeof(unsigned long long), "counters");
  if (st == HR_OK) st = bake_tables(ctx, &ctx->im32, &ctx->im16);
  if (st == HR_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = HR_ECUDA;
  if (st != HR_OK) {
    hr_destroy(ctx);
    return st;
  }
  *out = ctx;
  return HR_OK;
}

hr_status hr_destroy(hr_ctx* ctx) {
  if (!ctx) return HR_EINVAL;
  if (ctx->server) hr_serve_stop(ctx);
  {
    DeviceGuard g(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->side) cudaStreamSynchronize(ctx->side);
    for (auto& s : ctx->scratch)
      if (s.p) cudaFree(s.p);
    if (ctx->im32) cudaFree(ctx->im32);
    if (ctx->im16) cudaFree(ctx->im16);
    if (ctx->d_overflow) cudaFree(ctx->d_overflow);
    if (ctx->d_counters) cudaFree(ctx->d_counters);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    for (int i = 0; i < 6; ++i)
      if (ctx->ph[i]) cudaEventDestroy(ctx->ph[i]);
    for (int i = 0; i < hr_ctx::kRing; ++i)
      for (int j = 0; j < 4; ++j)
        if (ctx->ring[i][j]) cudaEventDestroy(ctx->ring[i][j]);
    if (ctx->ev_built) cudaEventDestroy(ctx->ev_built);
    if (ctx->ev_fit) cudaEventDestroy(ctx->ev_fit);
    if (ctx->ev_update) cudaEventDestroy(ctx->ev_update);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  }
  delete ctx;
  return HR_OK;
}

const char* hr_last_error(hr_ctx* ctx) {
  if (!ctx) return "null context";
  std::lock_guard<std::mutex> g(ctx->err_mu);
  return ctx->last_error.c_str();
}

uint64_t hr_bytes_in_use(hr_ctx* ctx) { return ctx ? ctx->used.load() : 0; }

uint64_t hr_kernel_launches(hr_ctx* ctx) { return ctx ? ctx->launches.load() : 0; }

hr_status hr_asset_create(hr_ctx* ctx, const hr_hair_desc* d, hr_asset** out) {
  API_ENTER(ctx);
  if (!d || !out || !d->vertices || !d->material || !d->shape)
    return set_error(ctx, HR_EINVAL, "hr_asset_create: null argument");
  *out = nullptr;
  if (d->n_strands < 1 || d->n_segments < 1 || d->n_segments > 4096 ||
      (uint64_t)d->n_strands * d->n_segments >= (1ull << 30))
    return set_error(ctx, HR_EINVAL, "hr_asset_create: sizes out of range");
  cudaStream_t st = ctx->stream;
  hr_asset* a = new hr_asset();
  a->ctx = ctx;
  a->N = d->n_strands;
  a->S = d->n_segments;
  const size_t nv = (size_t)a->N * (a->S + 1);
  hr_status s = dalloc(ctx, (void**)&a->verts, nv * sizeof(float4), "vertices");
  if (s == HR_OK) s = dalloc(ctx, (void**)&a->mat, (size_t)a->N * HR_MAT_FLOATS * 4, "materials");
  if (s == HR_OK) s = dalloc(ctx, (void**)&a->shape, (size_t)a->N * sizeof(float2), "shape");
  a->mat_cap = a->N;
  if (s == HR_OK) s = to_device(ctx, a->verts, d->vertices, nv * sizeof(float4), st);
  if (s == HR_OK) s = to_device(ctx, a->mat, d->material, (size_t)a->N * HR_MAT_FLOATS * 4, st);
  if (s == HR_OK) s = to_device(ctx, a->shape, d->shape, (size_t)a->N * sizeof(float2), st);
  if (s == HR_OK) s = build_strand_prims(ctx, a);
  if (s != HR_OK) {
    hr_asset_destroy(ctx, a);
    return s;
  }
  *out = a;
  return HR_OK;
}

hr_status hr_asset_update(hr_ctx* ctx, hr_asset* a, const float* vertices) {
  API_ENTER(ctx);
  if (!a || !vertices) return set_error(ctx, HR_EINVAL, "hr_asset_update: null argument");
  if (ctx->server) serve_forget_asset(ctx, ctx->server, a);
  cudaStream_t st = ctx->stream;
  // a device-readable source (device memory, page-locked host memory) is read
  // once by the kernel that rebuilds the records, so the transfer overlaps
  // the build; anything else is copied first
  const float4* view = static_cast<const float4*>(device_view(vertices));
  // Pipelining: right after hr_render_frame, the new positions go to the
  // asset's other set of vertex and record buffers on the side stream, while
  // the frame in flight keeps reading the set it was launched with; the next
  // hr_render_frame's clusters and fit follow them there.  The other set was
  // last read by the frame before, which ended before the last BVH was built.
  const uint64_t ns = (uint64_t)a->N * a->S;
  if (ctx->prev_kind == kFrameCall && !ctx->server && view && a->S + 1 <= kUpdateMaxVerts &&
      a->n_prims_total >= ns) {
    const uint64_t P = a->n_prims_total;
    const size_t nv = (size_t)a->N * (a->S + 1);
    if (a->other_total != P) {  // (re)size the other set to the current records
      if (a->verts_other) dfree(ctx, a->verts_other, nv * sizeof(float4)), a->verts_other = nullptr;
      if (a->xf_other) dfree(ctx, a->xf_other, (size_t)a->other_total * 3 * sizeof(float4)), a->xf_other = nullptr;
      if (a->box_other) dfree(ctx, a->box_other, (size_t)a->other_total * 2 * sizeof(float4)), a->box_other = nullptr;
      if (a->aux_other) dfree(ctx, a->aux_other, (size_t)a->other_total * sizeof(float4)), a->aux_other = nullptr;
      a->other_total = 0;
      HR_TRY(dalloc(ctx, (void**)&a->verts_other, nv * sizeof(float4), "vertices (second set)"));
      HR_TRY(dalloc(ctx, (void**)&a->xf_other, P * 3 * sizeof(float4), "records (second set)"));
      HR_TRY(dalloc(ctx, (void**)&a->box_other, P * 2 * sizeof(float4), "boxes (second set)"));
      HR_TRY(dalloc(ctx, (void**)&a->aux_other, P * sizeof(float4), "aux (second set)"));
      a->other_total = (uint32_t)P;
    }
    cudaStream_t sd = ctx->side;
    HR_CUDA(ctx, cudaStreamWaitEvent(sd, ctx->ev_built, 0));
    if (P > ns) {  // the thick-hair records too, so the new set is whole whatever comes next
      HR_CUDA(ctx, cudaMemcpyAsync(a->xf_other + 3 * ns, a->prim_xf + 3 * ns, (P - ns) * 3 * sizeof(float4),
                                   cudaMemcpyDeviceToDevice, sd));
      HR_CUDA(ctx, cudaMemcpyAsync(a->box_other + 2 * ns, a->prim_box + 2 * ns, (P - ns) * 2 * sizeof(float4),
                                   cudaMemcpyDeviceToDevice, sd));
      HR_CUDA(ctx, cudaMemcpyAsync(a->aux_other + ns, a->prim_aux + ns, (P - ns) * sizeof(float4),
                                   cudaMemcpyDeviceToDevice, sd));
    }
    std::swap(a->verts, a->verts_other);
    std::swap(a->prim_xf, a->xf_other);
    std::swap(a->prim_box, a->box_other);
    std::swap(a->prim_aux, a->aux_other);
    HR_TRY(update_strands(ctx, a, view, sd));
    // everything enqueued on the main stream from here on sees the new set
    HR_CUDA(ctx, cudaEventRecord(ctx->ev_update, sd));
    HR_CUDA(ctx, cudaStreamWaitEvent(st, ctx->ev_update, 0));
    a->bvh.valid = 0;
    ctx->call_kind = kUpdateCall;
    return HR_OK;
  }
  if (view && a->S + 1 <= kUpdateMaxVerts) {
    HR_TRY(update_strands(ctx, a, view));
  } else {
    HR_TRY(to_device(ctx, a->verts, vertices, (size_t)a->N * (a->S + 1) * sizeof(float4), st));
    HR_TRY(refresh_strand_prims(ctx, a));
  }
  a->bvh.valid = 0;
  return HR_OK;
}

hr_status hr_asset_destroy(hr_ctx* ctx, hr_asset* a) {
  API_ENTER(ctx);
  if (!a) return HR_EINVAL;
  if (ctx->server) serve_forget_asset(ctx, ctx->server, a);
  cudaStreamSynchronize(ctx->stream);
  cudaStreamSynchronize(ctx->side);
  const size_t S1 = a->S + 1;
  dfree(ctx, a->verts, (size_t)a->N * S1 * sizeof(float4));
  dfree(ctx, a->mat, a->mat_cap * HR_MAT_FLOATS * 4);
  dfree(ctx, a->shape, (size_t)a->N * sizeof(float2));
  if (a->order) dfree(ctx, a->order, (size_t)a->N * 4);
  if (a->cluster_of) dfree(ctx, a->cluster_of, (size_t)a->N * 4);
  if (a->cl_first) dfree(ctx, a->cl_first, (size_t)(a->C + 1) * 4);
  if (a->xsec) dfree(ctx, a->xsec, (size_t)a->E * S1 * 3 * sizeof(float4));
  if (a->xsec_other) dfree(ctx, a->xsec_other, (size_t)a->E * S1 * 3 * sizeof(float4));
  if (a->verts_other) dfree(ctx, a->verts_other, (size_t)a->N * S1 * sizeof(float4));
  if (a->xf_other) dfree(ctx, a->xf_other, (size_t)a->other_total * 3 * sizeof(float4));
  if (a->box_other) dfree(ctx, a->box_other, (size_t)a->other_total * 2 * sizeof(float4));
  if (a->aux_other) dfree(ctx, a->aux_other, (size_t)a->other_total * sizeof(float4));
  if (a->lod) dfree(ctx, a->lod, a->C);
  if (a->sched) dfree(ctx, a->sched, sizeof(TileSched));
  drop_guides(ctx, a);
  const uint64_t P = a->n_prims_total;
  if (a->prim_xf) dfree(ctx, a->prim_xf, P * 3 * sizeof(float4));
  if (a->prim_box) dfree(ctx, a->prim_box, P * 2 * sizeof(float4));
  if (a->prim_aux) dfree(ctx, a->prim_aux, P * sizeof(float4));
  if (a->d_bounds) dfree(ctx, a->d_bounds, 8 * sizeof(uint32_t));
  free_bvh(ctx, a->bvh);
  delete a;
  return HR_OK;
}

hr_status hr_build_clusters(hr_ctx* ctx, hr_asset* a, uint32_t C, uint32_t max_levels,
                            uint32_t* cluster_of_out, uint32_t* order_out) {
  API_ENTER(ctx);
  if (!a) return set_error(ctx, HR_EINVAL, "null asset");
  if (C < 1 || C > a->N || C > (1u << 20)) return set_error(ctx, HR_EINVAL, "n_clusters out of range");
  // served BVHs of this asset reference its primitive records, rewritten here
  if (ctx->server) serve_forget_asset(ctx, ctx->server, a);
  HR_TRY(build_hierarchy(ctx, a, C, max_levels));
  cudaStream_t st = ctx->stream;
  if (cluster_of_out) {
    const bool dev = is_device_ptr(cluster_of_out);
    HR_CUDA(ctx, cudaMemcpyAsync(cluster_of_out, a->cluster_of, (size_t)a->N * 4,
                                 dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  }
  if (order_out) {
    const bool dev = is_device_ptr(order_out);
    HR_CUDA(ctx, cudaMemcpyAsync(order_out, a->order, (size_t)a->N * 4,
                                 dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  }
  HR_CUDA(ctx, cudaStreamSynchronize(st));
  return HR_OK;
}

hr_status hr_build_guided_clusters(hr_ctx* ctx, hr_asset* a, uint32_t n_guides, uint32_t iterations,
                                   uint32_t max_levels, uint32_t* cluster_of_out,
                                   uint32_t* order_out) {
  API_ENTER(ctx);
  if (!a) return set_error(ctx, HR_EINVAL, "null asset");
  if (iterations > 1000) return set_error(ctx, HR_EINVAL, "iterations out of 0..1000");
  if (ctx->server) serve_forget_asset(ctx, ctx->server, a);
  HR_TRY(build_guided_hierarchy(ctx, a, n_guides, iterations, max_levels));
  cudaStream_t st = ctx->stream;
  if (cluster_of_out)
    HR_CUDA(ctx, cudaMemcpyAsync(cluster_of_out, a->cluster_of, (size_t)a->N * 4,
                                 is_device_ptr(cluster_of_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  if (order_out)
    HR_CUDA(ctx, cudaMemcpyAsync(order_out, a->order, (size_t)a->N * 4,
                                 is_device_ptr(order_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  HR_CUDA(ctx, cudaStreamSynchronize(st));
  return HR_OK;
}

hr_status hr_guides_export(hr_ctx* ctx, hr_asset* a, int32_t* guides_out,
                           uint32_t* cluster_guides_out) {
  API_ENTER(ctx);
  if (!a) return set_error(ctx, HR_EINVAL, "null asset");
  if (a->G == 0) return set_error(ctx, HR_ESTATE, "no guides: call hr_build_guided_clusters");
  cudaStream_t st = ctx->stream;
  if (guides_out)
    HR_CUDA(ctx, cudaMemcpyAsync(guides_out, a->guides, (size_t)a->G * 4,
                                 is_device_ptr(guides_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  if (cluster_guides_out) {
    std::vector<uint32_t> key(a->C), tri((size_t)a->C * 3);
    HR_CUDA(ctx, cudaMemcpyAsync(key.data(), a->cl_tri, (size_t)a->C * 4, cudaMemcpyDeviceToHost, st));
    HR_CUDA(ctx, cudaStreamSynchronize(st));
    for (uint32_t c = 0; c < a->C; ++c) {
      tri[3 * c] = key[c] >> 20;
      tri[3 * c + 1] = (key[c] >> 10) & 1023u;
      tri[3 * c + 2] = key[c] & 1023u;
    }
    HR_CUDA(ctx, cudaMemcpyAsync(cluster_guides_out, tri.data(), tri.size() * 4,
                                 is_device_ptr(cluster_guides_out) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, st));
  }
  HR_CUDA(ctx, cudaStreamSynchronize(st));
  return HR_OK;
}

hr_status hr_asset_skin(hr_ctx* ctx, hr_asset* a, const float* guide_vertices) {
  API_ENTER(ctx);
  if (!a || !guide_vertices) return set_error(ctx, HR_EINVAL, "hr_asset_skin: null argument");
  if (a->G == 0 || !a->w_strand || a->guided_C != a->C || a->guided_E != a->E)
    return set_error(ctx, HR_ESTATE, "no guide-driven hierarchy: call hr_build_guided_clusters");
  if (ctx->server) serve_forget_asset(ctx, ctx->server, a);
  cudaStream_t st = ctx->stream;
  const size_t bytes = (size_t)a->G * (a->S + 1) * sizeof(float4);
  float4* gv = nullptr;
  HR_TRY(scratch(ctx, 62, bytes, (void**)&gv));
  HR_TRY(to_device(ctx, gv, guide_vertices, bytes, st));
  HR_TRY(skin_asset(ctx, a, gv));
  return HR_OK;
}

hr_status hr_vertex_export(hr_ctx* ctx, hr_asset* a, float* verts_out) {
  API_ENTER(ctx);
  if (!a || !verts_out) return set_error(ctx, HR_EINVAL, "null argument");
  cudaStream_t st = ctx->stream;
  HR_CUDA(ctx, cudaMemcpyAsync(verts_out, a->verts, (size_t)a->N * (a->S + 1) * sizeof(float4),
                               is_device_ptr(verts_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  HR_CUDA(ctx, cudaStreamSynchronize(st));
  return HR_OK;
}

hr_status hr_hierarchy_info(hr_ctx* ctx, hr_asset* a, uint32_t* C, uint32_t* L, uint32_t* E) {
  API_ENTER(ctx);
  if (!a) return set_error(ctx, HR_EINVAL, "null asset");
  if (C) *C = a->C;
  if (L) *L = a->n_levels;
  if (E) *E = a->E;
  return HR_OK;
}

hr_status hr_eth_export(hr_ctx* ctx, hr_asset* a, float* xsec, uint32_t* counts, float* mat) {
  API_ENTER(ctx);
  if (!a) return set_error(ctx, HR_EINVAL, "null asset");
  if (a->E == 0) return set_error(ctx, HR_ESTATE, "no thick hairs: call hr_build_clusters");
  cudaStream_t st = ctx->stream;
  const size_t S1 = a->S + 1;
  if (xsec) {
    HR_CUDA(ctx, cudaMemcpyAsync(xsec, a->xsec, (size_t)a->E * S1 * 3 * sizeof(float4),
                                 is_device_ptr(xsec) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  }
  if (mat) {
    HR_CUDA(ctx, cudaMemcpyAsync(mat, a->mat + (size_t)a->N * HR_MAT_FLOATS,
                                 (size_t)a->E * HR_MAT_FLOATS * 4,
                                 is_device_ptr(mat) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  }
  if (counts) {
    std::vector<uint32_t> first(a->C + 1), cnt(a->E);
    HR_CUDA(ctx, cudaMemcpyAsync(first.data(), a->cl_first, (a->C + 1) * 4, cudaMemcpyDeviceToHost, st));
    HR_CUDA(ctx, cudaStreamSynchronize(st));
    for (uint32_t k = 0; k < a->n_levels; ++k) {
      const uint64_t sub = 1ull << (2 * k);
      for (uint32_t c = 0; c < a->C; ++c) {
        const uint64_t m = first[c + 1] - first[c];
        for (uint64_t j = 0; j < sub; ++j) {
          const uint64_t lo = (j * m + sub - 1) / sub, hi = ((j + 1) * m + sub - 1) / sub;
          cnt[a->eth_offset[k] + c * sub + j] = (uint32_t)(hi - lo);
        }
      }
    }
    HR_CUDA(ctx, cudaMemcpyAsync(counts, cnt.data(), (size_t)a->E * 4,
                                 is_device_ptr(counts) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, st));
  }
  HR_CUDA(ctx, cudaStreamSynchronize(st));
  return HR_OK;
}

hr_status hr_lod_widths(hr_ctx* ctx, hr_asset* a, const hr_camera* cam, float* width_out) {
  API_ENTER(ctx);
  if (!a || !cam || !width_out) return set_error(ctx, HR_EINVAL, "null argument");
  if (a->n_levels == 0) return set_error(ctx, HR_ESTATE, "no thick-hair levels");
  cudaStream_t st = ctx->stream;
  const size_t bytes = (size_t)a->C * a->n_levels * 4;
  if (is_device_ptr(width_out)) {
    HR_TRY(lod_widths(ctx, a, cam, width_out, st));
  } else {
    float* tmp = nullptr;
    HR_TRY(scratch(ctx, 40, bytes, (void**)&tmp));
    HR_TRY(lod_widths(ctx, a, cam, tmp, st));
    HR_CUDA(ctx, cudaMemcpyAsync(width_out, tmp, bytes, cudaMemcpyDeviceToHost, st));
  }
  HR_CUDA(ctx, cudaStreamSynchronize(st));
  return HR_OK;
}

hr_status hr_select_lod(hr_ctx* ctx, hr_asset* a, const hr_camera* cam, float eps, int mode,
                        int bias, uint8_t* lod_inout) {
  API_ENTER(ctx);
  if (!a || !cam) return set_error(ctx, HR_EINVAL, "null argument");
  if (a->n_levels == 0) return set_error(ctx, HR_ESTATE, "no thick-hair levels: call hr_build_clusters");
  if (mode < 0 || mode > 2 || bias < 0) return set_error(ctx, HR_EINVAL, "mode / bias");
  if (mode >= 1 && !lod_inout) return set_error(ctx, HR_EINVAL, "deferred mode needs lod_inout");
  cudaStream_t st = ctx->stream;
  uint8_t* prev = nullptr;
  if (mode >= 1) {
    HR_TRY(scratch(ctx, 41, a->C, (void**)&prev));
    HR_TRY(to_device(ctx, prev, lod_inout, a->C, st));
  }
  HR_TRY(lod_select(ctx, a, cam, eps, mode, bias, prev, a->lod, st));
  a->lod_valid = 1;
  if (lod_inout) {
    HR_CUDA(ctx, cudaMemcpyAsync(lod_inout, a->lod, a->C,
                                 is_device_ptr(lod_inout) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  }
  HR_CUDA(ctx, cudaStreamSynchronize(st));
  return HR_OK;
}

hr_status hr_build_bvh(hr_ctx* ctx, hr_asset* a, const uint8_t* lod) {
  API_ENTER(ctx);
  if (!a) return set_error(ctx, HR_EINVAL, "null asset");
  cudaStream_t st = ctx->stream;
  const uint8_t* lod_dev = nullptr;
  if (a->n_levels > 0) {
    if (lod) {
      HR_TRY(to_device(ctx, a->lod, lod, a->C, st));
      a->lod_valid = 1;
      lod_dev = a->lod;
    } else if (a->lod_valid) {
      lod_dev = a->lod;
    }
  }
  HR_TRY(build_bvh(ctx, a, lod_dev, a->bvh, st));
  HR_CUDA(ctx, cudaStreamSynchronize(st));
  return HR_OK;
}

hr_status hr_bvh_export(hr_ctx* ctx, hr_asset* a, uint32_t* leaf_ids, uint32_t* n_active) {
  API_ENTER(ctx);
  if (!a) return set_error(ctx, HR_EINVAL, "null asset");
  if (!a->bvh.valid) return set_error(ctx, HR_ESTATE, "no BVH: call hr_build_bvh");
  if (n_active) *n_active = a->bvh.n;
  if (leaf_ids && a->bvh.n) {
    HR_CUDA(ctx, cudaMemcpyAsync(leaf_ids, a->bvh.leaf_id, (size_t)a->bvh.n * 4,
                                 is_device_ptr(leaf_ids) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 ctx->stream));
    HR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return HR_OK;
}

hr_status hr_sort_pairs(hr_ctx* ctx, uint32_t* keys, uint32_t* vals, uint32_t n, uint32_t bits,
                        int count_earlier) {
  API_ENTER(ctx);
  if (n == 0) return HR_OK;
  if (!keys || !vals || !is_device_ptr(keys) || !is_device_ptr(vals))
    return set_error(ctx, HR_EINVAL, "hr_sort_pairs: keys and vals must be device memory");
  if (bits < 1 || bits > 32 || n >= (1u << 30))
    return set_error(ctx, HR_EINVAL, "hr_sort_pairs: bits out of 1..32 or n >= 2^30");
  cudaStream_t st = ctx->stream;
  uint32_t *k2 = nullptr, *v2 = nullptr;
  HR_TRY(scratch(ctx, 49, (size_t)n * 4, (void**)&k2));
  HR_TRY(scratch(ctx, 50, (size_t)n * 4, (void**)&v2));
  HR_TRY(radix_sort_pairs(ctx, keys, vals, k2, v2, n, (int)bits, st,
                          count_earlier ? 0 : kLookbackPolls));
  HR_CUDA(ctx, cudaStreamSynchronize(st));
  return HR_OK;
}

hr_status hr_table_export(hr_ctx* ctx, float* im32_out, uint16_t* im16_out, uint32_t* n_theta,
                          uint32_t* n_beta) {
  API_ENTER(ctx);
  if (n_theta) *n_theta = kImNT;
  if (n_beta) *n_beta = kImNB;
  cudaStream_t st = ctx->stream;
  const size_t n = (size_t)kImNT * kImNB;
  if (im32_out)
    HR_CUDA(ctx, cudaMemcpyAsync(im32_out, ctx->im32, n * sizeof(float),
                                 is_device_ptr(im32_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  if (im16_out)
    HR_CUDA(ctx, cudaMemcpyAsync(im16_out, ctx->im16, n * sizeof(__half),
                                 is_device_ptr(im16_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  HR_CUDA(ctx, cudaStreamSynchronize(st));
  return HR_OK;
}

hr_status hr_im_lookup(hr_ctx* ctx, const float* theta, const float* beta, uint32_t m,
                       int precision, float* out) {
  API_ENTER(ctx);
  if (m == 0) return HR_OK;
  if (!theta || !beta || !out) return set_error(ctx, HR_EINVAL, "null argument");
  if (precision != HR_PREC_FP32 && precision != HR_PREC_FP16)
    return set_error(ctx, HR_EINVAL, "hr_im_lookup: precision must be HR_PREC_FP32 or HR_PREC_FP16");
  cudaStream_t st = ctx->stream;
  float* buf = nullptr;
  HR_TRY(scratch(ctx, 51, (size_t)m * 3 * sizeof(float), (void**)&buf));
  HR_TRY(to_device(ctx, buf, theta, (size_t)m * 4, st));
  HR_TRY(to_device(ctx, buf + m, beta, (size_t)m * 4, st));
  HR_TRY(launch_im_lookup(ctx, precision, buf, buf + m, m, buf + 2 * (size_t)m, st));
  HR_CUDA(ctx, cudaMemcpyAsync(out, buf + 2 * (size_t)m, (size_t)m * 4,
                               is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  HR_CUDA(ctx, cudaStreamSynchronize(st));
  return HR_OK;
}

// The asset's warp-tile schedule (TileSched), allocated (cleared) on first use.
static hr_status tile_schedule(hr_ctx* ctx, hr_asset* a, FrameArgs& fa, cudaStream_t st) {
  if (!a->sched) {
    HR_TRY(dalloc(ctx, (void**)&a->sched, sizeof(TileSched), "tile schedule"));
    HR_CUDA(ctx, cudaMemsetAsync(a->sched, 0, sizeof(TileSched), st));
  }
  fa.sched = a->sched;
  return HR_OK;
}

static hr_status render_impl(hr_ctx* ctx, hr_asset* a, const hr_render_desc* desc, float* rgb_out,
                             hr_stats* stats, hr_tile_record* tiles = nullptr,
                             uint32_t tile_cap = 0, uint32_t* n_tiles = nullptr,
                             cudaEvent_t t_begin = nullptr, cudaEvent_t t_end = nullptr) {
  if (!a || !rgb_out) return set_error(ctx, HR_EINVAL, "null argument");
  HR_TRY(check_desc(ctx, desc));
  if (!a->bvh.valid) return set_error(ctx, HR_ESTATE, "no BVH: call hr_build_bvh");
  cudaStream_t st = ctx->stream;
  const size_t bytes = (size_t)desc->camera.width * desc->camera.height * 3 * sizeof(float);
  const bool dev_out = is_device_ptr(rgb_out);
  float* out = rgb_out;
  if (!dev_out) HR_TRY(scratch(ctx, 42, bytes, (void**)&out));
  FrameArgs fa = frame_args(ctx, a, a->bvh, *desc);
  const bool profile = tiles != nullptr || n_tiles != nullptr;
  const bool count = (desc->flags & HR_FLAG_COUNT) != 0 || profile;
  hr_tile_record* tlog = nullptr;
  if (profile) {
    const bool dev_tiles = tiles && is_device_ptr(tiles);
    tlog = dev_tiles ? tiles : nullptr;
    if (!dev_tiles) HR_TRY(scratch(ctx, 37, (size_t)std::max(tile_cap, 1u) * sizeof(hr_tile_record), (void**)&tlog));
    HR_TRY(scratch(ctx, 38, 4, (void**)&fa.tile_count));
    HR_CUDA(ctx, cudaMemsetAsync(fa.tile_count, 0, 4, st));
    fa.tile_log = tlog;
    fa.tile_cap = tiles ? tile_cap : 0;
  }
  if (stats || count) {
    HR_CUDA(ctx, cudaMemsetAsync(ctx->d_overflow, 0, 4, st));
    HR_CUDA(ctx, cudaMemsetAsync(ctx->d_counters, 0, 8 * sizeof(unsigned long long), st));
  }
  // Right after an overlapped hr_asset_update the frame shares the GPU with
  // the upload kernel on the side stream; there the ray-by-ray hand-outs ran
  // far slower (animated frames through the C ABI: the frame kernel 1.3-2.0
  // instead of 0.82 ms), so such a frame keeps the fixed order and leaves the
  // schedule as it is.
  if (!count && !(desc->flags & HR_FLAG_FIXED_TILE_ORDER) && ctx->prev_kind != kUpdateCall)
    HR_TRY(tile_schedule(ctx, a, fa, st));
  if (stats) HR_CUDA(ctx, cudaEventRecord(ctx->ev0, st));
  if (t_begin) HR_CUDA(ctx, cudaEventRecord(t_begin, st));
  HR_TRY(launch_frame(ctx, fa, desc->precision, count, out, st));
  if (t_end) HR_CUDA(ctx, cudaEventRecord(t_end, st));
  if (stats) HR_CUDA(ctx, cudaEventRecord(ctx->ev1, st));
  if (!dev_out) HR_CUDA(ctx, cudaMemcpyAsync(rgb_out, out, bytes, cudaMemcpyDeviceToHost, st));
  if (profile) {
    uint32_t nt = 0;
    HR_CUDA(ctx, cudaMemcpyAsync(&nt, fa.tile_count, 4, cudaMemcpyDeviceToHost, st));
    HR_CUDA(ctx, cudaStreamSynchronize(st));
    if (n_tiles) *n_tiles = nt;
    const uint32_t nw = std::min(nt, fa.tile_cap);
    if (tiles && tlog != tiles && nw)
      HR_CUDA(ctx, cudaMemcpyAsync(tiles, tlog, (size_t)nw * sizeof(hr_tile_record),
                                   cudaMemcpyDeviceToHost, st));
    if (!stats) HR_CUDA(ctx, cudaStreamSynchronize(st));
  }
  if (stats) {
    uint32_t ovf = 0, heavy = 0;
    unsigned long long cnt[8] = {0};
    HR_CUDA(ctx, cudaMemcpyAsync(&ovf, ctx->d_overflow, 4, cudaMemcpyDeviceToHost, st));
    if (fa.sched) HR_CUDA(ctx, cudaMemcpyAsync(&heavy, &fa.sched->n_heavy, 4, cudaMemcpyDeviceToHost, st));
    HR_CUDA(ctx, cudaMemcpyAsync(cnt, ctx->d_counters, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    HR_CUDA(ctx, cudaStreamSynchronize(st));
    float ms = 0.f;
    HR_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    std::memset(stats, 0, sizeof(*stats));
    stats->render_ms = ms;
    stats->n_samples = (uint64_t)desc->camera.width * desc->camera.height * desc->spp;
    stats->n_active_prims = a->bvh.n;
    stats->n_eth_prims = a->bvh.n_eth;
    stats->n_strand_prims = a->bvh.n - a->bvh.n_eth;
    stats->stack_overflows = ovf;
    stats->node_visits = cnt[0];
    stats->prim_tests = cnt[1];
    stats->strand_shades = cnt[2];
    stats->eth_shades = cnt[3];
    stats->shaded_hits = cnt[4];
    stats->traced_samples = cnt[5];
    stats->refined_tests = cnt[6];
    stats->refined_entries = cnt[7];
    stats->heavy_tiles = heavy;
  } else if (!dev_out) {
    HR_CUDA(ctx, cudaStreamSynchronize(st));
  }
  return HR_OK;
}

hr_status hr_render(hr_ctx* ctx, hr_asset* a, const hr_render_desc* desc, float* rgb_out,
                    hr_stats* stats) {
  API_ENTER(ctx);
  return render_impl(ctx, a, desc, rgb_out, stats);
}

hr_status hr_render_profile(hr_ctx* ctx, hr_asset* a, const hr_render_desc* desc, float* rgb_out,
                            hr_stats* stats, hr_tile_record* tiles_out, uint32_t capacity,
                            uint32_t* n_tiles) {
  API_ENTER(ctx);
  if (!tiles_out && capacity) return set_error(ctx, HR_EINVAL, "hr_render_profile: null tiles_out");
  hr_tile_record dummy;
  return render_impl(ctx, a, desc, rgb_out, stats, tiles_out ? tiles_out : &dummy,
                     tiles_out ? capacity : 0, n_tiles);
}

hr_status hr_render_samples(hr_ctx* ctx, hr_asset* a, const hr_render_desc* desc,
                            const uint32_t* sample_ids, uint32_t m, float* radiance_out,
                            int32_t* hit_out) {
  API_ENTER(ctx);
  if (!a || (m && (!sample_ids || !radiance_out || !hit_out)))
    return set_error(ctx, HR_EINVAL, "null argument");
  HR_TRY(check_desc(ctx, desc));
  if (!a->bvh.valid) return set_error(ctx, HR_ESTATE, "no BVH: call hr_build_bvh");
  if (m == 0) return HR_OK;
  cudaStream_t st = ctx->stream;
  const uint64_t total = (uint64_t)desc->camera.width * desc->camera.height * desc->spp;
  if (total > 0xffffffffull) return set_error(ctx, HR_EINVAL, "sample ids exceed 32 bits");
  const uint32_t* sid = sample_ids;
  if (!is_device_ptr(sample_ids)) {
    uint32_t* t = nullptr;
    HR_TRY(scratch(ctx, 43, (size_t)m * 4, (void**)&t));
    HR_CUDA(ctx, cudaMemcpyAsync(t, sample_ids, (size_t)m * 4, cudaMemcpyHostToDevice, st));
    sid = t;
  }
  const bool dr = is_device_ptr(radiance_out), dh = is_device_ptr(hit_out);
  float* rad = radiance_out;
  int32_t* hit = hit_out;
  if (!dr) HR_TRY(scratch(ctx, 44, (size_t)m * 12, (void**)&rad));
  const size_t hit_bytes = (size_t)m * desc->k_depth * 4;
  if (!dh) HR_TRY(scratch(ctx, 45, hit_bytes, (void**)&hit));
  FrameArgs fa = frame_args(ctx, a, a->bvh, *desc);
  HR_CUDA(ctx, cudaMemsetAsync(ctx->d_overflow, 0, 4, st));
  HR_TRY(launch_samples(ctx, fa, desc->precision, sid, m, rad, hit, st));
  if (!dr) HR_CUDA(ctx, cudaMemcpyAsync(radiance_out, rad, (size_t)m * 12, cudaMemcpyDeviceToHost, st));
  if (!dh) HR_CUDA(ctx, cudaMemcpyAsync(hit_out, hit, hit_bytes, cudaMemcpyDeviceToHost, st));
  HR_CUDA(ctx, cudaStreamSynchronize(st));
  return HR_OK;
}

hr_status hr_render_frame(hr_ctx* ctx, hr_asset* a, uint32_t n_clusters, float eps_w_px,
                          int budget_bias, const hr_render_desc* desc, float* rgb_out,
                          hr_stats* stats) {
  API_ENTER(ctx);
  if (!a || !desc) return set_error(ctx, HR_EINVAL, "null argument");
  HR_TRY(check_desc(ctx, desc));
  cudaStream_t st = ctx->stream;
  const uint8_t* lod_dev = nullptr;
  // phase events: 0 start, 3 hierarchy end, 4 LoD end, 5 BVH end; the fit's
  // and the frame's begin / end go to this call's slot of the frame-time ring
  cudaEvent_t* ph = ctx->ph;
  cudaEvent_t* rg = ctx->ring[ctx->ring_n % hr_ctx::kRing];
  bool fit_ran = false;
  const bool keep = (desc->flags & HR_FLAG_KEEP_HIERARCHY) != 0;
  // Pipelining: when the previous API call was hr_render_frame, this frame's
  // clusters and fit (which only the hierarchy build and the LoD read) run on
  // the side stream as soon as the previous frame's BVH is built, overlapping
  // that frame's rendering; they write the other cross-section buffer, so the
  // frame in flight keeps reading its own.  The thick-hair records and
  // materials, which that frame reads, follow on the main stream after it.
  // Only for a hierarchy of the same shape (no reallocation) and without a
  // serving loop.
  const bool pipe = ctx->prev_kind != 0 && !ctx->server && !keep && n_clusters > 0 &&
                    n_clusters <= a->N && a->order && a->C == n_clusters && a->E > 0 &&
                    a->xsec && !a->G;
  cudaStream_t sh = pipe ? ctx->side : st;  // the stream of the clusters and the fit
  if (pipe) {
    if (!a->xsec_other)
      HR_TRY(dalloc(ctx, (void**)&a->xsec_other, (size_t)a->E * (a->S + 1) * 3 * sizeof(float4),
                    "cross-sections (second buffer)"));
    std::swap(a->xsec, a->xsec_other);
    HR_CUDA(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_built, 0));
  }
  if (stats) HR_CUDA(ctx, cudaEventRecord(ph[0], sh));
  if (keep) {
    if (a->C == 0) return set_error(ctx, HR_ESTATE, "HR_FLAG_KEEP_HIERARCHY: no hierarchy built");
  } else if (n_clusters > 0) {
    if (n_clusters > a->N) return set_error(ctx, HR_EINVAL, "n_clusters out of range");
    HR_TRY(build_hierarchy(ctx, a, n_clusters, 0, rg[0], rg[1], pipe ? ctx->side : nullptr));
    fit_ran = a->E > 0;
  }
  const bool clustered = keep || n_clusters > 0;
  if (stats) HR_CUDA(ctx, cudaEventRecord(ph[3], st));
  const bool deferred = (desc->flags & HR_FLAG_DEFERRED_LOD) && a->lod_valid;
  if (clustered && a->n_levels > 0) {
    // Eq. 14 reads the previous selection and writes the new one in place
    const int mode = !deferred ? 0 : ((desc->flags & HR_FLAG_LOD_HYSTERESIS) ? 2 : 1);
    HR_TRY(lod_select(ctx, a, &desc->camera, eps_w_px, mode, budget_bias,
                      deferred ? a->lod : nullptr, a->lod, st));
    a->lod_valid = 1;
    lod_dev = a->lod;
  }
  if (stats) HR_CUDA(ctx, cudaEventRecord(ph[4], st));
  bool refit = false;
  if (desc->flags & HR_FLAG_REFIT) {
    refit = refit_bvh(ctx, a, lod_dev, a->bvh, st) == HR_OK;
    if (!refit) set_error(ctx, HR_OK, "");  // not refittable: rebuild
  }
  if (!refit) HR_TRY(build_bvh(ctx, a, lod_dev, a->bvh, st));
  if (stats) HR_CUDA(ctx, cudaEventRecord(ph[5], st));
  // the next frame's clusters and fit may start from here
  HR_CUDA(ctx, cudaEventRecord(ctx->ev_built, st));
  ctx->ring_fit[ctx->ring_n % hr_ctx::kRing] = (fit_ran ? 1 : 0) | (refit ? 2 : 0);
  ++ctx->ring_n;
  HR_TRY(render_impl(ctx, a, desc, rgb_out, stats, nullptr, 0, nullptr, rg[2], rg[3]));
  if (stats) {
    float h = 0.f, f = 0.f, l = 0.f, b = 0.f;
    HR_CUDA(ctx, cudaEventElapsedTime(&h, ph[0], ph[3]));
    if (fit_ran) HR_CUDA(ctx, cudaEventElapsedTime(&f, rg[0], rg[1]));
    HR_CUDA(ctx, cudaEventElapsedTime(&l, ph[3], ph[4]));
    HR_CUDA(ctx, cudaEventElapsedTime(&b, ph[4], ph[5]));
    stats->hierarchy_ms = h;
    stats->fit_ms = f;
    stats->lod_ms = l;
    stats->bvh_ms = b;
    stats->bvh_refit = refit ? 1u : 0u;
    stats->lod_deferred = deferred && clustered && a->n_levels > 0 ? 1u : 0u;
  }
  ctx->call_kind = kFrameCall;
  return HR_OK;
}

hr_status hr_frame_times(hr_ctx* ctx, uint32_t n, float* frame_ms, float* fit_ms, uint32_t* flags,
                         uint32_t* n_out) {
  API_ENTER(ctx);
  const uint64_t have = std::min<uint64_t>(ctx->ring_n, (uint64_t)hr_ctx::kRing);
  const uint32_t m = (uint32_t)std::min<uint64_t>(n, have);
  for (uint32_t i = 0; i < m; ++i) {
    const uint64_t slot = (ctx->ring_n - m + i) % hr_ctx::kRing;
    cudaEvent_t* rg = ctx->ring[slot];
    HR_CUDA(ctx, cudaEventSynchronize(rg[3]));
    float f = 0.f, g = 0.f;
    HR_CUDA(ctx, cudaEventElapsedTime(&f, rg[2], rg[3]));
    if (ctx->ring_fit[slot] & 1) HR_CUDA(ctx, cudaEventElapsedTime(&g, rg[0], rg[1]));
    if (frame_ms) frame_ms[i] = f;
    if (fit_ms) fit_ms[i] = g;
    if (flags) flags[i] = ctx->ring_fit[slot];
  }
  if (n_out) *n_out = m;
  return HR_OK;
}

}  // extern "C"
