// Serving runtime: continuous batching of render requests.
//
// A scheduler thread owns a CUDA stream and a fixed number of slots.  A
// submitted request waits in a FIFO queue until a slot is free and the
// context's bytes in use plus the request's estimate stay under the HBM budget;
// admission then selects its LoD (initial rule with the request's epsilon_w and
// budget bias) and builds its BVH into slot-resident, grow-only buffers.  Each
// scheduling round packs tiles of every active request (a fair share each,
// oldest first) into one persistent launch of the batched tile kernel, so
// requests that arrive while others render join the next launch and their work
// shares the device.  Batches are double-buffered; a request completes when the
// event recorded after its last tile (and its copy to a host buffer) fires, and
// its completion time is read from that event.  Nothing on the device ever
// waits: host waits are polls of events with bounded sleeps.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>
#include <vector>

#include "serve.h"

namespace hr {

Server** ctx_server_slot(hr_ctx* ctx);
uint64_t ctx_budget(hr_ctx* ctx);

namespace {

// A BVH kept resident for an (asset, LoD) pair; requests with the same pair
// share it.
struct CachedBvh {
  hr_asset* asset = nullptr;
  std::vector<uint8_t> lod;
  Bvh bvh;
  int refs = 0;
  uint64_t last_use = 0;
};

struct Slot {
  uint8_t* lod = nullptr;
  uint32_t lod_cap = 0;
  float4* rect = nullptr;  // the request's projected scene rectangle (device)
  float* out = nullptr;  // device staging when the caller's buffer is host memory
  size_t out_cap = 0;
  bool busy = false;
};

struct Request {
  uint64_t ticket = 0;
  hr_request req{};
  double submit_ms = 0, admit_ms = -1, done_ms = -1, ready_ms = -1;
  hr_status status = HR_ENOTREADY;
  int slot = -1;
  uint32_t tiles_total = 0, tiles_issued = 0;
  bool host_out = false;
  bool finished_issue = false;
  cudaEvent_t done_ev = nullptr;
  CachedBvh* entry = nullptr;
  int kmax = 1;
  FrameArgs fa{};
  float4 rect{};   // projected scene rectangle (pixels)
  WarpGrid grid{};  // warp tiles over it (tiles_total of them)
  float* dev_out = nullptr;
  int64_t delay_ms = 0;
};

}  // namespace

struct Server {
  hr_ctx* ctx = nullptr;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  bool stop = false;
  std::deque<Request*> pending;
  std::vector<Request*> active;
  std::map<uint64_t, Request*> all;
  std::vector<Slot> slots;
  uint64_t max_batch_samples = 0;
  cudaStream_t stream = nullptr;
  ServeItem* h_items[2] = {nullptr, nullptr};
  ServeItem* d_items[2] = {nullptr, nullptr};
  uint32_t* h_starts[2] = {nullptr, nullptr};
  uint32_t* d_starts[2] = {nullptr, nullptr};
  uint32_t* d_work = nullptr;
  cudaEvent_t batch_ev[2] = {nullptr, nullptr};
  cudaEvent_t ref_ev = nullptr;
  double ref_ms = 0;
  int buf = 0;
  uint32_t max_items = 0;
  uint64_t next_ticket = 1;
  int inject_nomem = 0;
  int64_t inject_delay = 0;
  uint64_t launches = 0;
  cudaStream_t build_stream = nullptr;  // LoD + BVH builds, overlapping the batches
  std::vector<CachedBvh*> cache;
  uint64_t use_clock = 0;
  uint64_t cache_hits = 0, cache_misses = 0;
};

namespace {

constexpr uint32_t kMaxItems = 4096;
constexpr size_t kMaxPending = 1 << 16;

double event_ms(Server* s, cudaEvent_t ev) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, s->ref_ev, ev) != cudaSuccess) {
    cudaGetLastError();
    return ctx_now_ms(s->ctx);
  }
  return s->ref_ms + ms;
}

// Upper bound of the device bytes admitting a request may add: a new resident
// BVH over every primitive of its asset (as if its LoD were not cached), and
// the growth of the slot's LoD and staging buffers.
uint64_t estimate_bytes(const Request* r, const Slot& sl) {
  const hr_asset* a = r->req.asset;
  uint64_t need = (uint64_t)a->n_prims_total * (4 * 16 + 3 * 16 + 16 + 4);
  const size_t out = (size_t)r->req.desc.camera.width * r->req.desc.camera.height * 12;
  if (r->host_out && out > sl.out_cap) need += out - sl.out_cap;
  if (a->C > sl.lod_cap) need += a->C - sl.lod_cap;
  return need;
}

constexpr size_t kMaxCached = 64;

// Free the least recently used resident BVHs that no request holds, while
// more than `keep` entries remain (keep = 0: every unreferenced one).
void evict(Server* s, size_t keep) {
  hr_ctx* ctx = s->ctx;
  for (;;) {
    if (s->cache.size() <= keep) return;
    int victim = -1;
    for (size_t i = 0; i < s->cache.size(); ++i)
      if (s->cache[i]->refs == 0 &&
          (victim < 0 || s->cache[i]->last_use < s->cache[victim]->last_use))
        victim = (int)i;
    if (victim < 0) return;
    free_bvh(ctx, s->cache[victim]->bvh);
    delete s->cache[victim];
    s->cache.erase(s->cache.begin() + victim);
  }
}

// Admission: LoD of one request, then its resident BVH (shared when the same
// asset and LoD are already resident, built otherwise), on the build stream
// and holding the API lock so the context scratch is not shared with a
// concurrent call.
hr_status admit(Server* s, Request* r) {
  hr_ctx* ctx = s->ctx;
  std::lock_guard<std::recursive_mutex> g(ctx_mutex(ctx));
  cudaStream_t bs = s->build_stream;
  Slot& sl = s->slots[r->slot];
  hr_asset* a = r->req.asset;
  const uint8_t* lod = nullptr;
  std::vector<uint8_t> lod_h;
  if (a->n_levels > 0) {
    if (sl.lod_cap < a->C) {
      if (sl.lod) {
        cudaStreamSynchronize(bs);
        dfree(ctx, sl.lod, sl.lod_cap);
        sl.lod = nullptr;
        sl.lod_cap = 0;
      }
      HR_TRY(dalloc(ctx, (void**)&sl.lod, a->C, "serving LoD"));
      sl.lod_cap = a->C;
    }
    HR_TRY(lod_select(ctx, a, &r->req.desc.camera, r->req.eps_w_px, 0, r->req.budget_bias,
                      nullptr, sl.lod, bs));
    lod = sl.lod;
    lod_h.resize(a->C);
    HR_CUDA(ctx, cudaMemcpyAsync(lod_h.data(), sl.lod, a->C, cudaMemcpyDeviceToHost, bs));
    HR_CUDA(ctx, cudaStreamSynchronize(bs));
  }
  CachedBvh* e = nullptr;
  for (CachedBvh* c : s->cache)
    if (c->asset == a && c->lod == lod_h) {
      e = c;
      break;
    }
  if (e) {
    s->cache_hits++;
  } else {
    s->cache_misses++;
    evict(s, kMaxCached - 1);
    e = new CachedBvh();
    e->asset = a;
    e->lod = lod_h;
    const hr_status st = build_bvh(ctx, a, lod, e->bvh, bs);
    if (st != HR_OK) {
      free_bvh(ctx, e->bvh);
      delete e;
      return st;
    }
    s->cache.push_back(e);
  }
  e->refs++;
  e->last_use = ++s->use_clock;
  r->entry = e;
  const size_t out = (size_t)r->req.desc.camera.width * r->req.desc.camera.height * 12;
  r->dev_out = r->req.rgb_out;
  if (r->host_out) {
    if (sl.out_cap < out) {
      if (sl.out) {
        cudaStreamSynchronize(s->stream);
        dfree(ctx, sl.out, sl.out_cap);
        sl.out = nullptr;
        sl.out_cap = 0;
      }
      HR_TRY(dalloc(ctx, (void**)&sl.out, out, "serving output"));
      sl.out_cap = out;
    }
    r->dev_out = sl.out;
  }
  // the warp tiles over the projected scene rectangle
  r->fa = frame_args(ctx, a, e->bvh, r->req.desc);
  r->kmax = kmax_for(r->req.desc.k_depth);
  if (!sl.rect) HR_TRY(dalloc(ctx, (void**)&sl.rect, sizeof(float4), "serving rect"));
  HR_TRY(launch_scene_rect(ctx, r->fa, sl.rect, bs));
  HR_CUDA(ctx, cudaMemcpyAsync(&r->rect, sl.rect, sizeof(float4), cudaMemcpyDeviceToHost, bs));
  // the build must be complete before the batches (another stream) read it,
  // and the scratch it used is shared with API calls
  HR_CUDA(ctx, cudaStreamSynchronize(bs));
  r->grid = warp_grid(r->rect, r->req.desc.camera.width, r->req.desc.camera.height, r->fa.grp);
  r->tiles_total = r->grid.n;
  // every pixel outside the warp tiles is background: clear the output on the
  // batch stream, ahead of the request's tiles
  HR_CUDA(ctx, cudaMemsetAsync(r->dev_out, 0, out, s->stream));
  if (r->tiles_total == 0) {  // nothing in view: complete with the background
    r->finished_issue = true;
    if (r->host_out)
      HR_CUDA(ctx, cudaMemcpyAsync(r->req.rgb_out, r->dev_out, out, cudaMemcpyDeviceToHost,
                                   s->stream));
    HR_CUDA(ctx, cudaEventRecord(r->done_ev, s->stream));
  }
  return HR_OK;
}

void finish(Server* s, Request* r, hr_status st, double done_ms) {
  r->status = st;
  r->done_ms = done_ms;
  r->ready_ms = ctx_now_ms(s->ctx) + (double)r->delay_ms;
  if (r->slot >= 0) s->slots[r->slot].busy = false;
  r->slot = -1;
  if (r->entry) {
    r->entry->refs--;
    r->entry = nullptr;
  }
}

void loop(Server* s) {
  hr_ctx* ctx = s->ctx;
  cudaSetDevice(ctx_device(ctx));
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    bool progressed = false;
    // 1. admissions (FIFO, while a slot is free and the budget allows)
    while (!s->pending.empty()) {
      Request* r = s->pending.front();
      // the free slot whose resident buffers need the least growth
      int slot = -1;
      uint64_t best = ~0ull;
      for (size_t i = 0; i < s->slots.size(); ++i)
        if (!s->slots[i].busy) {
          const uint64_t nd = estimate_bytes(r, s->slots[i]);
          if (nd < best) {
            best = nd;
            slot = (int)i;
          }
        }
      if (slot < 0) break;
      if (s->inject_nomem) {
        s->inject_nomem = 0;
        s->pending.pop_front();
        finish(s, r, HR_ENOMEM, ctx_now_ms(ctx));
        s->cv_done.notify_all();
        progressed = true;
        continue;
      }
      // admission by free HBM: the bytes the slot must grow by have to fit in
      // the context budget (or, without one, in the device's free memory)
      uint64_t need = estimate_bytes(r, s->slots[slot]);
      auto fits = [&]() {
        if (need == 0) return true;
        const uint64_t budget = ctx_budget(ctx);
        if (budget) return hr_bytes_in_use(ctx) + need <= budget;
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
          cudaGetLastError();
          return false;
        }
        return need <= fr;
      };
      if (!fits()) {
        // reclaim unreferenced resident BVHs and idle slots' buffers, retry
        std::lock_guard<std::recursive_mutex> g(ctx_mutex(ctx));
        cudaStreamSynchronize(s->stream);
        evict(s, 0);
        for (size_t i = 0; i < s->slots.size(); ++i) {
          Slot& sl = s->slots[i];
          if (sl.busy || (int)i == slot) continue;
          if (sl.lod) dfree(ctx, sl.lod, sl.lod_cap);
          if (sl.out) dfree(ctx, sl.out, sl.out_cap);
          sl.lod = nullptr;
          sl.out = nullptr;
          sl.lod_cap = 0;
          sl.out_cap = 0;
        }
        need = estimate_bytes(r, s->slots[slot]);
      }
      if (!fits()) {
        if (!s->active.empty()) break;  // wait for running requests to finish
        s->pending.pop_front();
        finish(s, r, HR_ENOMEM, ctx_now_ms(ctx));
        s->cv_done.notify_all();
        progressed = true;
        continue;
      }
      s->pending.pop_front();
      r->slot = slot;
      s->slots[slot].busy = true;
      lk.unlock();
      hr_status st = admit(s, r);
      lk.lock();
      if (st != HR_OK) {
        finish(s, r, st, ctx_now_ms(ctx));
        s->cv_done.notify_all();
      } else {
        r->admit_ms = ctx_now_ms(ctx);
        s->active.push_back(r);
      }
      progressed = true;
    }
    // 2. one batch: requests with tiles left that share the oldest one's
    //    kernel variant, a fair share of tiles each
    Request* head = nullptr;
    for (Request* r : s->active)
      if (!r->finished_issue) {
        head = r;
        break;
      }
    if (head) {
      const int kmax = head->kmax, prec = head->req.desc.precision;
      std::vector<Request*> grp;
      for (Request* r : s->active)
        if (!r->finished_issue && r->kmax == kmax && r->req.desc.precision == prec) grp.push_back(r);
      uint64_t budget = s->max_batch_samples;
      const int b = s->buf;
      lk.unlock();
      cudaEventSynchronize(s->batch_ev[b]);  // the buffers of two batches ago are free
      lk.lock();
      uint32_t n_items = 0, total = 0;
      std::vector<Request*> completing;
      const uint64_t share = std::max<uint64_t>(1, budget / grp.size());
      for (Request* r : grp) {
        if (n_items >= s->max_items) break;
        // samples per warp tile: 32 / grp pixels of spp samples each
        const uint64_t spt = (uint64_t)(32u / r->fa.grp) * r->req.desc.spp;
        uint32_t take = (uint32_t)std::max<uint64_t>(1, share / spt);
        take = std::min(take, r->tiles_total - r->tiles_issued);
        ServeItem& it = s->h_items[b][n_items];
        it.fa = r->fa;
        it.rgb = r->dev_out;
        it.rect = r->rect;
        it.grid = r->grid;
        it.wt0 = r->tiles_issued;
        it.nwt = take;
        s->h_starts[b][n_items] = total;
        total += take;
        ++n_items;
        r->tiles_issued += take;
        if (r->tiles_issued == r->tiles_total) {
          r->finished_issue = true;
          completing.push_back(r);
        }
      }
      s->h_starts[b][n_items] = total;
      lk.unlock();
      cudaStream_t st = s->stream;
      cudaMemcpyAsync(s->d_items[b], s->h_items[b], n_items * sizeof(ServeItem),
                      cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(s->d_starts[b], s->h_starts[b], (n_items + 1) * 4, cudaMemcpyHostToDevice, st);
      cudaMemsetAsync(s->d_work + b, 0, 4, st);
      hr_status ls = launch_serve_batch(ctx, kmax, prec, s->d_items[b], s->d_starts[b], n_items,
                                        total, s->d_work + b, serve_grid(kmax, prec), st);
      cudaEventRecord(s->batch_ev[b], st);
      for (Request* r : completing) {
        if (r->host_out)
          cudaMemcpyAsync(r->req.rgb_out, r->dev_out,
                          (size_t)r->req.desc.camera.width * r->req.desc.camera.height * 12,
                          cudaMemcpyDeviceToHost, st);
        cudaEventRecord(r->done_ev, st);
      }
      lk.lock();
      s->launches++;
      s->buf ^= 1;
      if (ls != HR_OK)
        for (Request* r : completing) r->status = ls;
      progressed = true;
    }
    // 3. completions
    for (size_t i = 0; i < s->active.size();) {
      Request* r = s->active[i];
      if (r->finished_issue && cudaEventQuery(r->done_ev) == cudaSuccess) {
        const hr_status st = r->status == HR_ENOTREADY ? HR_OK : r->status;
        finish(s, r, st, event_ms(s, r->done_ev));
        s->active.erase(s->active.begin() + i);
        s->cv_done.notify_all();
        progressed = true;
      } else {
        ++i;
      }
    }
    if (!progressed) s->cv.wait_for(lk, std::chrono::microseconds(200));
  }
}

}  // namespace

void serve_forget_asset(hr_ctx* ctx, Server* s, hr_asset* a) {
  std::unique_lock<std::mutex> lk(s->mu);
  for (auto it = s->pending.begin(); it != s->pending.end();) {
    if ((*it)->req.asset == a) {
      finish(s, *it, HR_ESTATE, ctx_now_ms(ctx));
      it = s->pending.erase(it);
    } else {
      ++it;
    }
  }
  s->cv_done.notify_all();
  for (int i = 0; i < 100000; ++i) {  // bounded: at most ~100 s
    bool busy = false;
    for (Request* r : s->active) busy |= r->req.asset == a;
    if (!busy) break;
    s->cv_done.wait_for(lk, std::chrono::milliseconds(1));
  }
  for (size_t i = 0; i < s->cache.size();) {
    CachedBvh* c = s->cache[i];
    if (c->asset == a && c->refs == 0) {
      free_bvh(ctx, c->bvh);
      delete c;
      s->cache.erase(s->cache.begin() + i);
    } else {
      ++i;
    }
  }
}

}  // namespace hr

using namespace hr;

extern "C" {

hr_status hr_serve_start(hr_ctx* ctx, uint32_t max_slots, uint64_t max_batch_samples) {
  if (!ctx) return HR_EINVAL;
  std::lock_guard<std::recursive_mutex> g(ctx_mutex(ctx));
  Server** slot = ctx_server_slot(ctx);
  if (*slot) return set_error(ctx, HR_ESTATE, "serving already started");
  if (max_slots < 1 || max_slots > 1024 || max_batch_samples < 1)
    return set_error(ctx, HR_EINVAL, "max_slots / max_batch_samples");
  cudaSetDevice(ctx_device(ctx));
  Server* s = new Server();
  s->ctx = ctx;
  s->slots.resize(max_slots);
  s->max_batch_samples = max_batch_samples;
  s->max_items = std::min<uint32_t>(kMaxItems, std::max<uint32_t>(max_slots, 1));
  bool ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&s->build_stream, cudaStreamNonBlocking) == cudaSuccess;
  for (int b = 0; b < 2 && ok; ++b) {
    const size_t ni = s->max_items;
    ok &= cudaMallocHost((void**)&s->h_items[b], ni * sizeof(ServeItem)) == cudaSuccess;
    ok &= cudaMallocHost((void**)&s->h_starts[b], (ni + 1) * 4) == cudaSuccess;
    ok &= dalloc(ctx, (void**)&s->d_items[b], ni * sizeof(ServeItem), "serve items") == HR_OK;
    ok &= dalloc(ctx, (void**)&s->d_starts[b], (ni + 1) * 4, "serve starts") == HR_OK;
    ok &= cudaEventCreateWithFlags(&s->batch_ev[b], cudaEventDisableTiming) == cudaSuccess;
  }
  ok = ok && dalloc(ctx, (void**)&s->d_work, 16, "serve work") == HR_OK;
  ok = ok && cudaEventCreate(&s->ref_ev) == cudaSuccess;
  if (ok) {
    cudaEventRecord(s->ref_ev, s->stream);
    cudaEventSynchronize(s->ref_ev);
    s->ref_ms = ctx_now_ms(ctx);
    for (int b = 0; b < 2; ++b) cudaEventRecord(s->batch_ev[b], s->stream);
  }
  *slot = s;
  if (!ok) {
    hr_serve_stop(ctx);
    return set_error(ctx, HR_ECUDA, "serving start failed");
  }
  s->th = std::thread(loop, s);
  return HR_OK;
}

hr_status hr_serve_stop(hr_ctx* ctx) {
  if (!ctx) return HR_EINVAL;
  Server* s = *ctx_server_slot(ctx);
  if (!s) return set_error(ctx, HR_ESTATE, "serving not started");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->th.joinable()) s->th.join();
  std::lock_guard<std::recursive_mutex> g(ctx_mutex(ctx));
  cudaSetDevice(ctx_device(ctx));
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto& kv : s->all) {
    Request* r = kv.second;
    if (r->done_ev) cudaEventDestroy(r->done_ev);
    delete r;
  }
  if (s->build_stream) cudaStreamSynchronize(s->build_stream);
  for (CachedBvh* c : s->cache) {
    free_bvh(ctx, c->bvh);
    delete c;
  }
  s->cache.clear();
  for (Slot& sl : s->slots) {
    if (sl.lod) dfree(ctx, sl.lod, sl.lod_cap);
    if (sl.out) dfree(ctx, sl.out, sl.out_cap);
    if (sl.rect) dfree(ctx, sl.rect, sizeof(float4));
  }
  for (int b = 0; b < 2; ++b) {
    if (s->h_items[b]) cudaFreeHost(s->h_items[b]);
    if (s->h_starts[b]) cudaFreeHost(s->h_starts[b]);
    if (s->d_items[b]) dfree(ctx, s->d_items[b], s->max_items * sizeof(ServeItem));
    if (s->d_starts[b]) dfree(ctx, s->d_starts[b], (s->max_items + 1) * 4);
    if (s->batch_ev[b]) cudaEventDestroy(s->batch_ev[b]);
  }
  if (s->d_work) dfree(ctx, s->d_work, 16);
  if (s->ref_ev) cudaEventDestroy(s->ref_ev);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->build_stream) cudaStreamDestroy(s->build_stream);
  delete s;
  *ctx_server_slot(ctx) = nullptr;
  return HR_OK;
}

hr_status hr_submit(hr_ctx* ctx, const hr_request* req, uint64_t* ticket) {
  if (!ctx || !req || !ticket) return HR_EINVAL;
  Server* s = *ctx_server_slot(ctx);
  if (!s) return set_error(ctx, HR_ESTATE, "serving not started");
  if (!req->asset || !req->rgb_out) return set_error(ctx, HR_EINVAL, "request asset / output");
  HR_TRY(check_desc(ctx, &req->desc));
  if (req->budget_bias < 0) return set_error(ctx, HR_EINVAL, "budget_bias");
  if (req->desc.flags & (HR_FLAG_SHADOWS | HR_FLAG_COUNT))
    return set_error(ctx, HR_EINVAL, "serving renders primary hits only (no shadow rays, no counting)");
  Request* r = new Request();
  r->req = *req;
  r->host_out = !is_device_ptr(req->rgb_out);
  {
    std::lock_guard<std::recursive_mutex> g(ctx_mutex(ctx));
    cudaSetDevice(ctx_device(ctx));
    if (cudaEventCreateWithFlags(&r->done_ev, cudaEventDefault) != cudaSuccess) {
      delete r;
      return set_error(ctx, HR_ECUDA, "event create");
    }
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->pending.size() >= kMaxPending) {
    cudaEventDestroy(r->done_ev);
    delete r;
    return set_error(ctx, HR_EBUSY, "serving queue full");
  }
  r->ticket = s->next_ticket++;
  r->submit_ms = ctx_now_ms(ctx);
  if (s->inject_delay) {
    r->delay_ms = s->inject_delay;
    s->inject_delay = 0;
  }
  s->pending.push_back(r);
  s->all[r->ticket] = r;
  *ticket = r->ticket;
  s->cv.notify_all();
  return HR_OK;
}

hr_status hr_poll(hr_ctx* ctx, uint64_t ticket, int timeout_ms, hr_result* res) {
  if (!ctx) return HR_EINVAL;
  Server* s = *ctx_server_slot(ctx);
  if (!s) return set_error(ctx, HR_ESTATE, "serving not started");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return set_error(ctx, HR_EINVAL, "unknown ticket");
  Request* r = it->second;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
  for (;;) {
    const bool done = r->status != HR_ENOTREADY && ctx_now_ms(ctx) >= r->ready_ms;
    if (done) break;
    if (std::chrono::steady_clock::now() >= deadline)
      return timeout_ms > 0 ? HR_ETIMEOUT : HR_ENOTREADY;
    s->cv_done.wait_until(lk, std::min(deadline, std::chrono::steady_clock::now() +
                                                     std::chrono::milliseconds(1)));
  }
  if (res) {
    res->status = r->status;
    res->submit_ms = r->submit_ms;
    res->admit_ms = r->admit_ms;
    res->done_ms = r->done_ms;
    res->n_samples = (uint64_t)r->req.desc.camera.width * r->req.desc.camera.height * r->req.desc.spp;
  }
  return HR_OK;
}

hr_status hr_serve_inject(hr_ctx* ctx, int kind, int64_t arg) {
  if (!ctx) return HR_EINVAL;
  Server* s = *ctx_server_slot(ctx);
  if (!s) return set_error(ctx, HR_ESTATE, "serving not started");
  std::lock_guard<std::mutex> lk(s->mu);
  if (kind == 1) s->inject_nomem = 1;
  else if (kind == 2) s->inject_delay = std::max<int64_t>(0, arg);
  else return set_error(ctx, HR_EINVAL, "inject kind");
  return HR_OK;
}

}  // extern "C"
