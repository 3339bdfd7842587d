// Serving runtime (continuous batching of render requests).
#pragma once

#include <mutex>

#include "common.cuh"

namespace hr {

struct Server;

std::recursive_mutex& ctx_mutex(hr_ctx* ctx);
double ctx_now_ms(hr_ctx* ctx);
int ctx_device(hr_ctx* ctx);
uint32_t* ctx_overflow(hr_ctx* ctx);
bool is_device_ptr(const void* p);
hr_status check_desc(hr_ctx* ctx, const hr_render_desc* d);
FrameArgs frame_args(hr_ctx* ctx, hr_asset* a, const Bvh& bv, const hr_render_desc& d);
int serve_grid(int kmax, int precision);

// Cancel pending requests on `a` and wait for its in-flight ones to finish.
void serve_forget_asset(hr_ctx* ctx, Server* s, hr_asset* a);

}  // namespace hr
