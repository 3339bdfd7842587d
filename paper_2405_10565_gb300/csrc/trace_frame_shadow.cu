// Frame kernel with dual-scattering shadow rays (HR_FLAG_SHADOWS), in its own
// translation unit so that it compiles in parallel with the plain one.
#include "trace_frame.cuh"

namespace hr {

hr_status launch_frame_shadow(hr_ctx* ctx, const FrameArgs& fa, int precision, bool count,
                              float* rgb_dev, cudaStream_t st) {
  return launch_frame_t<true>(ctx, fa, precision, count, rgb_dev, st);
}

}  // namespace hr
