// Serving runtime (placeholder until continuous batching lands).
#include "internal.h"

namespace srt3d {
void serving_destroy(srt3d_ctx*) {}
}  // namespace srt3d

using namespace srt3d;

extern "C" srt3d_status srt3d_submit(srt3d_ctx* ctx, uint64_t, uint32_t, uint32_t, uint32_t, uint32_t, const float*,
                                     const srt3d_params*, const uint16_t*, const uint32_t*, int) {
  return set_error(ctx, SRT3D_EINVAL, "serving not available in this build");
}

extern "C" srt3d_status srt3d_poll(srt3d_ctx* ctx, uint64_t, uint32_t, float*, float*, uint8_t*, float*, uint32_t*) {
  return set_error(ctx, SRT3D_EINVAL, "serving not available in this build");
}
