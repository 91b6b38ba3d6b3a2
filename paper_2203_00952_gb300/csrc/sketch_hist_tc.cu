// Tensor-core histogram sketch (placeholder until the tcgen05 kernel lands).
#include "internal.h"

namespace srt3d {

srt3d_status launch_sketch_hist_tc(srt3d_ctx* ctx, const uint16_t*, uint32_t, uint32_t, uint32_t, int, float2*,
                                   uint32_t*, cudaStream_t) {
  return set_error(ctx, SRT3D_EINVAL, "tensor-core histogram sketch not available in this build");
}

}  // namespace srt3d
