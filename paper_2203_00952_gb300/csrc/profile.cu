// Per-kernel CUDA-event timing (a measurement aid; no counterpart in the paper).
#include "internal.h"

namespace srt3d {

static const char* kKernelNames[KID_COUNT] = {
    "sketch_stream", "finalize", "hist_from_stream", "sketch_hist_fp32", "sketch_hist_tc",
    "prep",          "init",     "grad",             "iter",             "iter_all",         "alpha0",
    "batch_graph",   "birth",    "bucket_stream",    "sketch_stream_tc"};

static cudaEvent_t take_event(Profiler& pf) {
  if (!pf.pool.empty()) {
    cudaEvent_t e = pf.pool.back();
    pf.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

ProfMark prof_begin(srt3d_ctx* ctx, uint32_t kid, cudaStream_t stream) {
  ProfMark mk;
  if (!ctx->prof.enabled) return mk;
  std::lock_guard<std::mutex> lock(ctx->prof.mu);
  mk.a = take_event(ctx->prof);
  mk.b = take_event(ctx->prof);
  if (mk.a) cudaEventRecord(mk.a, stream);
  (void)kid;
  return mk;
}

void prof_end(srt3d_ctx* ctx, uint32_t kid, const ProfMark& mk, cudaStream_t stream, uint32_t kernels) {
  if (!mk.a || !mk.b) return;
  cudaEventRecord(mk.b, stream);
  std::lock_guard<std::mutex> lock(ctx->prof.mu);
  ctx->prof.pending.push_back({kid, mk.a, mk.b, kernels});
}

static void drain(Profiler& pf) {
  for (auto& p : pf.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      pf.total_ms[p.kid] += ms;
      pf.launches[p.kid] += p.kernels;
    }
    pf.pool.push_back(p.a);
    pf.pool.push_back(p.b);
  }
  pf.pending.clear();
}

}  // namespace srt3d

using namespace srt3d;

extern "C" {

srt3d_status srt3d_profile_enable(srt3d_ctx* ctx, int enable) {
  if (!ctx) return SRT3D_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->prof.mu);
  drain(ctx->prof);
  if (enable) {
    for (uint32_t k = 0; k < KID_COUNT; ++k) {
      ctx->prof.total_ms[k] = 0.0;
      ctx->prof.launches[k] = 0;
    }
  }
  ctx->prof.enabled = enable != 0;
  return SRT3D_OK;
}

srt3d_status srt3d_profile_read(srt3d_ctx* ctx, uint32_t kernel, double* total_ms, uint64_t* launches) {
  if (!ctx || kernel >= KID_COUNT) return SRT3D_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->prof.mu);
  drain(ctx->prof);
  if (total_ms) *total_ms = ctx->prof.total_ms[kernel];
  if (launches) *launches = ctx->prof.launches[kernel];
  return SRT3D_OK;
}

uint32_t srt3d_kernel_count(void) { return KID_COUNT; }

const char* srt3d_kernel_name(uint32_t kernel) { return kernel < KID_COUNT ? kKernelNames[kernel] : "unknown"; }

}  // extern "C"
