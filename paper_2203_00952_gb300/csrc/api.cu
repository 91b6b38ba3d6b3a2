// C-ABI entry points of libsrt3d.so: context, error reporting, phase tables,
// and the argument checks of the sketch entry points (Sec. 2, Eqs. 2-3).
#include <cmath>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace srt3d {

srt3d_status set_error(srt3d_ctx* ctx, srt3d_status st, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return st;
}

srt3d_status cuda_error(srt3d_ctx* ctx, cudaError_t err, const char* what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorName(err) + " (" + cudaGetErrorString(err) + ")";
  srt3d_status st = (err == cudaErrorMemoryAllocation) ? SRT3D_ENOMEM : SRT3D_ECUDA;
  return set_error(ctx, st, msg);
}

srt3d_status grow(srt3d_ctx* ctx, DevBuf* buf, size_t bytes) {
  if (buf->bytes >= bytes) return SRT3D_OK;
  if (buf->ptr) {
    SRT3D_CUDA_TRY(ctx, cudaDeviceSynchronize());
    SRT3D_CUDA_TRY(ctx, cudaFree(buf->ptr));
    buf->ptr = nullptr;
    buf->bytes = 0;
  }
  size_t want = (bytes + 255) & ~size_t(255);
  SRT3D_CUDA_TRY(ctx, cudaMalloc(&buf->ptr, want));
  buf->bytes = want;
  return SRT3D_OK;
}

// cos/sin of 2 pi k / T in double, rounded once to float.
uint32_t phase_table_host(uint32_t T, float2* out, bool* two_level) {
  const double two_pi_over_T = 2.0 * M_PI / double(T);
  if (T <= kDirectTableMax) {
    *two_level = false;
    for (uint32_t k = 0; k < T; ++k) {
      double a = two_pi_over_T * double(k);
      out[k] = make_float2(float(std::cos(a)), float(std::sin(a)));
    }
    return T;
  }
  *two_level = true;
  const uint32_t nhi = (T + 255) / 256;
  for (uint32_t k = 0; k < 256; ++k) {
    double a = two_pi_over_T * double(k);
    out[k] = make_float2(float(std::cos(a)), float(std::sin(a)));
  }
  for (uint32_t k = 0; k < nhi; ++k) {
    double a = two_pi_over_T * double(256u * k);
    out[256 + k] = make_float2(float(std::cos(a)), float(std::sin(a)));
  }
  return 256 + nhi;
}

srt3d_status get_phase_table(srt3d_ctx* ctx, uint32_t T, PhaseTable* out) {
  std::lock_guard<std::mutex> lock(ctx->mu);
  auto it = ctx->tables.find(T);
  if (it != ctx->tables.end()) {
    *out = it->second;
    return SRT3D_OK;
  }
  PhaseTable tab;
  std::vector<float2> host(kDirectTableMax);
  tab.entries = phase_table_host(T, host.data(), &tab.two_level);
  SRT3D_CUDA_TRY(ctx, cudaMalloc(&tab.dev, size_t(tab.entries) * sizeof(float2)));
  SRT3D_CUDA_TRY(ctx, cudaMemcpy(tab.dev, host.data(), size_t(tab.entries) * sizeof(float2), cudaMemcpyHostToDevice));
  ctx->tables[T] = tab;
  *out = tab;
  return SRT3D_OK;
}

srt3d_status validate_params(srt3d_ctx* ctx, uint32_t rows, uint32_t cols, uint32_t T, uint32_t m,
                             const srt3d_params* prm) {
  if (!prm) return set_error(ctx, SRT3D_EINVAL, "params is NULL");
  if (rows == 0 || cols == 0) return set_error(ctx, SRT3D_EINVAL, "rows and cols must be >= 1");
  if (uint64_t(rows) * cols >= (1ull << 31)) return set_error(ctx, SRT3D_EINVAL, "too many pixels");
  if (T < 2 || T > 65536) return set_error(ctx, SRT3D_EINVAL, "T must be in [2, 65536]");
  if (m < 1 || m > 32 || m >= T) return set_error(ctx, SRT3D_EINVAL, "m must be in [1, min(32, T-1)]");
  if (prm->k_max < 1 || prm->k_max > 4) return set_error(ctx, SRT3D_EINVAL, "k_max must be 1..4");
  if (prm->radius < 1 || prm->radius > 3) return set_error(ctx, SRT3D_EINVAL, "radius must be 1..3");
  if (prm->init_mode != SRT3D_INIT_MATCHED && prm->init_mode != SRT3D_INIT_GIVEN)
    return set_error(ctx, SRT3D_EINVAL, "unknown init_mode");
  if (!(prm->apss_h > 0.f) || !(prm->d_max > 0.f && prm->d_max <= 1e6f) ||
      !(prm->depth_scale > 0.f && prm->depth_scale <= 1e3f) ||
      !(prm->prune_alpha >= 0.f) || !(prm->smooth_lambda >= 0.f && prm->smooth_lambda <= 1.f) ||
      !(prm->min_sep >= 0.f))
    return set_error(ctx, SRT3D_EINVAL, "invalid float parameter");
  if (prm->iters > 100000) return set_error(ctx, SRT3D_EINVAL, "iters too large");
  if (prm->weighting != 0 && prm->weighting != 1) return set_error(ctx, SRT3D_EINVAL, "weighting must be 0 or 1");
  if (prm->weighting && prm->regularize)
    return set_error(ctx, SRT3D_EINVAL, "the weighted loss is available in pixelwise mode (regularize = 0)");
  return SRT3D_OK;
}

}  // namespace srt3d

using namespace srt3d;

extern "C" {

const char* srt3d_status_string(srt3d_status s) {
  switch (s) {
    case SRT3D_OK: return "SRT3D_OK";
    case SRT3D_EINVAL: return "SRT3D_EINVAL";
    case SRT3D_ENOMEM: return "SRT3D_ENOMEM";
    case SRT3D_ERANGE: return "SRT3D_ERANGE";
    case SRT3D_ECUDA: return "SRT3D_ECUDA";
    case SRT3D_EAGAIN: return "SRT3D_EAGAIN";
    case SRT3D_ETIMEDOUT: return "SRT3D_ETIMEDOUT";
    case SRT3D_EBUSY: return "SRT3D_EBUSY";
    case SRT3D_ENOTFOUND: return "SRT3D_ENOTFOUND";
    case SRT3D_EOFFSETS: return "SRT3D_EOFFSETS";
    default: return "SRT3D_UNKNOWN";
  }
}

const char* srt3d_last_error(srt3d_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "NULL context"; }

srt3d_status srt3d_create(int device, size_t hbm_budget_bytes, srt3d_ctx** out) {
  if (!out) return SRT3D_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count <= 0) {
    cudaGetLastError();
    return SRT3D_ECUDA;
  }
  if (device < 0 || device >= count) return SRT3D_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return SRT3D_ECUDA;
  srt3d_ctx* ctx = new srt3d_ctx();
  ctx->device = device;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete ctx;
    return SRT3D_ECUDA;
  }
  ctx->num_sms = prop.multiProcessorCount;
  ctx->smem_optin = prop.sharedMemPerBlockOptin;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  ctx->hbm_budget = hbm_budget_bytes ? hbm_budget_bytes : (free_b / 4) * 3;
  if (cudaMalloc(&ctx->d_flags, sizeof(uint32_t)) != cudaSuccess ||
      cudaMemset(ctx->d_flags, 0, sizeof(uint32_t)) != cudaSuccess) {
    delete ctx;
    return SRT3D_ENOMEM;
  }
  noalloc_forget_device(device);
  if (coop_chain_init(ctx) != SRT3D_OK) {
    cudaFree(ctx->d_flags);
    delete ctx;
    return SRT3D_ECUDA;
  }
  *out = ctx;
  return SRT3D_OK;
}

void srt3d_destroy(srt3d_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  serving_destroy(ctx);
  batch_destroy(ctx);
  cudaDeviceSynchronize();
  for (auto& kv : ctx->tables) cudaFree(kv.second.dev);
  for (auto& kv : ctx->fourier) cudaFree(kv.second.ptr);
  if (ctx->rc_scratch.ptr) cudaFree(ctx->rc_scratch.ptr);
  if (ctx->hist_scratch.ptr) cudaFree(ctx->hist_scratch.ptr);
  if (ctx->d_flags) cudaFree(ctx->d_flags);
  delete ctx;
}

srt3d_status srt3d_sync(srt3d_ctx* ctx, void* stream) {
  if (!ctx) return SRT3D_EINVAL;
  SRT3D_CUDA_TRY(ctx, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  uint32_t flags = 0;
  SRT3D_CUDA_TRY(ctx, cudaMemcpy(&flags, ctx->d_flags, sizeof(flags), cudaMemcpyDeviceToHost));
  if (flags) SRT3D_CUDA_TRY(ctx, cudaMemset(ctx->d_flags, 0, sizeof(uint32_t)));
  if (flags & FLAG_OFFSETS) return set_error(ctx, SRT3D_EOFFSETS, "malformed CSR offsets seen by a kernel");
  if (flags & (FLAG_STAMP_RANGE | FLAG_COUNT_RANGE))
    return set_error(ctx, SRT3D_ERANGE,
                     (flags & FLAG_STAMP_RANGE) ? "a stamp >= T was skipped" : "a count > 65535 saturated");
  if (flags & FLAG_DEVICE_TIMEOUT) return set_error(ctx, SRT3D_ETIMEDOUT, "a device wait gave up");
  return SRT3D_OK;
}

srt3d_status srt3d_hist_from_stream(srt3d_ctx* ctx, const uint16_t* stamps, const uint32_t* offsets,
                                    uint64_t num_stamps, uint32_t num_pixels, uint32_t T, uint16_t* hist,
                                    void* stream) {
  if (!ctx) return SRT3D_EINVAL;
  if (!offsets || !hist || (num_stamps && !stamps)) return set_error(ctx, SRT3D_EINVAL, "NULL pointer");
  if (T < 1 || T > 65536) return set_error(ctx, SRT3D_EINVAL, "T must be in [1, 65536]");
  if (num_stamps >= (1ull << 32)) return set_error(ctx, SRT3D_EINVAL, "num_stamps must be < 2^32");
  if (num_pixels == 0) return SRT3D_OK;
  return launch_hist_from_stream(ctx, stamps, offsets, num_stamps, num_pixels, T, hist,
                                 static_cast<cudaStream_t>(stream));
}

srt3d_status srt3d_sketch_stream(srt3d_ctx* ctx, const uint16_t* stamps, const uint32_t* offsets,
                                 uint64_t num_stamps, uint32_t num_pixels, uint32_t T, uint32_t m,
                                 int accumulate, float* S, uint32_t* n, void* stream) {
  if (!ctx) return SRT3D_EINVAL;
  if (!offsets || !S || !n || (num_stamps && !stamps)) return set_error(ctx, SRT3D_EINVAL, "NULL pointer");
  if (T < 1 || T > 65536) return set_error(ctx, SRT3D_EINVAL, "T must be in [1, 65536]");
  if (m < 1 || m > 32) return set_error(ctx, SRT3D_EINVAL, "m must be in [1, 32]");
  if (num_stamps >= (1ull << 32) - 16) return set_error(ctx, SRT3D_EINVAL, "num_stamps must be < 2^32 - 16");
  if (reinterpret_cast<uintptr_t>(S) % 8) return set_error(ctx, SRT3D_EINVAL, "S must be 8-byte aligned");
  if (num_pixels == 0) return SRT3D_OK;
  // 0 overwrite, 1 accumulate (any other nonzero value too), 2 store z = S / n
  const int mode = accumulate == 2 ? 2 : (accumulate ? 1 : 0);
  return launch_sketch_stream(ctx, stamps, offsets, num_stamps, num_pixels, T, m, mode,
                              reinterpret_cast<float2*>(S), n, static_cast<cudaStream_t>(stream));
}

srt3d_status srt3d_finalize(srt3d_ctx* ctx, const float* S, const uint32_t* n, uint32_t num_pixels,
                            uint32_t m, float* z, void* stream) {
  if (!ctx) return SRT3D_EINVAL;
  if (!S || !n || !z) return set_error(ctx, SRT3D_EINVAL, "NULL pointer");
  if (m < 1 || m > 32) return set_error(ctx, SRT3D_EINVAL, "m must be in [1, 32]");
  if ((reinterpret_cast<uintptr_t>(S) | reinterpret_cast<uintptr_t>(z)) % 8)
    return set_error(ctx, SRT3D_EINVAL, "S and z must be 8-byte aligned");
  if (num_pixels == 0) return SRT3D_OK;
  return launch_finalize(ctx, reinterpret_cast<const float2*>(S), n, num_pixels, m,
                         reinterpret_cast<float2*>(z), static_cast<cudaStream_t>(stream));
}

}  // extern "C"

extern "C" srt3d_status srt3d_plan(uint32_t rows, uint32_t cols, uint32_t T, uint32_t m, uint32_t k_max,
                                   uint32_t radius, double mean_photons_per_pixel, uint32_t num_sms,
                                   uint32_t ctas_per_sm, srt3d_plan_info* out) {
  using namespace srt3d;
  if (!out || rows == 0 || cols == 0 || T < 2 || T > 65536 || m < 1 || m > 32 || k_max < 1 || k_max > 4 ||
      radius < 1 || radius > 3 || num_sms == 0 || num_sms > 4096 || ctas_per_sm == 0 || ctas_per_sm > 64 ||
      !(mean_photons_per_pixel >= 0.0))
    return SRT3D_EINVAL;
  srt3d_plan_info info{};
  info.sketch_m = uint32_t(sketch_round_m(m));
  info.sketch_lanes = 1u << sketch_default_glog2(mean_photons_per_pixel);
  info.init_m = uint32_t(init_round_m(m));
  info.init_grid_spacing = mf_grid_spacing_host(T, m);
  info.init_grid_points = (T + info.init_grid_spacing - 1) / info.init_grid_spacing;
  info.tile_height = plan_tile_height(k_max, radius, rows, cols, int(num_sms), int(ctas_per_sm));
  const uint32_t tiles_x = (cols + 15u) / 16u;
  info.tiles = info.tile_height ? tiles_x * ((rows + info.tile_height - 1) / info.tile_height) : 0u;
  info.serving_frame_bytes = uint64_t(serving_frame_bytes(rows, cols, T, m, k_max));
  *out = info;
  return SRT3D_OK;
}
