// Histogram sketch (Sec. 2, Eqs. 2-3): Z[P x 2m] = Y[P x T] F[T x 2m] with
// F[b][2(l-1)] = cos(2 pi ((l b) mod T) / T), F[b][2(l-1)+1] = sin(...).
//
// SRT3D_FP32: CUDA-core product. A 256-thread CTA owns 64 pixels x 64
// columns; bins stream through shared memory in chunks of 64 (Y as float,
// transposed, F generated from the exact integer phase and the cos/sin
// table). Each thread accumulates a 4 x 4 register tile; every chunk's
// partial products are summed separately before joining the running total,
// so the FP32 rounding error grows with T/64 + 64 terms rather than T.
// The tensor-core precisions live in sketch_hist_tc.cu.
#include "device_util.cuh"
#include "internal.h"

namespace srt3d {

srt3d_status launch_sketch_hist_tc(srt3d_ctx* ctx, const uint16_t* hist, uint32_t P, uint32_t T, uint32_t m,
                                   int precision, float2* S, uint32_t* n, cudaStream_t stream);
size_t stream_tc_fused_scratch_bytes(uint64_t num_stamps, uint32_t P, uint32_t T);
srt3d_status launch_sketch_stream_tc_fused(srt3d_ctx* ctx, const uint16_t* stamps, const uint32_t* offsets,
                                           uint64_t num_stamps, uint32_t P, uint32_t T, uint32_t m, int precision,
                                           float2* S, uint32_t* n, void* scratch, cudaStream_t stream);

namespace {

constexpr int kTileP = 64;
constexpr int kTileB = 64;
constexpr int kCols = 64;

__global__ void __launch_bounds__(256) k_sketch_hist_fp32(const uint16_t* __restrict__ hist, uint32_t P, uint32_t T,
                                                          uint32_t m, const float2* __restrict__ table,
                                                          uint32_t entries, int two_level, float2* __restrict__ S,
                                                          uint32_t* __restrict__ n) {
  extern __shared__ float2 s_tab[];
  __shared__ __align__(16) float s_y[kTileB][kTileP + 4];
  __shared__ __align__(16) float s_f[kTileB][kCols];
  __shared__ uint32_t s_n[kTileP];
  for (uint32_t i = threadIdx.x; i < entries; i += blockDim.x) s_tab[i] = table[i];
  if (threadIdx.x < kTileP) s_n[threadIdx.x] = 0u;
  __syncthreads();
  const bool tl = two_level != 0;
  const float invT = 1.0f / float(T);
  const uint32_t tx = threadIdx.x & 15u, ty = threadIdx.x >> 4;
  const uint32_t p0 = blockIdx.x * kTileP;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  const uint32_t lb = threadIdx.x & 63u, lp = threadIdx.x >> 6;  // loader: bin, pixel phase
  for (uint32_t b0 = 0; b0 < T; b0 += kTileB) {
    // Y chunk: consecutive threads read consecutive bins of one pixel.
#pragma unroll 4
    for (uint32_t pp = lp; pp < kTileP; pp += 4) {
      const uint32_t p = p0 + pp, b = b0 + lb;
      uint32_t y = 0;
      if (p < P && b < T) y = hist[size_t(p) * T + b];
      s_y[lb][pp] = float(y);
    }
    // F chunk: 64 bins x 2m columns (zero beyond 2m).
    for (uint32_t i = threadIdx.x; i < kTileB * (kCols / 2); i += blockDim.x) {
      const uint32_t bb = i / (kCols / 2), l = i - bb * (kCols / 2);
      const uint32_t b = b0 + bb;
      float2 e = make_float2(0.f, 0.f);
      if (l < m && b < T) e = phase(s_tab, mulmod(l + 1u, b, T, invT), tl);
      s_f[bb][2 * l] = e.x;
      s_f[bb][2 * l + 1] = e.y;
    }
    __syncthreads();
    float part[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) part[i][j] = 0.f;
#pragma unroll 8
    for (int k = 0; k < kTileB; ++k) {
      const float4 yv = *reinterpret_cast<const float4*>(&s_y[k][4 * ty]);
      const float4 fv = *reinterpret_cast<const float4*>(&s_f[k][4 * tx]);
      const float ya[4] = {yv.x, yv.y, yv.z, yv.w};
      const float fa[4] = {fv.x, fv.y, fv.z, fv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) part[i][j] = fmaf(ya[i], fa[j], part[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += part[i][j];
    __syncthreads();
  }
  // n[p] = sum_b y[p][b], exact in integers (one warp per pixel row).
  for (uint32_t pp = threadIdx.x >> 5; pp < kTileP; pp += blockDim.x >> 5) {
    const uint32_t p = p0 + pp;
    uint32_t c = 0;
    if (p < P)
      for (uint32_t b = threadIdx.x & 31u; b < T; b += 32u) c += hist[size_t(p) * T + b];
    for (int off = 16; off; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31u) == 0) s_n[pp] = c;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t p = p0 + 4 * ty + i;
    if (p >= P) continue;
#pragma unroll
    for (int j = 0; j < 4; j += 2) {
      const uint32_t l = (4 * tx + j) / 2;
      if (l < m) S[size_t(p) * m + l] = make_float2(acc[i][j], acc[i][j + 1]);
    }
  }
  if (threadIdx.x < kTileP && p0 + threadIdx.x < P) n[p0 + threadIdx.x] = s_n[threadIdx.x];
}

}  // namespace

srt3d_status launch_sketch_hist_fp32(srt3d_ctx* ctx, const uint16_t* hist, uint32_t P, uint32_t T, uint32_t m,
                                     float2* S, uint32_t* n, cudaStream_t stream) {
  PhaseTable tab;
  srt3d_status st = get_phase_table(ctx, T, &tab);
  if (st != SRT3D_OK) return st;
  const size_t smem = size_t(tab.entries) * sizeof(float2);
  if (smem + sizeof(float) * (kTileB * (kTileP + 4) + kTileB * kCols) + 4 * kTileP > 48 * 1024)
    SRT3D_CUDA_TRY(ctx, cudaFuncSetAttribute(k_sketch_hist_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smem)));
  const uint32_t grid = (P + kTileP - 1) / kTileP;
  const ProfMark mk = prof_begin(ctx, KID_SKETCH_HIST_FP32, stream);
  k_sketch_hist_fp32<<<grid, 256, smem, stream>>>(hist, P, T, m, tab.dev, tab.entries, tab.two_level ? 1 : 0, S,
                                                  n);
  prof_end(ctx, KID_SKETCH_HIST_FP32, mk, stream);
  SRT3D_CUDA_TRY(ctx, cudaGetLastError());
  return SRT3D_OK;
}

}  // namespace srt3d

using namespace srt3d;

extern "C" srt3d_status srt3d_sketch_hist(srt3d_ctx* ctx, const uint16_t* hist, uint32_t num_pixels, uint32_t T,
                                          uint32_t m, int precision, float* S, uint32_t* n, void* stream) {
  if (!ctx) return SRT3D_EINVAL;
  if (!hist || !S || !n) return set_error(ctx, SRT3D_EINVAL, "NULL pointer");
  if (T < 1 || T > 65536) return set_error(ctx, SRT3D_EINVAL, "T must be in [1, 65536]");
  if (m < 1 || m > 32) return set_error(ctx, SRT3D_EINVAL, "m must be in [1, 32]");
  if (reinterpret_cast<uintptr_t>(S) % 8) return set_error(ctx, SRT3D_EINVAL, "S must be 8-byte aligned");
  if (num_pixels == 0) return SRT3D_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == SRT3D_FP32)
    return launch_sketch_hist_fp32(ctx, hist, num_pixels, T, m, reinterpret_cast<float2*>(S), n, s);
  if (precision == SRT3D_FP16_SPLIT || precision == SRT3D_BF16) {
    if (T % 64 != 0) return set_error(ctx, SRT3D_EINVAL, "tensor-core precisions need T % 64 == 0");
    if (num_pixels >= (1u << 31)) return set_error(ctx, SRT3D_EINVAL, "tensor-core precisions need num_pixels < 2^31");
    if (reinterpret_cast<uintptr_t>(hist) % 16) return set_error(ctx, SRT3D_EINVAL, "hist must be 16-byte aligned");
    return launch_sketch_hist_tc(ctx, hist, num_pixels, T, m, precision, reinterpret_cast<float2*>(S), n, s);
  }
  return set_error(ctx, SRT3D_EINVAL, "unknown precision");
}

// Stream sketch through a device histogram and the tensor cores: the photons
// of every pixel are binned (Sec. 2, Eq. 2, one bin per stamp value), and the
// histogram sketch Y F (Eq. 3) is taken on the tensor cores. The cost depends
// on P x T and hardly on m or on the photons per pixel, so it beats the
// per-photon stream kernel at large m or dense pixels.
extern "C" srt3d_status srt3d_sketch_stream_tc(srt3d_ctx* ctx, const uint16_t* stamps, const uint32_t* offsets,
                                               uint64_t num_stamps, uint32_t num_pixels, uint32_t T, uint32_t m,
                                               int precision, float* S, uint32_t* n, void* stream) {
  if (!ctx) return SRT3D_EINVAL;
  if (!offsets || !S || !n || (num_stamps && !stamps)) return set_error(ctx, SRT3D_EINVAL, "NULL pointer");
  if (T < 64 || T > 65536 || T % 64 != 0) return set_error(ctx, SRT3D_EINVAL, "T must be a multiple of 64 in [64, 65536]");
  if (m < 1 || m > 32) return set_error(ctx, SRT3D_EINVAL, "m must be in [1, 32]");
  if (precision != SRT3D_FP16_SPLIT && precision != SRT3D_BF16)
    return set_error(ctx, SRT3D_EINVAL, "precision must be SRT3D_FP16_SPLIT or SRT3D_BF16");
  if (num_stamps >= (1ull << 32)) return set_error(ctx, SRT3D_EINVAL, "num_stamps must be < 2^32");
  if (num_pixels >= (1u << 31)) return set_error(ctx, SRT3D_EINVAL, "num_pixels must be < 2^31");
  if (reinterpret_cast<uintptr_t>(S) % 8) return set_error(ctx, SRT3D_EINVAL, "S must be 8-byte aligned");
  if (num_pixels == 0) return SRT3D_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = size_t(num_pixels) * T * sizeof(uint16_t);
  srt3d_status st;
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    st = grow(ctx, &ctx->hist_scratch, bytes);
  }
  if (st != SRT3D_OK) return st;
  uint16_t* hist = static_cast<uint16_t*>(ctx->hist_scratch.ptr);
  st = launch_hist_from_stream(ctx, stamps, offsets, num_stamps, num_pixels, T, hist, s);
  if (st != SRT3D_OK) return st;
  return launch_sketch_hist_tc(ctx, hist, num_pixels, T, m, precision, reinterpret_cast<float2*>(S), n, s);
}

// The same stream sketch with the histogram built in shared memory, one
// tensor-core stage (64 bins of 128 pixels) at a time, from the stamps
// counting-sorted by stage (k_bucket_stream). Only the stamps and their 2-byte
// sorted entries cross HBM, not the num_pixels x T histogram.
extern "C" srt3d_status srt3d_sketch_stream_tc_fused(srt3d_ctx* ctx, const uint16_t* stamps,
                                                     const uint32_t* offsets, uint64_t num_stamps,
                                                     uint32_t num_pixels, uint32_t T, uint32_t m, int precision,
                                                     float* S, uint32_t* n, void* stream) {
  if (!ctx) return SRT3D_EINVAL;
  if (!offsets || !S || !n || (num_stamps && !stamps)) return set_error(ctx, SRT3D_EINVAL, "NULL pointer");
  if (T < 64 || T > 65536 || T % 64 != 0) return set_error(ctx, SRT3D_EINVAL, "T must be a multiple of 64 in [64, 65536]");
  if (m < 1 || m > 32) return set_error(ctx, SRT3D_EINVAL, "m must be in [1, 32]");
  if (precision != SRT3D_FP16_SPLIT && precision != SRT3D_BF16)
    return set_error(ctx, SRT3D_EINVAL, "precision must be SRT3D_FP16_SPLIT or SRT3D_BF16");
  if (num_stamps >= (1ull << 32)) return set_error(ctx, SRT3D_EINVAL, "num_stamps must be < 2^32");
  if (num_pixels >= (1u << 31)) return set_error(ctx, SRT3D_EINVAL, "num_pixels must be < 2^31");
  if (reinterpret_cast<uintptr_t>(S) % 8) return set_error(ctx, SRT3D_EINVAL, "S must be 8-byte aligned");
  if (num_pixels == 0) return SRT3D_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  srt3d_status st;
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    st = grow(ctx, &ctx->hist_scratch, stream_tc_fused_scratch_bytes(num_stamps, num_pixels, T));
  }
  if (st != SRT3D_OK) return st;
  return launch_sketch_stream_tc_fused(ctx, stamps, offsets, num_stamps, num_pixels, T, m, precision,
                                       reinterpret_cast<float2*>(S), n, ctx->hist_scratch.ptr, s);
}
