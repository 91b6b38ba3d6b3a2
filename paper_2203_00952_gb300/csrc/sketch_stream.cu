// Stream-path kernels (Sec. 2):
//   k_sketch_stream   S[p][l-1] = sum_x exp(i 2 pi ((l x) mod T) / T)   (Eq. 3)
//   k_hist_from_stream  y[p][b] = #{x = b}                               (Eq. 2)
//   k_finalize        z = S / n                                          (Eq. 3)
//
// Sketch kernel layout: a group of G lanes (G in {4, 8, 16, 32}) owns one
// pixel at a time; its lanes read the pixel's stamps as 16-byte words
// (8 stamps) from an aligned base, so loads are coalesced whatever the
// pixel's offset. Per photon the exact integer phase x (and (l x) mod T at
// every 16th harmonic) indexes a shared-memory cos/sin table; the harmonics
// in between are obtained by complex rotation e_l = e_{l-1} e_1, so the
// rounding error stays below ~16 (2^-23) per term. Each lane keeps m complex
// FP32 partial sums; the group reduces them with xor shuffles at the end of
// the pixel. No floating-point atomics: the result for a pixel does not
// depend on what else runs.
#include <cmath>
#include <cstdio>

#include "device_util.cuh"
#include "internal.h"

namespace srt3d {
namespace {

constexpr int kBlock = 256;
constexpr int kResync = 16;  // table lookup every kResync harmonics

template <int M>
__device__ __forceinline__ void add_photon(float2 (&acc)[M], uint32_t x, const float2* tab, bool two_level,
                                           uint32_t T, float invT) {
  const float2 e1 = phase(tab, x, two_level);
  float2 e = e1;
  acc[0].x += e.x;
  acc[0].y += e.y;
#pragma unroll
  for (int j = 2; j <= M; ++j) {
    if ((j - 1) % kResync == 0)
      e = phase(tab, mulmod(uint32_t(j), x, T, invT), two_level);
    else
      e = cmul(e, e1);
    acc[j - 1].x += e.x;
    acc[j - 1].y += e.y;
  }
}

__device__ __forceinline__ uint4 ld_stream(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// One pixel of the stream, processed by a group of G lanes: coalesced 16-byte
// words from the aligned base, per-lane partial sums, xor-shuffle reduction,
// store (or accumulate) of S[p][0..m) and n[p].
template <int M>
__device__ __forceinline__ void sketch_pixel(const uint4* __restrict__ words, uint32_t shift,
                                             const uint32_t* __restrict__ offsets, uint32_t num_stamps, uint32_t p,
                                             uint32_t T, float invT, uint32_t m, uint32_t G, uint32_t gl,
                                             unsigned gmask, int accumulate, const float2* s_tab, bool tl,
                                             float2* __restrict__ S, uint32_t* __restrict__ n,
                                             uint32_t* __restrict__ flags) {
  uint32_t s = __ldg(offsets + p), e = __ldg(offsets + p + 1);
  if (e < s || e > num_stamps) {
    if (gl == 0) atomicOr(flags, FLAG_OFFSETS);
    s = e = 0;
  }
  float2 acc[M];
#pragma unroll
  for (int j = 0; j < M; ++j) acc[j] = make_float2(0.f, 0.f);
  const uint32_t a = s + shift, b = e + shift;
  bool bad = false;
  for (uint32_t w = (a >> 3) + gl; w < ((b + 7u) >> 3); w += G) {
    const uint4 v = ld_stream(words + w);
    const uint32_t x[8] = {v.x & 0xffffu, v.x >> 16, v.y & 0xffffu, v.y >> 16,
                           v.z & 0xffffu, v.z >> 16, v.w & 0xffffu, v.w >> 16};
    const uint32_t base = w << 3;
    uint32_t mx = max(max(max(x[0], x[1]), max(x[2], x[3])), max(max(x[4], x[5]), max(x[6], x[7])));
    if (base >= a && base + 8u <= b && mx < T) {
#pragma unroll
      for (int i = 0; i < 8; ++i) add_photon<M>(acc, x[i], s_tab, tl, T, invT);
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const uint32_t idx = base + uint32_t(i);
        if (idx >= a && idx < b) {
          if (x[i] < T)
            add_photon<M>(acc, x[i], s_tab, tl, T, invT);
          else
            bad = true;
        }
      }
    }
  }
  if (bad) atomicOr(flags, FLAG_STAMP_RANGE);
#pragma unroll
  for (int j = 0; j < M; ++j) {
    for (uint32_t off = G >> 1; off > 0; off >>= 1) {
      acc[j].x += __shfl_xor_sync(gmask, acc[j].x, off);
      acc[j].y += __shfl_xor_sync(gmask, acc[j].y, off);
    }
  }
  float2* Sp = S + size_t(p) * m;
#pragma unroll
  for (int j = 0; j < M; ++j) {
    if (uint32_t(j) < m && (uint32_t(j) & (G - 1u)) == gl) {
      float2 v = acc[j];
      if (accumulate) {
        const float2 o = Sp[j];
        v.x += o.x;
        v.y += o.y;
      }
      Sp[j] = v;
    }
  }
  if (gl == 0) n[p] = (accumulate ? n[p] : 0u) + (e - s);
}

template <int M>
__global__ void __launch_bounds__(kBlock) k_sketch_stream(
    const uint16_t* __restrict__ stamps, const uint32_t* __restrict__ offsets, uint32_t num_stamps,
    uint32_t P, uint32_t T, uint32_t m, int glog2, int accumulate, const float2* __restrict__ table,
    uint32_t tab_entries, int two_level, float2* __restrict__ S, uint32_t* __restrict__ n,
    uint32_t* __restrict__ flags) {
  extern __shared__ float2 s_tab[];
  for (uint32_t i = threadIdx.x; i < tab_entries; i += blockDim.x) s_tab[i] = table[i];
  __syncthreads();
  const bool tl = two_level != 0;
  const float invT = 1.0f / float(T);
  const uint32_t G = 1u << glog2;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t gl = lane & (G - 1u);
  const unsigned gmask = (G == 32u) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1u)));
  const uint32_t gid = (blockIdx.x * blockDim.x + threadIdx.x) >> glog2;
  const uint32_t ngroups = (gridDim.x * blockDim.x) >> glog2;
  const uintptr_t addr = reinterpret_cast<uintptr_t>(stamps);
  const uint4* words = reinterpret_cast<const uint4*>(addr & ~uintptr_t(15));
  const uint32_t shift = uint32_t(addr & 15u) >> 1;
  for (uint32_t p = gid; p < P; p += ngroups)
    sketch_pixel<M>(words, shift, offsets, num_stamps, p, T, invT, m, G, gl, gmask, accumulate, s_tab, tl, S, n,
                    flags);
}

// Batched sketch of several frames in one persistent launch: the work list
// holds (frame, first pixel, last pixel) items of roughly equal photon
// counts; a CTA walks items blockIdx.x, blockIdx.x + gridDim.x, ..., reloading
// the phase table when the frame changes. Lanes per pixel come from the
// frame's descriptor (autotuned per photon-density class).
template <int M>
__global__ void __launch_bounds__(kBlock) k_sketch_batch(const BatchFrame* __restrict__ frames,
                                                         const uint3* __restrict__ items, uint32_t num_items,
                                                         uint32_t* __restrict__ flags) {
  extern __shared__ float2 s_tab[];
  uint32_t cur = 0xffffffffu;
  for (uint32_t it = blockIdx.x; it < num_items; it += gridDim.x) {
    const uint3 item = items[it];
    const BatchFrame& f = frames[item.x];
    if (item.x != cur) {
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < f.tab_entries; i += blockDim.x) s_tab[i] = f.table[i];
      __syncthreads();
      cur = item.x;
    }
    const bool tl = f.two_level != 0;
    const float invT = 1.0f / float(f.T);
    const uint32_t G = 1u << f.glog2;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t gl = lane & (G - 1u);
    const unsigned gmask = (G == 32u) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1u)));
    const uint32_t gid = threadIdx.x >> f.glog2;
    const uint32_t ngroups = blockDim.x >> f.glog2;
    const uintptr_t addr = reinterpret_cast<uintptr_t>(f.stamps);
    const uint4* words = reinterpret_cast<const uint4*>(addr & ~uintptr_t(15));
    const uint32_t shift = uint32_t(addr & 15u) >> 1;
    for (uint32_t p = item.y + gid; p < item.z; p += ngroups)
      sketch_pixel<M>(words, shift, f.offsets, f.num_stamps, p, f.T, invT, f.m, G, gl, gmask, 0, s_tab, tl, f.S,
                      f.n, flags);
  }
}

// Harmonic counts with their own instantiation; other m use the next one up.
constexpr int kInstM[] = {1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 20, 24, 28, 32};

using SketchFn = void (*)(const uint16_t*, const uint32_t*, uint32_t, uint32_t, uint32_t, uint32_t, int,
                          int, const float2*, uint32_t, int, float2*, uint32_t*, uint32_t*);

SketchFn sketch_fn(int M) {
  switch (M) {
#define CASE(k) \
  case k: return &k_sketch_stream<k>;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10)
    CASE(11) CASE(12) CASE(13) CASE(14) CASE(15) CASE(16) CASE(20) CASE(24) CASE(28) CASE(32)
#undef CASE
    default: return nullptr;
  }
}

using BatchFn = void (*)(const BatchFrame*, const uint3*, uint32_t, uint32_t*);

BatchFn batch_fn(int M) {
  switch (M) {
#define CASE(k) \
  case k: return &k_sketch_batch<k>;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10)
    CASE(11) CASE(12) CASE(13) CASE(14) CASE(15) CASE(16) CASE(20) CASE(24) CASE(28) CASE(32)
#undef CASE
    default: return nullptr;
  }
}

}  // namespace

int sketch_round_m(uint32_t m) {
  for (int k : kInstM)
    if (uint32_t(k) >= m) return k;
  return -1;
}

namespace {

__global__ void k_finalize(const float2* __restrict__ S, const uint32_t* __restrict__ n, uint32_t P, uint32_t m,
                           float2* __restrict__ z) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= size_t(P) * m) return;
  const uint32_t cnt = __ldg(n + i / m);
  const float2 s = S[i];
  const float nf = float(cnt);
  z[i] = cnt ? make_float2(s.x / nf, s.y / nf) : make_float2(0.f, 0.f);
}

// z = S / n for every frame of a batch (blockIdx.y = frame).
__global__ void k_finalize_batch(const BatchFrame* __restrict__ frames) {
  const BatchFrame& f = frames[blockIdx.y];
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= size_t(f.P) * f.m) return;
  const uint32_t cnt = f.n[i / f.m];
  const float2 s = f.S[i];
  const float nf = float(cnt);
  f.S[i] = cnt ? make_float2(s.x / nf, s.y / nf) : make_float2(0.f, 0.f);
}

// One CTA per pixel at a time; u32 counters in shared memory over a window of
// at most kHistWindow bins (the pixel's stamps are re-scanned per window).
constexpr uint32_t kHistWindow = 16384;

__global__ void __launch_bounds__(kBlock) k_hist_from_stream(const uint16_t* __restrict__ stamps,
                                                             const uint32_t* __restrict__ offsets,
                                                             uint32_t num_stamps, uint32_t P, uint32_t T,
                                                             uint16_t* __restrict__ hist,
                                                             uint32_t* __restrict__ flags) {
  extern __shared__ uint32_t s_cnt[];
  for (uint32_t p = blockIdx.x; p < P; p += gridDim.x) {
    uint32_t s = __ldg(offsets + p), e = __ldg(offsets + p + 1);
    if (e < s || e > num_stamps) {
      if (threadIdx.x == 0) atomicOr(flags, FLAG_OFFSETS);
      s = e = 0;
    }
    for (uint32_t b0 = 0; b0 < T; b0 += kHistWindow) {
      const uint32_t nb = min(kHistWindow, T - b0);
      for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) s_cnt[i] = 0u;
      __syncthreads();
      bool bad = false;
      for (uint32_t i = s + threadIdx.x; i < e; i += blockDim.x) {
        const uint32_t x = __ldg(stamps + i);
        if (x >= T)
          bad = true;
        else if (x - b0 < nb)
          atomicAdd(&s_cnt[x - b0], 1u);
      }
      if (bad && b0 == 0) atomicOr(flags, FLAG_STAMP_RANGE);
      __syncthreads();
      uint16_t* row = hist + size_t(p) * T + b0;
      bool over = false;
      for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) {
        uint32_t c = s_cnt[i];
        if (c > 65535u) {
          over = true;
          c = 65535u;
        }
        row[i] = uint16_t(c);
      }
      if (over) atomicOr(flags, FLAG_COUNT_RANGE);
      __syncthreads();
    }
  }
}

}  // namespace

int sketch_default_glog2(double mean) {
  return mean >= 192.0 ? 5 : mean >= 96.0 ? 4 : mean >= 32.0 ? 3 : 2;
}

srt3d_status launch_sketch_stream_g(srt3d_ctx* ctx, const uint16_t* stamps, const uint32_t* offsets,
                                    uint64_t num_stamps, uint32_t P, uint32_t T, uint32_t m, int accumulate,
                                    float2* S, uint32_t* n, cudaStream_t stream, uint32_t* flags, int glog2) {
  PhaseTable tab;
  srt3d_status st = get_phase_table(ctx, T, &tab);
  if (st != SRT3D_OK) return st;
  const int M = sketch_round_m(m);
  SketchFn fn = sketch_fn(M);
  if (!fn) return set_error(ctx, SRT3D_EINVAL, "unsupported m");
  if (glog2 < 0) {
    // lanes per pixel: the autotuned value for this density class if there is
    // one, else a whole warp for dense pixels and narrower groups for sparse ones
    const double mean = P ? double(num_stamps) / double(P) : 0.0;
    glog2 = sketch_default_glog2(mean);
    std::lock_guard<std::mutex> lock(ctx->mu);
    const int bucket = mean < 1.0 ? 0 : int(std::log2(mean));
    auto it = ctx->tuned.find((uint64_t(M) << 40) | (uint64_t(tab.two_level) << 32) | uint64_t(bucket));
    if (it != ctx->tuned.end()) glog2 = it->second;
  }
  const size_t smem = size_t(tab.entries) * sizeof(float2);
  if (smem > 48 * 1024)
    SRT3D_CUDA_TRY(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  int bps = 0;
  SRT3D_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kBlock, smem));
  if (bps < 1) bps = 1;
  const uint64_t groups_per_block = kBlock >> glog2;
  const uint64_t need = (uint64_t(P) + groups_per_block - 1) / groups_per_block;
  const uint64_t grid = std::min<uint64_t>(need, uint64_t(ctx->num_sms) * bps);
  const ProfMark mk = prof_begin(ctx, KID_SKETCH_STREAM, stream);
  fn<<<dim3(uint32_t(grid)), dim3(kBlock), smem, stream>>>(stamps, offsets, uint32_t(num_stamps), P, T, m, glog2,
                                                          accumulate, tab.dev, tab.entries, tab.two_level ? 1 : 0,
                                                          S, n, flags ? flags : ctx->d_flags);
  prof_end(ctx, KID_SKETCH_STREAM, mk, stream);
  SRT3D_CUDA_TRY(ctx, cudaGetLastError());
  return SRT3D_OK;
}

srt3d_status launch_sketch_stream(srt3d_ctx* ctx, const uint16_t* stamps, const uint32_t* offsets,
                                  uint64_t num_stamps, uint32_t P, uint32_t T, uint32_t m, int accumulate,
                                  float2* S, uint32_t* n, cudaStream_t stream, uint32_t* flags) {
  return launch_sketch_stream_g(ctx, stamps, offsets, num_stamps, P, T, m, accumulate, S, n, stream, flags, -1);
}

srt3d_status launch_sketch_batch(srt3d_ctx* ctx, const BatchFrame* d_frames, const uint3* d_items,
                                 uint32_t num_items, int M, uint32_t max_tab_entries, cudaStream_t stream) {
  BatchFn fn = batch_fn(M);
  if (!fn) return set_error(ctx, SRT3D_EINVAL, "unsupported m");
  const size_t smem = size_t(max_tab_entries) * sizeof(float2);
  if (smem > 48 * 1024)
    SRT3D_CUDA_TRY(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  int bps = 0;
  SRT3D_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kBlock, smem));
  if (bps < 1) bps = 1;
  const uint32_t grid = std::min<uint32_t>(num_items, uint32_t(ctx->num_sms) * uint32_t(bps));
  const ProfMark mk = prof_begin(ctx, KID_SKETCH_STREAM, stream);
  fn<<<grid, kBlock, smem, stream>>>(d_frames, d_items, num_items, ctx->d_flags);
  prof_end(ctx, KID_SKETCH_STREAM, mk, stream);
  SRT3D_CUDA_TRY(ctx, cudaGetLastError());
  return SRT3D_OK;
}

srt3d_status launch_finalize(srt3d_ctx* ctx, const float2* S, const uint32_t* n, uint32_t P, uint32_t m,
                             float2* z, cudaStream_t stream) {
  const size_t total = size_t(P) * m;
  const uint32_t grid = uint32_t((total + kBlock - 1) / kBlock);
  const ProfMark mk = prof_begin(ctx, KID_FINALIZE, stream);
  k_finalize<<<grid, kBlock, 0, stream>>>(S, n, P, m, z);
  prof_end(ctx, KID_FINALIZE, mk, stream);
  SRT3D_CUDA_TRY(ctx, cudaGetLastError());
  return SRT3D_OK;
}

srt3d_status launch_finalize_batch(srt3d_ctx* ctx, const BatchFrame* d_frames, uint32_t nframes, uint32_t max_pm,
                                   cudaStream_t stream) {
  const dim3 grid((max_pm + kBlock - 1) / kBlock, nframes);
  const ProfMark mk = prof_begin(ctx, KID_FINALIZE, stream);
  k_finalize_batch<<<grid, kBlock, 0, stream>>>(d_frames);
  prof_end(ctx, KID_FINALIZE, mk, stream);
  SRT3D_CUDA_TRY(ctx, cudaGetLastError());
  return SRT3D_OK;
}

srt3d_status launch_hist_from_stream(srt3d_ctx* ctx, const uint16_t* stamps, const uint32_t* offsets,
                                     uint64_t num_stamps, uint32_t P, uint32_t T, uint16_t* hist,
                                     cudaStream_t stream) {
  const size_t smem = size_t(std::min(T, kHistWindow)) * sizeof(uint32_t);
  int bps = 0;
  SRT3D_CUDA_TRY(ctx, cudaFuncSetAttribute(k_hist_from_stream, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           int(kHistWindow * sizeof(uint32_t))));
  SRT3D_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_hist_from_stream, kBlock, smem));
  if (bps < 1) bps = 1;
  const uint32_t grid = uint32_t(std::min<uint64_t>(P, uint64_t(ctx->num_sms) * bps));
  const ProfMark mk = prof_begin(ctx, KID_HIST_FROM_STREAM, stream);
  k_hist_from_stream<<<grid, kBlock, smem, stream>>>(stamps, offsets, uint32_t(num_stamps), P, T, hist,
                                                     ctx->d_flags);
  prof_end(ctx, KID_HIST_FROM_STREAM, mk, stream);
  SRT3D_CUDA_TRY(ctx, cudaGetLastError());
  return SRT3D_OK;
}

}  // namespace srt3d
