// Histogram sketch on the tcgen05 tensor cores (Sec. 2, Eqs. 2-3):
//   Z[P x N] = Y[P x T] F^T[N x T]^T, F^T[2(l-1)][b] = cos(2 pi ((l b) mod T) / T),
//   F^T[2(l-1)+1][b] = sin(...), N = 2m rounded up to 16 (x2 for the split).
//
// Persistent, warp-specialised CTA (512 threads, one per SM), M = 128 pixels
// per tile, K = 64 bins per pipeline stage, as many stages (up to 8) as fit in
// shared memory next to one shared A2 slot:
//   warp 0      TMA producer: Y tile [128 x 64] u16 and F^T tile [N x 64],
//               both 128-byte swizzled (the canonical K-major operand layout)
//   warps 4-11  converters: two threads per pixel row convert the stage in
//               place to FP16 (exact for counts <= 2048; larger counts are
//               split exactly into (y & ~31) in A and (y & 31) in the A2
//               slot, shared by all stages) or to BF16; they also count the
//               row's photons (n) in integers
//   warp 1      MMA issuer: tcgen05.mma.kind::f16 into a double-buffered FP32
//               accumulator in TMEM; A2 only for stages that hold a count > 2048
//               (a converter writes the A2 slot only after the MMAs of the
//               previous stage have completed, so big counts serialise the
//               pipeline while they last and cost nothing otherwise)
//   warps 12-15 epilogue: tcgen05.ld of the accumulator, hi + lo, store S
// SRT3D_FP16_SPLIT uses F = F_hi + F_lo (both FP16, stacked along N, one MMA
// computes both products); SRT3D_BF16 uses a single BF16 F and BF16 counts.
// Every mbarrier wait is bounded: on timeout the kernel latches an error flag,
// lets every role leave its loop, waits (bounded) for its own TMA copies and
// MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>

#include "internal.h"

namespace srt3d {

namespace {

constexpr int kThreads = 512;
constexpr int kTileM = 128;
constexpr int kTileK = 64;  // bins per stage: 64 x 2 B = one 128-byte swizzle row
constexpr uint32_t kABytes = kTileM * kTileK * 2;
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at 2 GHz

// ------------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(bar),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false when the wait gave up (here or in another role).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          uint32_t* gflags) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      atomicOr(gflags, FLAG_DEVICE_TIMEOUT);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"(map), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (FP16 or BF16 inputs, FP32 accumulator).
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive on `bar` once every tcgen05 operation issued so far by this thread completes.
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3FFFFu) >> 4);  // start address
  d |= uint64_t(1) << 16;                  // leading byte offset (unused for this layout)
  d |= uint64_t(1024 >> 4) << 32;          // stride byte offset
  d |= uint64_t(1) << 46;                  // version
  d |= uint64_t(2) << 61;                  // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, A/B format (0 FP16,
// 1 BF16), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t M, uint32_t N, uint32_t ab_fmt) {
  return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

constexpr int kMaxStages = 8;

template <int PREC>
struct TcCfg {
  static constexpr bool kSplit = (PREC == SRT3D_FP16_SPLIT);
};

// ------------------------------------------------------------------ the kernel

template <int PREC>
__global__ void __launch_bounds__(kThreads, 1)
    k_sketch_hist_tc(const __grid_constant__ CUtensorMap mapY, const __grid_constant__ CUtensorMap mapF,
                     uint32_t P, uint32_t T, uint32_t m, uint32_t N2, uint32_t ncols_alloc, uint32_t ST,
                     float2* __restrict__ S, uint32_t* __restrict__ n, uint32_t* __restrict__ gflags) {
  using Cfg = TcCfg<PREC>;
  constexpr bool kSplit = Cfg::kSplit;
  const uint32_t N = kSplit ? 2u * N2 : N2;  // MMA N (rows of F^T per stage)
  const uint32_t b_bytes = N * 128u;
  const uint32_t stage_bytes = kABytes + b_bytes;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* a2_slot = base + ST * stage_bytes;  // FP16 split only
  uint64_t* bars = reinterpret_cast<uint64_t*>(a2_slot + (kSplit ? kABytes : 0u));
  // barrier slots: full[8], conv[8], empty[8], tfull[2], tempty[2], drain
  uint64_t* full = bars;
  uint64_t* conv = bars + kMaxStages;
  uint64_t* empty = bars + 2 * kMaxStages;
  uint64_t* tfull = bars + 3 * kMaxStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  uint32_t* split_gen = tmem_slot + 1;  // [8]
  volatile int* abort_flag = reinterpret_cast<volatile int*>(split_gen + kMaxStages);

  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint32_t ntiles = (P + kTileM - 1) / kTileM;
  const uint32_t KT = T / kTileK;

  auto sA = [&](uint32_t s) { return base + s * stage_bytes; };
  auto sB = [&](uint32_t s) { return base + s * stage_bytes + kABytes; };

  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < ST; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&conv[s]), 256);
      mbar_init(smem_u32(&empty[s]), 1);
      split_gen[s] = 0xffffffffu;
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&tfull[a]), 1);
      mbar_init(smem_u32(&tempty[a]), 128);
    }
    mbar_init(smem_u32(drain), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&mapY) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&mapF) : "memory");
  }
  if (warp == 2) {
    tmem_alloc(smem_u32(tmem_slot), ncols_alloc);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      uint32_t it = 0, s = 0, ph = 0;
      for (uint32_t tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
        for (uint32_t kt = 0; kt < KT; ++kt, ++it) {
          if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1u, abort_flag, gflags)) break;
          mbar_arrive_expect_tx(smem_u32(&full[s]), kABytes + b_bytes);
          tma_load_2d(smem_u32(sA(s)), &mapY, smem_u32(&full[s]), int(kt * kTileK), int(tile * kTileM));
          tma_load_2d(smem_u32(sB(s)), &mapF, smem_u32(&full[s]), int(kt * kTileK), 0);
          if (++s == ST) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
      // no copy may be in flight when the CTA leaves: wait for the last stages issued
      const uint32_t first = it > ST ? it - ST : 0u;
      for (uint32_t j = first; j < it; ++j) {
        const uint32_t s = j % ST, ph = (j / ST) & 1u;
        const long long t0 = clock64();
        while (!mbar_try_wait(smem_u32(&full[s]), ph) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = make_idesc(kTileM, N, PREC == SRT3D_BF16 ? 1u : 0u);
      const uint32_t acc_cols = ncols_alloc / 2;
      uint32_t it = 0, lt = 0, s = 0, ph = 0;
      bool ok = true;
      for (uint32_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++lt) {
        const uint32_t acc = lt & 1u, aph = (lt >> 1) & 1u;
        if (!(ok = mbar_wait(smem_u32(&tempty[acc]), aph ^ 1u, abort_flag, gflags))) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * acc_cols;
        for (uint32_t kt = 0; kt < KT; ++kt, ++it) {
          if (!(ok = mbar_wait(smem_u32(&conv[s]), ph, abort_flag, gflags))) break;
          tc_fence_after();
          const bool split = kSplit && split_gen[s] == it;
          const uint64_t da = sw128_desc(smem_u32(sA(s)));
          const uint64_t da2 = sw128_desc(smem_u32(a2_slot));
          const uint64_t db = sw128_desc(smem_u32(sB(s)));
#pragma unroll
          for (uint32_t k = 0; k < kTileK / 16; ++k) {
            // advance 16 elements (32 bytes) along K inside the swizzled row
            umma_f16(d_tmem, da + 2 * k, db + 2 * k, idesc, (kt | k) != 0u ? 1u : 0u);
            if (split) umma_f16(d_tmem, da2 + 2 * k, db + 2 * k, idesc, 1u);
          }
          umma_commit(smem_u32(&empty[s]));
          if (++s == ST) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (!ok) break;
        umma_commit(smem_u32(&tfull[acc]));
      }
      // every MMA issued must be complete before TMEM is released
      umma_commit(smem_u32(drain));
      const long long t0 = clock64();
      while (!mbar_try_wait(smem_u32(drain), 0u) && clock64() - t0 < kWaitCycles) {
      }
    }
  } else if (warp >= 4 && warp < 12) {
    // ---------------------------------------------------------------- converters
    // 256 threads: thread (half, row) owns four 16-byte chunks of one pixel
    // row (128 bytes) of every stage. Chunks are visited in swizzled order
    // (c ^ (row & 7)) so the 32 rows of a warp cover all banks; the conversion
    // is elementwise, so the order does not matter. Small counts take an exact
    // bit-pattern path (FP16: (0x6400 | y) - 1024 for y < 1024; BF16:
    // (0x4300 | y) - 128 for y < 128); others take the rounding conversion.
    // The A2 slot (FP16 split) starts zeroed; a thread rewrites its A2 chunks
    // only while they hold, or last held, a count above 2048, and only after
    // the previous stage's MMAs, the last that may have read the slot, have
    // completed (the empty barrier of that stage's slot).
    const uint32_t ct = threadIdx.x - 128u;
    const uint32_t row = ct & 127u, c0 = (ct >> 7) * 4u;
    const uint32_t sw = row & 7u;
    bool dirty = false;  // this thread's A2 chunks are nonzero
    if (kSplit) {
      uint8_t* ra2 = a2_slot + row * 128u;
#pragma unroll
      for (uint32_t c = 0; c < 4; ++c)
        *reinterpret_cast<uint4*>(ra2 + (((c0 + c) ^ sw) << 4)) = make_uint4(0u, 0u, 0u, 0u);
      fence_proxy_async_smem();
    }
    // a halfword exceeds the bit-pattern limit (1023 FP16, 127 BF16) iff one
    // of its bits above the limit is set: test the OR of the stage's words
    constexpr uint32_t kOverMask = kSplit ? 0xFC00FC00u : 0xFF80FF80u;
    uint32_t it = 0, s = 0, ph = 0;
    uint32_t ps = 0, pph = 0;  // slot and phase parity of stage it - 1
    bool ok = true;
    for (uint32_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      uint32_t cnt = 0;
      for (uint32_t kt = 0; kt < KT; ++kt, ++it) {
        if (!(ok = mbar_wait(smem_u32(&full[s]), ph, abort_flag, gflags))) break;
        uint8_t* ra = sA(s) + row * 128u;
        uint8_t* ra2 = a2_slot + row * 128u;
        uint32_t w[16];
#pragma unroll
        for (uint32_t c = 0; c < 4; ++c) {
          const uint4 v = *reinterpret_cast<const uint4*>(ra + (((c0 + c) ^ sw) << 4));
          w[4 * c] = v.x;
          w[4 * c + 1] = v.y;
          w[4 * c + 2] = v.z;
          w[4 * c + 3] = v.w;
        }
        uint32_t any = 0u, big = 0u;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          cnt = __dp2a_lo(w[q], 0x00000101u, cnt);  // + low half + high half
          any |= w[q];
        }
        const uint32_t over = any & kOverMask;
        if (kSplit && over != 0u) {
#pragma unroll
          for (int q = 0; q < 16; ++q) big |= __vcmpgtu2(w[q], 0x08000800u);
        }
        uint32_t hi[16], lo[16];
        if (over == 0u) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            if (kSplit) {
              __half2 h = __halves2half2(__ushort_as_half(0), __ushort_as_half(0));
              const uint32_t bits = w[q] | 0x64006400u;
              memcpy(&h, &bits, 4);
              h = __hsub2(h, __halves2half2(__ushort_as_half(0x6400), __ushort_as_half(0x6400)));
              memcpy(&hi[q], &h, 4);
            } else {
              __nv_bfloat162 h;
              const uint32_t bits = w[q] | 0x43004300u;
              memcpy(&h, &bits, 4);
              h = __hsub2(h, __halves2bfloat162(__ushort_as_bfloat16(0x4300), __ushort_as_bfloat16(0x4300)));
              memcpy(&hi[q], &h, 4);
            }
            lo[q] = 0u;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            uint32_t y0 = w[q] & 0xffffu, y1 = w[q] >> 16;
            if (kSplit) {
              uint32_t l0 = 0u, l1 = 0u;
              if (y0 > 2048u) {
                l0 = y0 & 31u;
                y0 &= ~31u;
              }
              if (y1 > 2048u) {
                l1 = y1 & 31u;
                y1 &= ~31u;
              }
              hi[q] = uint32_t(__half_as_ushort(__uint2half_rn(y0))) |
                      (uint32_t(__half_as_ushort(__uint2half_rn(y1))) << 16);
              lo[q] = uint32_t(__half_as_ushort(__uint2half_rn(l0))) |
                      (uint32_t(__half_as_ushort(__uint2half_rn(l1))) << 16);
            } else {
              hi[q] = uint32_t(__bfloat16_as_ushort(__uint2bfloat16_rn(y0))) |
                      (uint32_t(__bfloat16_as_ushort(__uint2bfloat16_rn(y1))) << 16);
              lo[q] = 0u;
            }
          }
        }
        const bool large = kSplit && big != 0u;
        const bool rewrite_a2 = kSplit && (large || dirty);
        // Stage it - 1's MMAs complete phase pph of empty[ps]. That barrier is
        // at most one phase behind it: this thread converted stage it - 1,
        // whose data the producer loaded only after the previous phase
        // completed. So the parity wait cannot alias an older phase.
        if (rewrite_a2 && it > 0u && !(ok = mbar_wait(smem_u32(&empty[ps]), pph, abort_flag, gflags))) break;
#pragma unroll
        for (uint32_t c = 0; c < 4; ++c) {
          const uint32_t off = ((c0 + c) ^ sw) << 4;
          *reinterpret_cast<uint4*>(ra + off) = make_uint4(hi[4 * c], hi[4 * c + 1], hi[4 * c + 2], hi[4 * c + 3]);
          if (rewrite_a2)
            *reinterpret_cast<uint4*>(ra2 + off) = make_uint4(lo[4 * c], lo[4 * c + 1], lo[4 * c + 2], lo[4 * c + 3]);
        }
        if (kSplit) {
          dirty = large;
          if (large) split_gen[s] = it;
        }
        fence_proxy_async_smem();
        mbar_arrive(smem_u32(&conv[s]));
        ps = s;
        pph = ph;
        if (++s == ST) {
          s = 0;
          ph ^= 1u;
        }
      }
      if (!ok) break;
      const uint32_t p = tile * kTileM + row;
      if (p < P) atomicAdd(n + p, cnt);  // two halves per row; n was zeroed before the launch
    }
  } else if (warp >= 12) {
    // ---------------------------------------------------------------- epilogue
    const uint32_t q = warp & 3u;  // TMEM lane quadrant of this warp
    const uint32_t acc_cols = ncols_alloc / 2;
    uint32_t lt = 0;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
      const uint32_t acc = lt & 1u, aph = (lt >> 1) & 1u;
      if (!mbar_wait(smem_u32(&tfull[acc]), aph, abort_flag, gflags)) break;
      tc_fence_after();
      const uint32_t taddr = tmem_base + ((q * 32u) << 16) + acc * acc_cols;
      const uint32_t p = tile * kTileM + q * 32u + lane;
      float2* Sp = S + size_t(p) * m;
      for (uint32_t c0 = 0; c0 < N2; c0 += 16u) {
        uint32_t vh[16], vl[16];
        tmem_ld16(taddr + c0, vh);
        if (kSplit) tmem_ld16(taddr + N2 + c0, vl);
        tmem_ld_wait();
        if (p < P) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const uint32_t l = (c0 >> 1) + uint32_t(j);
            if (l < m) {
              float re = __uint_as_float(vh[2 * j]), im = __uint_as_float(vh[2 * j + 1]);
              if (kSplit) {
                re += __uint_as_float(vl[2 * j]);
                im += __uint_as_float(vl[2 * j + 1]);
              }
              Sp[l] = make_float2(re, im);
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&tempty[acc]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem_base, ncols_alloc);
  }
}

// ------------------------------------------------------------------ host side

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D u16 map: rows x T elements, box {64, box_rows}, 128-byte swizzle.
bool encode_map(CUtensorMap* map, const void* ptr, uint64_t rows, uint32_t T, uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {T, rows};
  const cuuint64_t strides[1] = {uint64_t(T) * 2u};
  const cuuint32_t box[2] = {uint32_t(kTileK), box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// F^T operand for (T, m, precision), built on the host from cos/sin in double:
// FP16_SPLIT: rows [0, N2) hold F_hi = fp16(F), rows [N2, 2 N2) F_lo = fp16(F - F_hi);
// BF16: rows [0, N2) hold bf16(F). Rows beyond 2m are zero.
srt3d_status get_fourier_operand(srt3d_ctx* ctx, uint32_t T, uint32_t m, int precision, uint32_t N2,
                                 const uint16_t** out) {
  std::lock_guard<std::mutex> lock(ctx->mu);
  auto key = std::make_tuple(T, m, precision);
  auto itf = ctx->fourier.find(key);
  if (itf != ctx->fourier.end()) {
    *out = static_cast<const uint16_t*>(itf->second.ptr);
    return SRT3D_OK;
  }
  const bool split = precision == SRT3D_FP16_SPLIT;
  const uint32_t rows = split ? 2 * N2 : N2;
  std::vector<uint16_t> host(size_t(rows) * T, 0);
  for (uint32_t l = 1; l <= m; ++l) {
    for (uint32_t b = 0; b < T; ++b) {
      const uint64_t k = (uint64_t(l) * b) % T;
      const double a = 2.0 * M_PI * double(k) / double(T);
      const double v[2] = {std::cos(a), std::sin(a)};
      for (int c = 0; c < 2; ++c) {
        const uint32_t r = 2 * (l - 1) + c;
        if (split) {
          const __half hi = __float2half_rn(float(v[c]));
          const __half lo = __float2half_rn(float(v[c] - double(__half2float(hi))));
          host[size_t(r) * T + b] = __half_as_ushort(hi);
          host[size_t(r + N2) * T + b] = __half_as_ushort(lo);
        } else {
          host[size_t(r) * T + b] = __bfloat16_as_ushort(__float2bfloat16_rn(float(v[c])));
        }
      }
    }
  }
  DevBuf buf;
  SRT3D_CUDA_TRY(ctx, cudaMalloc(&buf.ptr, host.size() * 2));
  buf.bytes = host.size() * 2;
  SRT3D_CUDA_TRY(ctx, cudaMemcpy(buf.ptr, host.data(), host.size() * 2, cudaMemcpyHostToDevice));
  ctx->fourier[key] = buf;
  *out = static_cast<const uint16_t*>(buf.ptr);
  return SRT3D_OK;
}

template <int PREC>
srt3d_status launch_tc(srt3d_ctx* ctx, const uint16_t* hist, uint32_t P, uint32_t T, uint32_t m, float2* S,
                       uint32_t* n, cudaStream_t stream) {
  using Cfg = TcCfg<PREC>;
  const uint32_t N2 = ((2 * m + 15) / 16) * 16;
  const uint32_t N = Cfg::kSplit ? 2 * N2 : N2;
  uint32_t ncols_alloc = 32;
  while (ncols_alloc < 2 * N) ncols_alloc <<= 1;
  const uint16_t* F = nullptr;
  srt3d_status st = get_fourier_operand(ctx, T, m, PREC, N2, &F);
  if (st != SRT3D_OK) return st;
  CUtensorMap mapY, mapF;
  if (!encode_map(&mapY, hist, P, T, kTileM) || !encode_map(&mapF, F, N, T, N))
    return set_error(ctx, SRT3D_ECUDA, "cuTensorMapEncodeTiled failed");
  // stages: as many as fit (at most kMaxStages) beside the A2 slot, the
  // 1024-byte alignment pad and the barrier block
  const size_t stage_bytes = size_t(kABytes) + size_t(N) * 128;
  const size_t fixed = 1024 + (Cfg::kSplit ? size_t(kABytes) : 0) + 512;
  const size_t fit = ctx->smem_optin > fixed ? (ctx->smem_optin - fixed) / stage_bytes : 0;
  const uint32_t ST = uint32_t(std::min<size_t>(kMaxStages, fit));
  if (ST < 2) return set_error(ctx, SRT3D_EINVAL, "tensor-core tile does not fit shared memory");
  const size_t smem = fixed + ST * stage_bytes;
  auto kfn = k_sketch_hist_tc<PREC>;
  SRT3D_CUDA_TRY(ctx, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  const uint32_t ntiles = (P + kTileM - 1) / kTileM;
  const uint32_t grid = std::min<uint32_t>(ntiles, uint32_t(ctx->num_sms));
  SRT3D_CUDA_TRY(ctx, cudaMemsetAsync(n, 0, size_t(P) * sizeof(uint32_t), stream));
  const ProfMark mk = prof_begin(ctx, KID_SKETCH_HIST_TC, stream);
  kfn<<<grid, kThreads, smem, stream>>>(mapY, mapF, P, T, m, N2, ncols_alloc, ST, S, n, ctx->d_flags);
  prof_end(ctx, KID_SKETCH_HIST_TC, mk, stream);
  SRT3D_CUDA_TRY(ctx, cudaGetLastError());
  return SRT3D_OK;
}

}  // namespace

srt3d_status launch_sketch_hist_tc(srt3d_ctx* ctx, const uint16_t* hist, uint32_t P, uint32_t T, uint32_t m,
                                   int precision, float2* S, uint32_t* n, cudaStream_t stream) {
  if (precision == SRT3D_FP16_SPLIT) return launch_tc<SRT3D_FP16_SPLIT>(ctx, hist, P, T, m, S, n, stream);
  return launch_tc<SRT3D_BF16>(ctx, hist, P, T, m, S, n, stream);
}

}  // namespace srt3d
