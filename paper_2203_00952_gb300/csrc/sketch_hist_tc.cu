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
//
// Fused stream route (FUSED = true): no histogram in HBM. k_bucket_stream
// first counting-sorts each tile's in-range stamps by bin / 64, the stage that
// consumes them, into 2-byte entries (row << 6) | (bin & 63), and writes n.
// The producer then loads only F^T; the converter warps become builders: per
// stage they zero the A slot, add the stage's entries into it by shared-memory
// reductions on the packed u16 bins (the slot's swizzled layout, i.e. the
// tile the TMA would have brought), and convert it in place as above; the next
// stage's first entries are loaded while the current one converts. The
// builders agree on every early exit through a barrier reduction, so none
// waits at a named barrier that another has left.
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
constexpr uint32_t kBuildRegs = 8;                 // fused builders: entries per thread per batch
constexpr uint32_t kBuildBatch = 256u * kBuildRegs;  // entries per batch of the 256 builders

template <int PREC>
struct TcCfg {
  static constexpr bool kSplit = (PREC == SRT3D_FP16_SPLIT);
};

// ------------------------------------------------------------------ the kernel

// Barrier 1 over the 256 converter threads: true on every thread when v is
// true on any (barrier.red also orders their shared-memory accesses).
__device__ __forceinline__ bool conv_bar_any(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.cta.red.or.pred q, 1, 256, p;\n"
      " selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"(uint32_t(v))
      : "memory");
  return r != 0u;
}

__device__ __forceinline__ void conv_bar() { asm volatile("barrier.cta.sync 1, 256;" ::: "memory"); }

__device__ __forceinline__ void red_shared_add(uint32_t saddr, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(saddr), "r"(v) : "memory");
}

template <int PREC, bool FUSED>
__global__ void __launch_bounds__(kThreads, 1)
    k_sketch_hist_tc(const __grid_constant__ CUtensorMap mapY, const __grid_constant__ CUtensorMap mapF,
                     uint32_t P, uint32_t T, uint32_t m, uint32_t N2, uint32_t ncols_alloc, uint32_t ST,
                     float2* __restrict__ S, uint32_t* __restrict__ n, uint32_t* __restrict__ gflags,
                     const uint16_t* __restrict__ ent, const uint32_t* __restrict__ tinfo) {
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
          if (FUSED) {
            mbar_arrive_expect_tx(smem_u32(&full[s]), b_bytes);
          } else {
            mbar_arrive_expect_tx(smem_u32(&full[s]), kABytes + b_bytes);
            tma_load_2d(smem_u32(sA(s)), &mapY, smem_u32(&full[s]), int(kt * kTileK), int(tile * kTileM));
          }
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
    bool fail = false;  // FUSED: a wait of this thread gave up; the next vote ends every builder's loop
    for (uint32_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      uint32_t cnt = 0;
      const uint32_t* ti = FUSED ? tinfo + size_t(tile) * (KT + 2u) : nullptr;
      const uint32_t ebase = FUSED ? __ldg(ti) : 0u;
      // stage kt's entries are ent[ebase + start[kt], ebase + start[kt + 1]);
      // the first kBuildBatch of them are loaded one stage ahead, into pe. A
      // thread takes kBuildRegs consecutive entries (a pixel's entries sit
      // together in a bucket, so a warp's lanes then meet less on one word)
      uint32_t e_lo = 0u, e_hi = 0u;
      uint32_t pe[kBuildRegs];
      if (FUSED) {
        e_lo = ebase + __ldg(ti + 1);
        e_hi = ebase + __ldg(ti + 2);
#pragma unroll
        for (uint32_t k = 0; k < kBuildRegs; ++k) {
          const uint32_t i = e_lo + ct * kBuildRegs + k;
          pe[k] = i < e_hi ? uint32_t(__ldg(ent + i)) : 0xffffffffu;
        }
      }
      for (uint32_t kt = 0; kt < KT; ++kt, ++it) {
        uint8_t* ra = sA(s) + row * 128u;
        uint8_t* ra2 = a2_slot + row * 128u;
        if (FUSED) {
          // full[s] completes once F^T landed, i.e. after the MMAs that last
          // read slot s completed: the slot is free to rebuild
          const bool go = mbar_wait(smem_u32(&full[s]), ph, abort_flag, gflags);
          if (go) {
#pragma unroll
            for (uint32_t c = 0; c < 4; ++c)
              *reinterpret_cast<uint4*>(ra + (((c0 + c) ^ sw) << 4)) = make_uint4(0u, 0u, 0u, 0u);
          }
          if (conv_bar_any(fail || !go)) {
            ok = false;
            break;
          }
          // the stage's entries: bins [64 kt, 64 kt + 64) of the tile's rows
          const uint32_t n_hi = kt + 1u < KT ? ebase + __ldg(ti + 3u + kt) : e_hi;  // next stage's end
          uint8_t* a = sA(s);
          auto count = [&](uint32_t e) {
            const uint32_t r = (e >> 6) & 127u, b = e & 63u;  // r < 128 by construction
            // the u32 word of (r, b) in the 128-byte swizzled row, and the half of it
            const uint32_t off = r * 128u + ((((b >> 3) ^ (r & 7u)) << 4) | ((b & 6u) << 1));
            // by shared-window address: the slot pointer is generic, and a
            // generic atomic would take the slow path
            red_shared_add(smem_u32(a + off), 1u << ((b & 1u) << 4));
          };
#pragma unroll
          for (uint32_t k = 0; k < kBuildRegs; ++k)
            if (pe[k] != 0xffffffffu) count(pe[k]);
          for (uint32_t i0 = e_lo + kBuildBatch + ct * kBuildRegs; i0 < e_hi; i0 += kBuildBatch) {
            uint32_t e[kBuildRegs];
#pragma unroll
            for (uint32_t k = 0; k < kBuildRegs; ++k) {
              const uint32_t i = i0 + k;
              e[k] = i < e_hi ? uint32_t(__ldg(ent + i)) : 0xffffffffu;
            }
#pragma unroll
            for (uint32_t k = 0; k < kBuildRegs; ++k)
              if (e[k] != 0xffffffffu) count(e[k]);
          }
          // the next stage's first batch, in flight while this stage converts
          e_lo = e_hi;
          e_hi = n_hi;
#pragma unroll
          for (uint32_t k = 0; k < kBuildRegs; ++k) {
            const uint32_t i = e_lo + ct * kBuildRegs + k;
            pe[k] = i < e_hi ? uint32_t(__ldg(ent + i)) : 0xffffffffu;
          }
          conv_bar();
        } else {
          if (!(ok = mbar_wait(smem_u32(&full[s]), ph, abort_flag, gflags))) break;
        }
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
        if (rewrite_a2 && it > 0u && !mbar_wait(smem_u32(&empty[ps]), pph, abort_flag, gflags)) {
          if (!FUSED) {
            ok = false;
            break;
          }
          // no early exit between the builders' barriers: skip this stage's
          // writes and leave at the next vote (or at the end of the loops)
          fail = true;
          ps = s;
          pph = ph;
          if (++s == ST) {
            s = 0;
            ph ^= 1u;
          }
          continue;
        }
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
      if (!FUSED && p < P) atomicAdd(n + p, cnt);  // two halves per row; n was zeroed before the launch
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

// ------------------------------------------------------------------ stamp buckets (fused route)

// k_bucket_stream: for every tile of kTileM pixels, the tile's in-range stamps
// counting-sorted by bin / kTileK (the tensor-core stage that consumes them)
// and each pixel's count n of them,
// each as a 2-byte entry (row << 6) | (bin & 63). tinfo[tile] holds
// {base, start[0], ..., start[KT]}: stage kt's entries are
// ent[base + start[kt], base + start[kt + 1]). The bins' counts are what the
// histogram of Eq. 2 holds, so the order inside a bucket does not matter.
//
// Pass 1 reads the tile's stamps and counts each bucket (shared-memory
// atomics); a block scan turns the counts into the bucket starts and one
// global atomic claims the tile's range of ent. Pass 2 re-reads the stamps in
// chunks of kBucketChunk, sorts each chunk in shared memory by bucket, and
// writes every bucket's run of the chunk contiguously after the bucket's
// previous runs, so the global stores are coalesced. The photons of a pixel
// crowd into one or two buckets (the surface's return), so every bucket's
// counters are replicated R times, the replica chosen by the stamp's index:
// at most 32 / R lanes of a warp meet on one counter. A pixel counts at most
// its first 65535 stamps (more raise FLAG_COUNT_RANGE: every bin count then
// fits the 16-bit counters of the builders); stamps >= T are skipped and raise
// FLAG_STAMP_RANGE, and offsets out of order or past num_stamps raise
// FLAG_OFFSETS and leave the pixel empty.
constexpr uint32_t kBucketThreads = 256;
constexpr uint32_t kBucketChunk = 8192;
constexpr uint32_t kBucketUnroll = 8;                   // stamp loads in flight per lane
constexpr uint32_t kBucketHead = 128 + 128 + 132 + 16;  // u32 words before the bucket arrays

__host__ __device__ constexpr uint32_t bucket_rep_log2(uint32_t KT) {
  // four replicas up to T = 32768 (four CTAs per SM at T = 4096: every tile
  // of a 256 x 256 frame in one round), two above
  return KT <= 512u ? 2u : 1u;
}
__host__ __device__ constexpr size_t bucket_al256(size_t b) { return (b + 255) & ~size_t(255); }
__host__ __device__ constexpr size_t bucket_ent_bytes(uint64_t num_stamps) {
  return bucket_al256(size_t(num_stamps > 0 ? num_stamps : 1) * sizeof(uint16_t));
}
__host__ __device__ constexpr size_t bucket_tinfo_bytes(uint64_t ntiles, uint32_t T) {
  return bucket_al256(size_t(ntiles) * (T / kTileK + 2u) * sizeof(uint32_t));
}
__host__ __device__ constexpr size_t bucket_smem_bytes(uint32_t KT) {
  return (kBucketHead + 4u * (size_t(KT) << bucket_rep_log2(KT)) + KT + 4u) * sizeof(uint32_t) +
         3u * kBucketChunk * sizeof(uint16_t);
}

// Exclusive prefix sum of in[0, K) into out (may alias in) over the whole
// block; returns the total. s_warp holds 8 words. Every thread must call it.
__device__ uint32_t bucket_scan(const uint32_t* in, uint32_t* out, uint32_t K, uint32_t* s_warp) {
  const uint32_t q = (K + kBucketThreads - 1) / kBucketThreads;
  const uint32_t a = threadIdx.x * q, lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint32_t sum = 0;
  for (uint32_t j = 0; j < q; ++j)
    if (a + j < K) sum += in[a + j];
  uint32_t x = sum;
#pragma unroll
  for (uint32_t o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31u) s_warp[warp] = x;
  __syncthreads();
  uint32_t run = x - sum, total = 0;
  for (uint32_t w = 0; w < kBucketThreads / 32u; ++w) {
    const uint32_t v = s_warp[w];
    if (w < warp) run += v;
    total += v;
  }
  for (uint32_t j = 0; j < q; ++j)
    if (a + j < K) {
      const uint32_t v = in[a + j];
      out[a + j] = run;
      run += v;
    }
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(kBucketThreads) k_bucket_stream(const uint16_t* __restrict__ stamps,
                                                                   const uint32_t* __restrict__ offsets,
                                                                   uint32_t num_stamps, uint32_t P, uint32_t T,
                                                                   uint16_t* __restrict__ ent, uint32_t cap,
                                                                   uint32_t* __restrict__ tinfo,
                                                                   uint32_t* __restrict__ claim,
                                                                   uint32_t* __restrict__ n,
                                                                   uint32_t* __restrict__ flags) {
  extern __shared__ __align__(16) uint32_t smb[];
  const uint32_t KT = T / kTileK;
  const uint32_t rl = bucket_rep_log2(KT), R = 1u << rl, KR = KT << rl;
  uint32_t* s_beg = smb;          // [128] first stamp of each row
  uint32_t* s_len = s_beg + 128;  // [128] stamps of each row counted (at most 65535)
  uint32_t* s_R = s_len + 128;    // [132] exclusive prefix of s_len
  uint32_t* s_misc = s_R + 132;   // [16] scan partials, the tile's base and whether it fits
  uint32_t* cntr = smb + kBucketHead;  // [KR] tile counts per (bucket, replica), then their starts
  uint32_t* lc = cntr + KR;            // [KR] the chunk's counts per (bucket, replica)
  uint32_t* lo = lc + KR;              // [KR + 1] exclusive prefix of lc, and the chunk's total
  uint32_t* lcur = lo + KR + 4;        // [KR] scatter cursors
  uint32_t* gcur = lcur + KR;          // [KT] each bucket's next position in ent (from base)
  uint16_t* xe = reinterpret_cast<uint16_t*>(gcur + KT);  // [chunk] entry of each staged stamp
  uint16_t* xb = xe + kBucketChunk;                       // [chunk] its (bucket, replica), 0xffff out of range
  uint16_t* xo = xb + kBucketChunk;                       // [chunk] entries sorted by bucket
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  constexpr uint32_t kWarps = kBucketThreads / 32u;
  const uint32_t ntiles = (P + kTileM - 1) / kTileM;
  bool bad = false, bad_off = false, over = false;
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();  // the previous tile's shared arrays are no longer read
    if (tid < kTileM) {
      const uint32_t p = tile * kTileM + tid;
      uint32_t b = 0, len = 0;
      if (p < P) {
        const uint32_t s = __ldg(offsets + p), e = __ldg(offsets + p + 1);
        if (e < s || e > num_stamps) {
          bad_off = true;
        } else {
          b = s;
          len = e - s;
          if (len > 65535u) {
            over = true;
            len = 65535u;
          }
        }
      }
      s_beg[tid] = b;
      s_len[tid] = len;
    }
    for (uint32_t k = tid; k < KR; k += kBucketThreads) {
      cntr[k] = 0u;
      lc[k] = 0u;
    }
    __syncthreads();
    const uint32_t L = bucket_scan(s_len, s_R, kTileM, s_misc);
    // pass 1: counts per (bucket, replica = lane mod R), kBucketUnroll loads in flight per lane
    const uint32_t rep1 = lane & (R - 1u);
    for (uint32_t r = warp; r < kTileM; r += kWarps) {
      const uint32_t b = s_beg[r], len = s_len[r];
      uint32_t inr = 0;  // the row's in-range stamps: n of Eq. 3
      for (uint32_t j0 = 0; j0 < len; j0 += 32u * kBucketUnroll) {
        uint32_t x[kBucketUnroll];
#pragma unroll
        for (uint32_t k = 0; k < kBucketUnroll; ++k) {
          const uint32_t j = j0 + lane + 32u * k;
          x[k] = j < len ? uint32_t(__ldg(stamps + b + j)) : 0xffffffffu;
        }
#pragma unroll
        for (uint32_t k = 0; k < kBucketUnroll; ++k) {
          if (x[k] == 0xffffffffu) continue;
          if (x[k] < T) {
            atomicAdd(&cntr[((x[k] / kTileK) << rl) | rep1], 1u);
            ++inr;
          } else {
            bad = true;
          }
        }
      }
      inr = __reduce_add_sync(0xffffffffu, inr);
      const uint32_t p = tile * kTileM + r;
      if (lane == 0 && p < P) n[p] = inr;
    }
    __syncthreads();
    const uint32_t V = bucket_scan(cntr, cntr, KR, s_misc);  // cntr[k R] = start of bucket k
    if (tid == 0) {
      const uint32_t base = atomicAdd(claim, V);
      const bool fits = uint64_t(base) + V <= cap;  // only overlapping pixel ranges can overrun
      if (!fits) bad_off = true;
      s_misc[8] = fits ? base : 0u;
      s_misc[9] = fits ? 1u : 0u;
    }
    __syncthreads();
    const uint32_t base = s_misc[8];
    const bool fits = s_misc[9] != 0u;
    uint32_t* ti = tinfo + size_t(tile) * (KT + 2u);
    if (tid == 0) ti[0] = base;
    for (uint32_t k = tid; k <= KT; k += kBucketThreads) {
      const uint32_t st = k < KT ? cntr[k << rl] : V;
      ti[1 + k] = fits ? st : 0u;
      if (k < KT) gcur[k] = st;
    }
    if (!fits) continue;
    // pass 2: chunks of the tile's stamps, sorted by bucket in shared memory;
    // the replica of the stamp at chunk position i is i mod R
    for (uint32_t c0 = 0; c0 < L; c0 += kBucketChunk) {
      const uint32_t nc = min(kBucketChunk, L - c0);
      for (uint32_t r = warp; r < kTileM; r += kWarps) {
        const uint32_t R0 = s_R[r], len = s_len[r];
        if (R0 + len <= c0 || R0 >= c0 + nc) continue;
        const uint32_t j0 = c0 > R0 ? c0 - R0 : 0u, j1 = min(len, c0 + nc - R0);
        const uint32_t b = s_beg[r];
        for (uint32_t jj = j0; jj < j1; jj += 32u * kBucketUnroll) {
          uint32_t x[kBucketUnroll];
#pragma unroll
          for (uint32_t k = 0; k < kBucketUnroll; ++k) {
            const uint32_t j = jj + lane + 32u * k;
            x[k] = j < j1 ? uint32_t(__ldg(stamps + b + j)) : 0xffffffffu;
          }
#pragma unroll
          for (uint32_t k = 0; k < kBucketUnroll; ++k) {
            if (x[k] == 0xffffffffu) continue;
            const uint32_t i = R0 + jj + lane + 32u * k - c0;
            if (x[k] < T) {
              const uint32_t kr = ((x[k] / kTileK) << rl) | (i & (R - 1u));
              xe[i] = uint16_t((r << 6) | (x[k] & (kTileK - 1)));
              xb[i] = uint16_t(kr);
              atomicAdd(&lc[kr], 1u);
            } else {
              xb[i] = 0xffffu;
            }
          }
        }
      }
      __syncthreads();
      const uint32_t nv = bucket_scan(lc, lo, KR, s_misc);
      for (uint32_t k = tid; k < KR; k += kBucketThreads) lcur[k] = lo[k];
      if (tid == 0) lo[KR] = nv;
      __syncthreads();
      for (uint32_t i = tid; i < nc; i += kBucketThreads) {
        const uint32_t kr = xb[i];
        if (kr != 0xffffu) xo[atomicAdd(&lcur[kr], 1u)] = xe[i];
      }
      __syncthreads();
      // bucket k's run of the chunk: xo[lo[k R], lo[(k + 1) R]) (its replicas are adjacent)
      for (uint32_t k = warp; k < KT; k += kWarps) {
        const uint32_t src = lo[k << rl], c = lo[(k + 1u) << rl] - src, dst = base + gcur[k];
        for (uint32_t j = lane; j < c; j += 32u) ent[dst + j] = xo[src + j];
        __syncwarp();
        if (lane == 0) gcur[k] += c;
      }
      for (uint32_t k = tid; k < KR; k += kBucketThreads) lc[k] = 0u;
      __syncthreads();
    }
  }
  if (bad_off) atomicOr(flags, FLAG_OFFSETS);
  if (bad) atomicOr(flags, FLAG_STAMP_RANGE);
  if (over) atomicOr(flags, FLAG_COUNT_RANGE);
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

// FUSED: hist is unused; ent / tinfo are k_bucket_stream's output.
template <int PREC, bool FUSED>
srt3d_status launch_tc(srt3d_ctx* ctx, const uint16_t* hist, uint32_t P, uint32_t T, uint32_t m, float2* S,
                       uint32_t* n, cudaStream_t stream, const uint16_t* ent = nullptr,
                       const uint32_t* tinfo = nullptr) {
  using Cfg = TcCfg<PREC>;
  const uint32_t N2 = ((2 * m + 15) / 16) * 16;
  const uint32_t N = Cfg::kSplit ? 2 * N2 : N2;
  uint32_t ncols_alloc = 32;
  while (ncols_alloc < 2 * N) ncols_alloc <<= 1;
  const uint16_t* F = nullptr;
  srt3d_status st = get_fourier_operand(ctx, T, m, PREC, N2, &F);
  if (st != SRT3D_OK) return st;
  CUtensorMap mapY, mapF;
  if (!encode_map(&mapF, F, N, T, N) || (FUSED ? (mapY = mapF, false) : !encode_map(&mapY, hist, P, T, kTileM)))
    return set_error(ctx, SRT3D_ECUDA, "cuTensorMapEncodeTiled failed");
  // stages: as many as fit (at most kMaxStages) beside the A2 slot, the
  // 1024-byte alignment pad and the barrier block
  const size_t stage_bytes = size_t(kABytes) + size_t(N) * 128;
  const size_t fixed = 1024 + (Cfg::kSplit ? size_t(kABytes) : 0) + 512;
  const size_t fit = ctx->smem_optin > fixed ? (ctx->smem_optin - fixed) / stage_bytes : 0;
  const uint32_t ST = uint32_t(std::min<size_t>(kMaxStages, fit));
  if (ST < 2) return set_error(ctx, SRT3D_EINVAL, "tensor-core tile does not fit shared memory");
  const size_t smem = fixed + ST * stage_bytes;
  auto kfn = k_sketch_hist_tc<PREC, FUSED>;
  SRT3D_CUDA_TRY(ctx, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  const uint32_t ntiles = (P + kTileM - 1) / kTileM;
  const uint32_t grid = std::min<uint32_t>(ntiles, uint32_t(ctx->num_sms));
  if (!FUSED) SRT3D_CUDA_TRY(ctx, cudaMemsetAsync(n, 0, size_t(P) * sizeof(uint32_t), stream));
  const int kid = FUSED ? KID_SKETCH_STREAM_TC : KID_SKETCH_HIST_TC;
  const ProfMark mk = prof_begin(ctx, kid, stream);
  kfn<<<grid, kThreads, smem, stream>>>(mapY, mapF, P, T, m, N2, ncols_alloc, ST, S, n, ctx->d_flags, ent, tinfo);
  prof_end(ctx, kid, mk, stream);
  SRT3D_CUDA_TRY(ctx, cudaGetLastError());
  return SRT3D_OK;
}

}  // namespace

srt3d_status launch_sketch_hist_tc(srt3d_ctx* ctx, const uint16_t* hist, uint32_t P, uint32_t T, uint32_t m,
                                   int precision, float2* S, uint32_t* n, cudaStream_t stream) {
  if (precision == SRT3D_FP16_SPLIT) return launch_tc<SRT3D_FP16_SPLIT, false>(ctx, hist, P, T, m, S, n, stream);
  return launch_tc<SRT3D_BF16, false>(ctx, hist, P, T, m, S, n, stream);
}

size_t stream_tc_fused_scratch_bytes(uint64_t num_stamps, uint32_t P, uint32_t T) {
  const uint64_t ntiles = (uint64_t(P) + kTileM - 1) / kTileM;
  return bucket_ent_bytes(num_stamps) + bucket_tinfo_bytes(ntiles, T) + 256;
}

srt3d_status launch_sketch_stream_tc_fused(srt3d_ctx* ctx, const uint16_t* stamps, const uint32_t* offsets,
                                           uint64_t num_stamps, uint32_t P, uint32_t T, uint32_t m, int precision,
                                           float2* S, uint32_t* n, void* scratch, cudaStream_t stream) {
  const uint32_t ntiles = (P + kTileM - 1) / kTileM;
  uint8_t* sc = static_cast<uint8_t*>(scratch);
  uint16_t* ent = reinterpret_cast<uint16_t*>(sc);
  uint32_t* tinfo = reinterpret_cast<uint32_t*>(sc + bucket_ent_bytes(num_stamps));
  uint32_t* claim = reinterpret_cast<uint32_t*>(sc + bucket_ent_bytes(num_stamps) + bucket_tinfo_bytes(ntiles, T));
  const uint32_t KT = T / kTileK;
  const size_t smem = bucket_smem_bytes(KT);
  SRT3D_CUDA_TRY(ctx, cudaFuncSetAttribute(k_bucket_stream, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  int bps = 0;
  SRT3D_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_bucket_stream, kBucketThreads, smem));
  if (bps < 1) bps = 1;
  const uint32_t grid = std::min<uint32_t>(ntiles, uint32_t(ctx->num_sms) * uint32_t(bps));
  SRT3D_CUDA_TRY(ctx, cudaMemsetAsync(claim, 0, sizeof(uint32_t), stream));
  const ProfMark mk = prof_begin(ctx, KID_BUCKET_STREAM, stream);
  k_bucket_stream<<<grid, kBucketThreads, smem, stream>>>(stamps, offsets, uint32_t(num_stamps), P, T, ent,
                                                          uint32_t(num_stamps), tinfo, claim, n, ctx->d_flags);
  prof_end(ctx, KID_BUCKET_STREAM, mk, stream);
  SRT3D_CUDA_TRY(ctx, cudaGetLastError());
  if (precision == SRT3D_FP16_SPLIT)
    return launch_tc<SRT3D_FP16_SPLIT, true>(ctx, nullptr, P, T, m, S, n, stream, ent, tinfo);
  return launch_tc<SRT3D_BF16, true>(ctx, nullptr, P, T, m, S, n, stream, ent, tinfo);
}

}  // namespace srt3d
