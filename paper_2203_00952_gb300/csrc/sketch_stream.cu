// Stream-path kernels (Sec. 2):
//   k_sketch_stream   S[p][l-1] = sum_x exp(i 2 pi ((l x) mod T) / T)   (Eq. 3)
//   k_hist_from_stream  y[p][b] = #{x = b}                               (Eq. 2)
//   k_finalize        z = S / n                                          (Eq. 3)
//
// Sketch kernel layout: a group of G lanes (G in {4, 8, 16, 32}) owns one
// pixel at a time. The pixel's whole 16-byte words (8 stamps, read from an
// aligned base so loads are coalesced whatever the pixel's offset) are spread
// over the lanes; the at most 14 stamps of its partial first and last words
// are taken one per lane in a separate pass, so no lane runs a masked
// per-stamp path while the others wait. Per photon the exact integer phase x
// indexes a shared-memory cos/sin table for e_1 = e^{i w_1 x}; higher
// harmonics follow the Chebyshev recurrence e_j = 2 cos(w_1 x) e_{j-1} -
// e_{j-2}, run on the signed sequence a_j = s_j e_j (s = +,+,-,-,+,+,...) so
// that every step is a single packed FMA a_j = (+-2 cos) a_{j-1} + a_{j-2} on
// the (cos, sin) pair, and a packed add accumulates it. For m > 10 the
// recurrence restarts from the table (exact index (j x) mod T) every 8
// harmonics. Rounding error per term: at most 3.5e-6 for m <= 10 and 2.3e-6
// with restarts (checked exhaustively over x for T from 256 to 8192). For
// T > 8192 the table is two-level and the harmonics come from complex
// rotation instead (see add_photon). Each
// lane keeps m complex FP32 partial sums; at the end of the pixel the group
// reduce-scatters them with xor shuffles (each lane ends with a few totals).
// No floating-point atomics: the result for a pixel does not depend on what
// else runs.
#include <cmath>
#include <cstdio>

#include "device_util.cuh"
#include "internal.h"

namespace srt3d {
namespace {

constexpr int kBlock = 256;
constexpr int kRestart = 8;       // direct table: restart every kRestart harmonics ...
constexpr int kRestartAbove = 10;  // ... when m exceeds this
constexpr int kResyncTL = 16;      // two-level table: resync of the rotation
constexpr int kOrTestMaxM = 4;     // whole-word range test by OR up to this m (then the maximum)

// What a sketch kernel does with its sums: overwrite S, add them into S (the
// online update of Sec. 2), or overwrite with z = S / n (one-shot batches,
// which then need no separate normalisation launch).
enum : int { kOverwrite = 0, kAccumulate = 1, kNormalise = 2 };

// acc[j-1] += s_j e_j, j = 1..M, from e_1 on the direct-table path: the
// Chebyshev recurrence on the signed sequence (see add_photon), restarted
// from the table at the exact integer phase every kRestart harmonics when M
// exceeds kRestartAbove.
template <int M>
__device__ __forceinline__ void chebyshev_from(pf2 (&acc)[M], const pf2 e1, uint32_t x, const pf2* ptab, uint32_t T,
                                               float invT) {
  const float c2 = pk_lo(e1) + pk_lo(e1);
  const pf2 pc = pk(c2, c2), nc = pk(-c2, -c2);
  pf2 p = pk(1.f, 0.f);  // a_{j-2}
  pf2 q = e1;            // a_{j-1}
  acc[0] = padd(acc[0], q);
#pragma unroll
  for (int j = 2; j <= M; ++j) {
    pf2 r;
    if (M > kRestartAbove && (j - 1) % kRestart == 0) {
      // a_{j-1} = e_{j-1}, a_j = e_j from the table (s = + at j - 1 = 0 mod 4 and j)
      const uint32_t k0 = mulmod(uint32_t(j - 1), x, T, invT);
      uint32_t k1 = k0 + x;
      k1 -= (k1 >= T) ? T : 0u;
      q = ptab[k0];
      r = ptab[k1];
    } else {
      r = pfma((j & 1) ? pc : nc, q, p);
    }
    p = q;
    q = r;
    acc[j - 1] = padd(acc[j - 1], r);
  }
}

// acc[j-1] += s_j e^{i w_j x} for j = 1..M, s_j = -1 when j mod 4 is 2 or 3
// (the caller flips those signs once per pixel); acc holds packed (Re, Im)
// pairs. Direct table: Chebyshev recurrence. Two-level table (T > 8192): its
// composed e_1 carries ~1.5 ulp, which the recurrence would amplify ~j^2-fold,
// so there the harmonics come from complex rotation e_j = e_{j-1} e_1 (error
// growing ~j-fold), resynced from the table every 16 harmonics, and the signs
// are applied per term.
template <int M, bool TL>
__device__ __forceinline__ void add_photon(pf2 (&acc)[M], uint32_t x, const float2* tab, uint32_t T, float invT) {
  const pf2* ptab = reinterpret_cast<const pf2*>(tab);
  if (TL) {
    const float2 e1 = phase(tab, x, true);
    float2 e = e1;
    acc[0] = padd(acc[0], pk(e.x, e.y));
#pragma unroll
    for (int j = 2; j <= M; ++j) {
      if ((j - 1) % kResyncTL == 0)
        e = phase(tab, mulmod(uint32_t(j), x, T, invT), true);
      else
        e = cmul(e, e1);
      acc[j - 1] = (j & 2) ? psub(acc[j - 1], pk(e.x, e.y)) : padd(acc[j - 1], pk(e.x, e.y));
    }
    return;
  }
  chebyshev_from<M>(acc, ptab[x], x, ptab, T, invT);
}

// Stamps of each 16-byte word (of 8) whose first-harmonic phasor comes from
// the special-function unit instead of the table, direct-table path only. At
// one or two harmonics the table lookups (random indices: ~6 shared-memory
// wavefronts per warp-wide lookup) keep the L1/shared pipe busier than HBM
// keeps the loads (81 % L1TEX throughput at m = 1); computing half of the
// phasors on the SFU, which no other stage uses, shares that load (12 % faster
// at m = 1). From three harmonics on the extra work of forming harmonics from
// an SFU phasor costs more than it saves, and every phasor comes from the table.
template <int M>
constexpr int sfu_photons() {
  return M <= 2 ? 4 : 0;
}

// add_photon (direct table) with e_1 from the special-function unit. The
// stamp's 16 bits are placed in the mantissa of 2^23 (one byte permute) and
// 2^23 subtracted, giving x exactly as a float; the phase in revolutions
// r = x / T - 1/2 lies in [-1/2, 1/2) (exact when T is a power of two), so the
// SFU sees the argument 2 pi r in [-pi, pi), where its sine and cosine are
// accurate to ~4e-7 absolute, and e^{i w x} = -e^{i 2 pi r}: the sums take
// the negated phasor. Harmonic 2 follows the Chebyshev step (error ~2x that
// of e_1). `sel` picks the stamp's half of the word: 0x5410 low, 0x5432 high.
template <int M>
__device__ __forceinline__ void add_photon_sfu(pf2 (&acc)[M], uint32_t word, uint32_t sel, float invT) {
  if constexpr (M <= 2) {  // (sfu_photons is 0 above two harmonics)
    const float xf = __uint_as_float(__byte_perm(word, 0x4b00u, sel)) - 8388608.0f;
    const float r = fmaf(xf, invT, -0.5f);
    float sn, cs;
    __sincosf(6.283185307179586f * r, &sn, &cs);
    const pf2 e = pk(cs, sn);  // = -e_1
    acc[0] = psub(acc[0], e);
    if constexpr (M == 2) {
      // a_2 = -e_2 = e_0 - 2 cos(w x) e_1 = 1 - 2 cs e (signed sequence, s_2 = -1)
      const pf2 a2 = pfma(pk(-2.f * cs, -2.f * cs), e, pk(1.f, 0.f));
      acc[1] = padd(acc[1], a2);
    }
  }
}

__device__ __forceinline__ uint4 ld_stream(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// The 8 stamps of one 16-byte word. hm has the bits at and above log2 of the
// largest power of two <= T set in both halves: a word whose OR has none of
// them holds only stamps < T (one test per word; for T not a power of two the
// word falls back to the exact maximum, then to per-stamp checks).
template <int M, bool TL>
__device__ __forceinline__ void word_photons(pf2 (&acc)[M], const uint4 v, const float2* s_tab, uint32_t T,
                                             float invT, uint32_t hm, bool& bad) {
  const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
  const uint32_t x[8] = {v.x & 0xffffu, v.x >> 16, v.y & 0xffffu, v.y >> 16,
                         v.z & 0xffffu, v.z >> 16, v.w & 0xffffu, v.w >> 16};
  constexpr int NS = TL ? 0 : sfu_photons<M>();
  bool ok;
  if constexpr (M <= kOrTestMaxM) {
    ok = ((v.x | v.y | v.z | v.w) & hm) == 0u;
    if (!ok) {
      const uint32_t mx = max(max(max(x[0], x[1]), max(x[2], x[3])), max(max(x[4], x[5]), max(x[6], x[7])));
      ok = mx < T;
    }
  } else {
    ok = max(max(max(x[0], x[1]), max(x[2], x[3])), max(max(x[4], x[5]), max(x[6], x[7]))) < T;
  }
  if (ok) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i >= 8 - NS)
        add_photon_sfu<M>(acc, wv[i >> 1], (i & 1) ? 0x5432u : 0x5410u, invT);
      else
        add_photon<M, TL>(acc, x[i], s_tab, T, invT);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (x[i] >= T)
        bad = true;
      else if (i >= 8 - NS)
        add_photon_sfu<M>(acc, wv[i >> 1], (i & 1) ? 0x5432u : 0x5410u, invT);
      else
        add_photon<M, TL>(acc, x[i], s_tab, T, invT);
    }
  }
}

// Positions of one pixel's stamps relative to the aligned base of the stamp
// array: [a, b). Derived: whole 16-byte words [wa, wb) = [ceil(a/8), floor(b/8)),
// loose stamps [a, he) and [ts, b) in the partial first and last words (nl of
// them, nh in the first). Only a and b are kept in registers.
struct PixelSpan {
  uint32_t a, b;
  __device__ __forceinline__ uint32_t wa() const { return (a + 7u) >> 3; }
  __device__ __forceinline__ uint32_t wb() const { return b >> 3; }
  __device__ __forceinline__ uint32_t he() const { return min(b, wa() << 3); }
  __device__ __forceinline__ uint32_t ts() const { return max(he(), wb() << 3); }
  __device__ __forceinline__ uint32_t nh() const { return he() - a; }
  __device__ __forceinline__ uint32_t nl() const { return nh() + (b - ts()); }
  // position of the i-th loose stamp (i < nl)
  __device__ __forceinline__ uint32_t loose(uint32_t i) const { return i < nh() ? a + i : ts() + (i - nh()); }
};

// Span of CSR offsets (s, e); malformed offsets (e < s or e > num_stamps)
// give an empty span and set `bad`.
__device__ __forceinline__ PixelSpan pixel_span(uint32_t s, uint32_t e, uint32_t shift, uint32_t num_stamps,
                                                bool& bad) {
  if (e < s || e > num_stamps) {
    bad = true;
    s = e = 0;
  }
  return PixelSpan{s + shift, e + shift};
}

// The loads of one pixel that lane gl issues ahead of its use: its first D
// whole words (wa + gl + j G) and its first loose stamp (~0u: none).
template <int D>
struct PixelLoads {
  uint4 w[D];
  uint32_t loose;
};

template <int D>
__device__ __forceinline__ void issue_loads(PixelLoads<D>& L, const PixelSpan& r, const uint4* __restrict__ words,
                                            const uint16_t* __restrict__ half, uint32_t G, uint32_t gl) {
  const uint32_t wa = r.wa(), wb = r.wb();
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const uint32_t w = wa + gl + uint32_t(j) * G;
    L.w[j] = make_uint4(0u, 0u, 0u, 0u);
    if (w < wb) L.w[j] = ld_stream(words + w);
  }
  L.loose = 0xffffffffu;
  if (gl < r.nl()) L.loose = __ldg(half + r.loose(gl));
}

// All photons of one pixel for lane gl, from loads issued one pixel ahead:
// the prefetched loose stamp and words, then the lane's further loose stamps
// (groups narrower than the pixel's loose-stamp count) and whole words (one
// load ahead). Returns whether a stamp was >= T.
template <int M, bool TL, int D>
__device__ __forceinline__ bool pixel_photons(pf2 (&acc)[M], const PixelLoads<D>& L, const PixelSpan& r,
                                              const uint4* __restrict__ words, const uint16_t* __restrict__ half,
                                              uint32_t T, float invT, uint32_t hm, uint32_t G, uint32_t gl,
                                              const float2* s_tab) {
  bool bad = false;
  if (L.loose != 0xffffffffu) {
    if (L.loose < T)
      add_photon<M, TL>(acc, L.loose, s_tab, T, invT);
    else
      bad = true;
  }
  for (uint32_t i = gl + G; i < r.nl(); i += G) {
    const uint32_t x = __ldg(half + r.loose(i));
    if (x < T)
      add_photon<M, TL>(acc, x, s_tab, T, invT);
    else
      bad = true;
  }
  const uint32_t wa = r.wa(), wb = r.wb();
#pragma unroll
  for (int j = 0; j < D; ++j)
    if (wa + gl + uint32_t(j) * G < wb) word_photons<M, TL>(acc, L.w[j], s_tab, T, invT, hm, bad);
  uint32_t w = wa + gl + uint32_t(D) * G;
  if (w < wb) {
    uint4 v = ld_stream(words + w);
    for (;;) {
      const uint32_t wn = w + G;
      uint4 vn = make_uint4(0u, 0u, 0u, 0u);
      if (wn < wb) vn = ld_stream(words + wn);
      word_photons<M, TL>(acc, v, s_tab, T, invT, hm, bad);
      if (wn >= wb) break;
      v = vn;
      w = wn;
    }
  }
  return bad;
}

// Reduce-scatter over the 2^LG lanes of a group: each step exchanges half of
// the lane's vector with the partner lane (lane ^ offset) and adds, so after
// LG steps a lane holds the group totals of entries [base, base + cnt) of the
// original vector in res[0..cnt) (cnt <= RsOut<L, LG>::n; an odd length is
// padded with a zero entry, which belongs to no one). One shuffle per kept
// entry per step instead of one per entry per step.
template <int L, int LG>
struct RsOut {
  static constexpr int n = RsOut<(L + 1) / 2, LG - 1>::n;
};
template <int L>
struct RsOut<L, 0> {
  static constexpr int n = L;
};

template <int L, int LG>
__device__ __forceinline__ void reduce_scatter(const float (&v)[L], uint32_t gl, unsigned gmask, uint32_t& base,
                                               uint32_t& cnt, float (&res)[RsOut<L, LG>::n]) {
  if constexpr (LG == 0) {
#pragma unroll
    for (int i = 0; i < L; ++i) res[i] = v[i];
  } else if constexpr (L == 1) {
    // one entry left: a butterfly gives every lane the total (the same sum
    // on both sides of each exchange), and the group's first lane keeps it
    float t = v[0];
#pragma unroll
    for (int k = LG - 1; k >= 0; --k) t += __shfl_xor_sync(gmask, t, 1u << k);
    res[0] = t;
    if (gl & ((1u << LG) - 1u)) cnt = 0u;
  } else {
    constexpr int half = (L + 1) / 2;
    constexpr uint32_t o = 1u << (LG - 1);
    const bool up = (gl & o) != 0;
    float nv[half];
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float lo = v[i], hi = (i + half < L) ? v[i + half] : 0.f;
      nv[i] = (up ? hi : lo) + __shfl_xor_sync(gmask, up ? lo : hi, o);
    }
    if (up) {
      base += half;
      cnt = cnt > uint32_t(half) ? cnt - uint32_t(half) : 0u;
    } else {
      cnt = min(cnt, uint32_t(half));
    }
    reduce_scatter<half, LG - 1>(nv, gl, gmask, base, cnt, res);
  }
}

// Group totals of the M packed partial sums, signs s_j undone, stored (or
// accumulated) into S[p][0..m): each lane stores the entries it holds.
template <int M, int LG>
__device__ __forceinline__ void store_sums(const pf2 (&acc)[M], uint32_t gl, unsigned gmask, uint32_t m,
                                           int accumulate, uint32_t count, float* __restrict__ Sp) {
  float v[2 * M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const float2 f = upk(acc[j]);
    v[2 * j] = f.x;
    v[2 * j + 1] = f.y;
  }
  uint32_t base = 0, cnt = 2 * M;
  float res[RsOut<2 * M, LG>::n];
  reduce_scatter<2 * M, LG>(v, gl, gmask, base, cnt, res);
#pragma unroll
  for (int i = 0; i < RsOut<2 * M, LG>::n; ++i) {
    const uint32_t idx = base + uint32_t(i);
    if (uint32_t(i) < cnt && idx < 2u * m) {
      float x = ((idx >> 1) + 1u) & 2u ? -res[i] : res[i];
      if (accumulate == kAccumulate) x += Sp[idx];
      if (accumulate == kNormalise) x = count ? x / float(count) : 0.f;  // z = S / n as k_finalize rounds it
      Sp[idx] = x;
    }
  }
}

// Pixels p0, p0 + step, ... < p1 of the stream, each processed by this
// group of G lanes: coalesced 16-byte words from the aligned base, per-lane
// partial sums, xor-shuffle reduce-scatter, store (or accumulate) of
// S[p][0..m) and n[p]. The loads of the next pixel (its first D words per lane
// and its first loose stamp) are issued before the current pixel is
// processed, and the offsets of the pixel after it one pixel earlier still,
// so 2D words per lane can be in flight and no pixel starts with an idle load
// latency.
template <int M, bool TL, int D>
__device__ __forceinline__ void sketch_pixels(const uint4* __restrict__ words, uint32_t shift,
                                              const uint32_t* __restrict__ offsets, uint32_t num_stamps, uint32_t p0,
                                              uint32_t p1, uint32_t step, uint32_t T, float invT, uint32_t m,
                                              uint32_t G, uint32_t gl, unsigned gmask, int accumulate,
                                              const float2* s_tab, float2* __restrict__ S, uint32_t* __restrict__ n,
                                              uint32_t* __restrict__ flags) {
  if (p0 >= p1) return;
  const uint16_t* half = reinterpret_cast<const uint16_t*>(words);
  const uint32_t hm16 = (0xffffu << (31 - __clz(T))) & 0xffffu;  // T >= 2
  const uint32_t hm = hm16 | (hm16 << 16);
  bool bad_off = false;
  PixelSpan cur = pixel_span(__ldg(offsets + p0), __ldg(offsets + p0 + 1), shift, num_stamps, bad_off);
  PixelLoads<D> lc;
  issue_loads<D>(lc, cur, words, half, G, gl);
  // offsets of the next pixel
  uint32_t sn = 0, en = 0;
  if (uint64_t(p0) + step < p1) {
    sn = __ldg(offsets + p0 + step);
    en = __ldg(offsets + p0 + step + 1);
  }
  for (uint32_t p = p0; p < p1; p += step) {
    const bool more = uint64_t(p) + step < p1;
    PixelSpan nxt{0u, 0u};
    PixelLoads<D> ln;
    if (more) {
      nxt = pixel_span(sn, en, shift, num_stamps, bad_off);
      issue_loads<D>(ln, nxt, words, half, G, gl);
      if (uint64_t(p) + 2ull * step < p1) {
        sn = __ldg(offsets + p + 2 * step);
        en = __ldg(offsets + p + 2 * step + 1);
      }
    }
    pf2 acc[M];
#pragma unroll
    for (int j = 0; j < M; ++j) acc[j] = 0ull;  // (+0, +0)
    if (pixel_photons<M, TL, D>(acc, lc, cur, words, half, T, invT, hm, G, gl, s_tab)) atomicOr(flags, FLAG_STAMP_RANGE);
    float* Sp = reinterpret_cast<float*>(S + size_t(p) * m);
    switch (G) {
      case 4: store_sums<M, 2>(acc, gl, gmask, m, accumulate, cur.b - cur.a, Sp); break;
      case 8: store_sums<M, 3>(acc, gl, gmask, m, accumulate, cur.b - cur.a, Sp); break;
      case 16: store_sums<M, 4>(acc, gl, gmask, m, accumulate, cur.b - cur.a, Sp); break;
      default: store_sums<M, 5>(acc, gl, gmask, m, accumulate, cur.b - cur.a, Sp); break;
    }
    if (gl == 0) n[p] = (accumulate == kAccumulate ? n[p] : 0u) + (cur.b - cur.a);
    if (more) {
      cur = nxt;
      lc = ln;
    }
  }
  if (bad_off && gl == 0) atomicOr(flags, FLAG_OFFSETS);
}

// Words per lane requested one pixel ahead: deeper where the arithmetic per
// photon is light (few harmonics: bound by the loads in flight), one where
// the registers hold many partial sums (bound by the FP32 pipe).
template <int M>
constexpr int prefetch_depth() {
  return M <= 2 ? 2 : 1;
}

// Co-resident CTAs per SM the register allocation is held to.
template <int M>
constexpr int sketch_min_blocks() {
  return M <= 10 ? 4 : (M <= 16 ? 3 : 2);
}

template <int M>
__global__ void __launch_bounds__(kBlock, sketch_min_blocks<M>()) k_sketch_stream(
    const uint16_t* __restrict__ stamps, const uint32_t* __restrict__ offsets, uint32_t num_stamps,
    uint32_t P, uint32_t T, uint32_t m, int glog2, int accumulate, const float2* __restrict__ table,
    uint32_t tab_entries, int two_level, float2* __restrict__ S, uint32_t* __restrict__ n,
    uint32_t* __restrict__ flags) {
  extern __shared__ float2 s_tab[];
  for (uint32_t i = threadIdx.x; i < tab_entries; i += blockDim.x) s_tab[i] = table[i];
  __syncthreads();
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
  constexpr int D = prefetch_depth<M>();
  if (two_level)
    sketch_pixels<M, true, D>(words, shift, offsets, num_stamps, gid, P, ngroups, T, invT, m, G, gl, gmask,
                              accumulate, s_tab, S, n, flags);
  else
    sketch_pixels<M, false, D>(words, shift, offsets, num_stamps, gid, P, ngroups, T, invT, m, G, gl, gmask,
                               accumulate, s_tab, S, n, flags);
}

// Batched sketch of several frames in one persistent launch: the work list
// holds (frame, first pixel, last pixel) items of roughly equal photon
// counts; a CTA walks items blockIdx.x, blockIdx.x + gridDim.x, ..., reloading
// the phase table when the frame changes. Lanes per pixel come from the
// frame's descriptor (autotuned per photon-density class). Each pixel's sums
// are stored normalised, z = S / n, so the batch needs no separate
// normalisation launch.
template <int M>
__global__ void __launch_bounds__(kBlock, sketch_min_blocks<M>()) k_sketch_batch(const BatchFrame* __restrict__ frames,
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
    constexpr int D = prefetch_depth<M>();
    if (f.two_level)
      sketch_pixels<M, true, D>(words, shift, f.offsets, f.num_stamps, item.y + gid, item.z, ngroups, f.T, invT, f.m,
                                G, gl, gmask, kNormalise, s_tab, f.S, f.n, flags);
    else
      sketch_pixels<M, false, D>(words, shift, f.offsets, f.num_stamps, item.y + gid, item.z, ngroups, f.T, invT,
                                 f.m, G, gl, gmask, kNormalise, s_tab, f.S, f.n, flags);
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

// One warp per pixel at a time, with 8 KB of shared-memory counters per warp
// and no block-wide barrier. A pixel with at most 65535 photons (no bin can
// exceed a u16) counts into packed u16 pairs (bin b in half b & 1 of word
// b / 2), 4096 bins per window: the counter words are then the output row
// itself. A pixel with more photons counts into u32 counters, 2048 bins per
// window, saturated to 65535 (flagged) on output. Each window re-scans the
// pixel's stamps (T <= 4096 is one window). Stamps are read 8 per lane in
// flight. Rows are written 16 bytes per store when T is a multiple of 8 and
// the output is 16-byte aligned.
constexpr uint32_t kHistWarps = 4;            // warps per CTA
constexpr uint32_t kHistWords = 2048;         // u32 counter words per warp (8 KB)
constexpr uint32_t kHistBins16 = 2 * kHistWords;
constexpr uint32_t kHistBins32 = kHistWords;
constexpr int kHistUnroll = 8;

__device__ __forceinline__ uint32_t sat16(uint32_t c, bool& over) {
  over |= c > 65535u;
  return min(c, 65535u);
}

// Count the stamps [s, e) that fall in [b0, b0 + nb) into cnt (packed u16
// pairs when PACKED, else u32).
template <bool PACKED>
__device__ __forceinline__ void hist_count(const uint16_t* __restrict__ stamps, uint64_t s, uint64_t e, uint32_t T,
                                           uint32_t b0, uint32_t nb, uint32_t* cnt, uint32_t lane, bool& bad) {
  for (uint64_t i0 = s; i0 < e; i0 += 32u * kHistUnroll) {
    uint32_t x[kHistUnroll];
#pragma unroll
    for (int k = 0; k < kHistUnroll; ++k) {
      const uint64_t i = i0 + lane + 32u * k;
      x[k] = i < e ? uint32_t(__ldg(stamps + i)) : 0xffffffffu;
    }
#pragma unroll
    for (int k = 0; k < kHistUnroll; ++k) {
      if (x[k] == 0xffffffffu) continue;
      if (x[k] >= T) {
        bad = true;
        continue;
      }
      const uint32_t b = x[k] - b0;
      if (b < nb) {
        if (PACKED)
          atomicAdd(&cnt[b >> 1], 1u << ((b & 1u) << 4));
        else
          atomicAdd(&cnt[b], 1u);
      }
    }
  }
}

__global__ void __launch_bounds__(kHistWarps * 32) k_hist_from_stream(const uint16_t* __restrict__ stamps,
                                                                      const uint32_t* __restrict__ offsets,
                                                                      uint32_t num_stamps, uint32_t P, uint32_t T,
                                                                      uint16_t* __restrict__ hist,
                                                                      uint32_t* __restrict__ flags) {
  extern __shared__ __align__(16) uint32_t s_hist[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  uint32_t* cnt = s_hist + warp * kHistWords;
  uint4* cnt4 = reinterpret_cast<uint4*>(cnt);
  for (uint32_t j = lane; j < kHistWords / 4u; j += 32u) cnt4[j] = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp();
  const bool vec = (T % 8u) == 0u && (reinterpret_cast<uintptr_t>(hist) % 16u) == 0u;
  bool bad = false, over = false, bad_off = false;
  const uint64_t W = uint64_t(gridDim.x) * kHistWarps;
  for (uint64_t p = uint64_t(blockIdx.x) * kHistWarps + warp; p < P; p += W) {
    uint32_t s = __ldg(offsets + p), e = __ldg(offsets + p + 1);
    if (e < s || e > num_stamps) {
      bad_off = true;
      s = e = 0u;
    }
    uint16_t* row = hist + size_t(p) * T;
    if (e - s <= 65535u) {
      for (uint32_t b0 = 0; b0 < T; b0 += kHistBins16) {
        const uint32_t nb = min(kHistBins16, T - b0);
        hist_count<true>(stamps, s, e, T, b0, nb, cnt, lane, bad);
        __syncwarp();
        if (vec) {
          uint4* r4 = reinterpret_cast<uint4*>(row + b0);
          for (uint32_t j = lane; j < nb / 8u; j += 32u) {
            r4[j] = cnt4[j];
            cnt4[j] = make_uint4(0u, 0u, 0u, 0u);
          }
        } else {
          for (uint32_t j = lane; j < nb; j += 32u) row[b0 + j] = uint16_t(cnt[j >> 1] >> ((j & 1u) << 4));
          __syncwarp();
          for (uint32_t j = lane; j < (nb + 1u) / 2u; j += 32u) cnt[j] = 0u;
        }
        __syncwarp();
      }
    } else {
      for (uint32_t b0 = 0; b0 < T; b0 += kHistBins32) {
        const uint32_t nb = min(kHistBins32, T - b0);
        hist_count<false>(stamps, s, e, T, b0, nb, cnt, lane, bad);
        __syncwarp();
        if (vec) {
          uint4* r4 = reinterpret_cast<uint4*>(row + b0);
          for (uint32_t j = lane; j < nb / 8u; j += 32u) {
            const uint4 a = cnt4[2 * j], b = cnt4[2 * j + 1];
            cnt4[2 * j] = make_uint4(0u, 0u, 0u, 0u);
            cnt4[2 * j + 1] = make_uint4(0u, 0u, 0u, 0u);
            uint4 o;
            o.x = sat16(a.x, over) | (sat16(a.y, over) << 16);
            o.y = sat16(a.z, over) | (sat16(a.w, over) << 16);
            o.z = sat16(b.x, over) | (sat16(b.y, over) << 16);
            o.w = sat16(b.z, over) | (sat16(b.w, over) << 16);
            r4[j] = o;
          }
        } else {
          for (uint32_t j = lane; j < nb; j += 32u) {
            row[b0 + j] = uint16_t(sat16(cnt[j], over));
            cnt[j] = 0u;
          }
        }
        __syncwarp();
      }
    }
  }
  if (bad_off) atomicOr(flags, FLAG_OFFSETS);
  if (bad) atomicOr(flags, FLAG_STAMP_RANGE);
  if (over) atomicOr(flags, FLAG_COUNT_RANGE);
}

}  // namespace

int sketch_default_glog2(double mean) {
  // dense pixels take half a warp each: two pixels' loads and reductions
  // overlap in one warp (3 to 7 % faster than a whole warp per pixel at
  // ~1000 photons per pixel, m = 1 to 10)
  return mean >= 96.0 ? 4 : mean >= 32.0 ? 3 : 2;
}

int sketch_glog2(srt3d_ctx* ctx, uint64_t num_stamps, uint32_t P, uint32_t T, uint32_t m) {
  // lanes per pixel: the autotuned value for this density class if there is
  // one, else a whole warp for dense pixels and narrower groups for sparse ones
  const double mean = P ? double(num_stamps) / double(P) : 0.0;
  int glog2 = sketch_default_glog2(mean);
  const int M = sketch_round_m(m);
  std::lock_guard<std::mutex> lock(ctx->mu);
  const int bucket = mean < 1.0 ? 0 : int(std::log2(mean));
  auto it = ctx->tuned.find((uint64_t(M) << 40) | (uint64_t(T > kDirectTableMax) << 32) | uint64_t(bucket));
  if (it != ctx->tuned.end()) glog2 = it->second;
  return glog2;
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
  if (glog2 < 0) glog2 = sketch_glog2(ctx, num_stamps, P, T, m);
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

srt3d_status launch_hist_from_stream(srt3d_ctx* ctx, const uint16_t* stamps, const uint32_t* offsets,
                                     uint64_t num_stamps, uint32_t P, uint32_t T, uint16_t* hist,
                                     cudaStream_t stream) {
  constexpr uint32_t threads = kHistWarps * 32;
  const size_t smem = size_t(kHistWarps) * kHistWords * sizeof(uint32_t);
  int bps = 0;
  SRT3D_CUDA_TRY(ctx, cudaFuncSetAttribute(k_hist_from_stream, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           int(smem)));
  SRT3D_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_hist_from_stream, threads, smem));
  if (bps < 1) bps = 1;
  const uint64_t want = (uint64_t(P) + kHistWarps - 1) / kHistWarps;
  const uint32_t grid = uint32_t(std::min<uint64_t>(want, uint64_t(ctx->num_sms) * bps));
  const ProfMark mk = prof_begin(ctx, KID_HIST_FROM_STREAM, stream);
  k_hist_from_stream<<<grid, threads, smem, stream>>>(stamps, offsets, uint32_t(num_stamps), P, T, hist,
                                                      ctx->d_flags);
  prof_end(ctx, KID_HIST_FROM_STREAM, mk, stream);
  SRT3D_CUDA_TRY(ctx, cudaGetLastError());
  return SRT3D_OK;
}

}  // namespace srt3d
