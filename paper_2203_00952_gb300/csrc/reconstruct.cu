// SRT3D reconstruction from sketches (Sec. 3, Eq. 8 with W = I).
//
// The paper replaces RT3D's histogram likelihood by the sketched loss
// n ||z - Psi_theta||^2 (Eq. 6) and keeps RT3D's point-cloud prior; the
// iteration implemented here (one reading of the cited RT3D) is, per pixel p
// with up to K = k_max <= 4 points (t_k, alpha_k):
//   k_prep    hhat_l = (1/H) sum_tau h(tau) e^{i w_l tau} (Eq. 4), the global
//             step sizes, and n_max
//   k_init    sketched matched filter (init.cu)
//   per iteration, one fused tile kernel (k_iter):
//             Jacobi gradient step on n ||z - Psi||^2 (t, alpha), alpha >= 0,
//             sum alpha <= 1; weighted least-squares plane normals over the
//             (2r+1)^2 x K neighbours gated by |dt| <= d_max and the APSS weight
//             (1 - d^2/h^2)^4; algebraic sphere fit with normals (Guennebaud &
//             Gross 2007) and projection along the line of sight; intensity
//             smoothing, pruning, alpha_0 = 1 - sum alpha
//   k_grad    the gradient step alone (pixelwise mode, no spatial prior)
// The iteration state lives in the caller's depth/alpha/active buffers (and,
// in the persistent kernel, in registers between iterations); the
// post-gradient state and the normals live in shared memory; hhat, the step
// sizes and the persistent kernel's exchange buffers live in a scratch block.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <utility>

#include "device_util.cuh"
#include "internal.h"

namespace srt3d {
namespace {

constexpr int kBlock = 256;
constexpr int kMaxM = 32;

struct Scratch {
  float* t1;
  float* a1;
  float* xch;  // exchange buffer 0 of the persistent kernel: t, alpha [P][K] f32, active [P][K] u8
  uint8_t* act1;
  float2* hh;
  float4* part;  // [m][kPrepSlices] partial sums (H, Re, Im) of hhat, slice after slice
  float* misc;
  unsigned* tile_flags;  // [kMaxTileFlags] progress of each tile of the persistent kernel
  // two tagged exchange buffers of the persistent kernel, [2][P][K] x 16 B
  // (nullptr when the block holds only the minimum layout)
  unsigned long long* xtag;
};

// Words of progress flags of the persistent kernel, one flag per tile every
// kTileFlagStride words (its own 32-byte L2 sector: flags that share a sector
// slow the polls down); frames with more tiles than fit run one launch per
// iteration.
constexpr uint32_t kMaxTileFlags = 4096;
// Slices of tau over which the CTAs of k_prep_part sum hhat.
constexpr uint32_t kPrepSlices = 8;
constexpr uint32_t kTileFlagStride = 8;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Bytes of the scratch block up to and including the progress flags (all a
// reconstruction needs) and of the tagged exchange buffers after them.
size_t scratch_min_bytes(uint32_t P, uint32_t K) {
  const size_t pk = size_t(P) * K;
  return align256(pk * 16) + 2 * align256(pk * sizeof(float)) + align256(pk) + align256(kMaxM * sizeof(float2)) +
         align256(kMaxM * kPrepSlices * sizeof(float4)) + align256(MISC_COUNT * sizeof(float)) +
         align256(kMaxTileFlags * sizeof(unsigned));
}
size_t scratch_xtag_bytes(uint32_t P, uint32_t K) { return align256(2 * size_t(P) * K * 16); }

Scratch carve(void* base, size_t bytes, uint32_t P, uint32_t K) {
  char* p = static_cast<char*>(base);
  Scratch s;
  const size_t pk = size_t(P) * K;
  s.xch = reinterpret_cast<float*>(p);
  p += align256(pk * 16);
  s.t1 = reinterpret_cast<float*>(p);
  p += align256(pk * sizeof(float));
  s.a1 = reinterpret_cast<float*>(p);
  p += align256(pk * sizeof(float));
  s.act1 = reinterpret_cast<uint8_t*>(p);
  p += align256(pk);
  s.hh = reinterpret_cast<float2*>(p);
  p += align256(kMaxM * sizeof(float2));
  s.part = reinterpret_cast<float4*>(p);
  p += align256(kMaxM * kPrepSlices * sizeof(float4));
  s.misc = reinterpret_cast<float*>(p);
  p += align256(MISC_COUNT * sizeof(float));
  s.tile_flags = reinterpret_cast<unsigned*>(p);
  p += align256(kMaxTileFlags * sizeof(unsigned));
  s.xtag = bytes >= scratch_min_bytes(P, K) + scratch_xtag_bytes(P, K) ? reinterpret_cast<unsigned long long*>(p)
                                                                       : nullptr;
  return s;
}

// hhat_l = (1/H) sum_tau h(tau) e^{i w_l tau} (Eq. 4) is summed over
// kPrepSlices slices of tau, each by a group of kPrepGroup threads (thread t
// takes tau = lo + t, lo + t + kPrepGroup, ... in order, kPrepUnroll terms
// per pass with their loads issued together; the group's warps reduce by xor
// shuffles and are added in warp order); the slices are then added in slice
// order. The single-frame path runs one group per CTA over many CTAs
// (k_prep_part, k_prep_final), the batch four groups per frame's CTA
// (k_prep_batch): the same sums in the same order, so both give the same
// hhat bit for bit. Phases from the table at the exact index (l tau) mod T.
constexpr int kPrepUnroll = 8;
constexpr uint32_t kPrepGroup = 256;
constexpr uint32_t kPrepGroupWarps = kPrepGroup / 32;

// This thread's (t in [0, kPrepGroup)) sums of slice sl of harmonic l,
// reduced over its warp (every lane gets the warp's sums).
__device__ __forceinline__ float3 prep_slice_warp(const float* __restrict__ h, uint32_t T, uint32_t l, uint32_t sl,
                                                  const float2* __restrict__ table, bool tl, uint32_t t) {
  const uint32_t lo = uint32_t(uint64_t(T) * sl / kPrepSlices), hi = uint32_t(uint64_t(T) * (sl + 1u) / kPrepSlices);
  const float invT = 1.0f / float(T);
  uint32_t tau = lo + t;
  uint32_t k = tau < hi ? mulmod(l, tau, T, invT) : 0u;
  const uint32_t dk = mulmod(l, kPrepGroup % T, T, invT);
  float hs = 0.f, re = 0.f, im = 0.f;
  for (; tau < hi; tau += kPrepUnroll * kPrepGroup) {
    float hv[kPrepUnroll];
    float2 e[kPrepUnroll];
#pragma unroll
    for (int j = 0; j < kPrepUnroll; ++j) {
      const uint32_t tj = tau + uint32_t(j) * kPrepGroup;  // terms past the slice add exact zeros
      hv[j] = tj < hi ? __ldg(h + tj) : 0.f;
      e[j] = tj < hi ? phase(table, k, tl) : make_float2(0.f, 0.f);
      k += dk;
      k -= (k >= T) ? T : 0u;
    }
#pragma unroll
    for (int j = 0; j < kPrepUnroll; ++j) {
      hs += hv[j];
      re = fmaf(hv[j], e[j].x, re);
      im = fmaf(hv[j], e[j].y, im);
    }
  }
  for (int off = 16; off; off >>= 1) {
    hs += __shfl_xor_sync(0xffffffffu, hs, off);
    re += __shfl_xor_sync(0xffffffffu, re, off);
    im += __shfl_xor_sync(0xffffffffu, im, off);
  }
  return make_float3(hs, re, im);
}

// The group's warps' sums added in warp order.
__device__ __forceinline__ float4 prep_slice_total(const float3* w) {
  float3 t = w[0];
  for (uint32_t i = 1; i < kPrepGroupWarps; ++i) {
    t.x += w[i].x;
    t.y += w[i].y;
    t.z += w[i].z;
  }
  return make_float4(t.x, t.y, t.z, 0.f);
}

// Warp 0: hhat from the slices (part[(l - 1) kPrepSlices + slice]), the
// step-size bases eta_t * n_max, eta_alpha * n_max and the misc scalars
// (n_max itself is left to the init kernels, which read every count anyway).
__device__ __forceinline__ void prep_final_warp(const float4* part, uint32_t T, uint32_t m, uint32_t K,
                                                float2* __restrict__ hh_out, float* __restrict__ misc) {
  const uint32_t lane = threadIdx.x & 31u;
  float sw = 0.f, sa = 0.f;
  if (lane < m) {
    float H = 0.f, R = 0.f, I = 0.f;
    for (uint32_t sl = 0; sl < kPrepSlices; ++sl) {
      const float4 v = part[lane * kPrepSlices + sl];
      H += v.x;
      R += v.y;
      I += v.z;
    }
    const float2 v = make_float2(R / H, I / H);
    hh_out[lane] = v;
    const float a = sqrtf(v.x * v.x + v.y * v.y);
    const float w = 6.283185307179586f * float(lane + 1u) / float(T);
    sw = w * w * a * (a + 2.f);
    sa = a * a;
  }
  for (int off = 16; off; off >>= 1) {
    sw += __shfl_xor_sync(0xffffffffu, sw, off);
    sa += __shfl_xor_sync(0xffffffffu, sa, off);
  }
  if (lane != 0) return;
  misc[MISC_ETA_T] = 1.f / (2.f * sw);
  misc[MISC_ETA_A] = 1.f / (2.f * float(K) * sa);
  misc[MISC_E2] = sa;
  reinterpret_cast<unsigned*>(misc)[MISC_NMAX] = 0u;  // n_max: atomicMax by the init kernels
  reinterpret_cast<unsigned*>(misc)[MISC_BAR] = 0u;
  reinterpret_cast<unsigned*>(misc)[MISC_BAR + 1] = 0u;
}

// Single frame: CTA (slice, l - 1) writes part[(l - 1) kPrepSlices + slice].
__global__ void __launch_bounds__(kPrepGroup) k_prep_part(const float* __restrict__ h, uint32_t T,
                                                          const float2* __restrict__ table, int two_level,
                                                          float4* __restrict__ part) {
  __shared__ float3 s_w[kPrepGroupWarps];
  const uint32_t sl = blockIdx.x, l = blockIdx.y + 1u;
  const float3 v = prep_slice_warp(h, T, l, sl, table, two_level != 0, threadIdx.x);
  if ((threadIdx.x & 31u) == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) part[(l - 1u) * kPrepSlices + sl] = prep_slice_total(s_w);
}

// Single frame: hhat and the scalars from the slices; zeroes the progress flags.
__global__ void __launch_bounds__(1024) k_prep_final(const float4* __restrict__ part, uint32_t T, uint32_t m,
                                                     uint32_t K, float2* __restrict__ hh_out,
                                                     float* __restrict__ misc, unsigned* __restrict__ tile_flags) {
  for (uint32_t i = threadIdx.x; i < kMaxTileFlags; i += blockDim.x) tile_flags[i] = 0u;
  if (threadIdx.x < 32) prep_final_warp(part, T, m, K, hh_out, misc);
}

// Batched: one block per frame of the batch, four slice groups at a time
// (each zeroes its tiles' flags).
__global__ void __launch_bounds__(1024) k_prep_batch(const BatchFrame* __restrict__ frames, uint32_t K,
                                                     unsigned* __restrict__ tile_flags) {
  constexpr uint32_t kGroups = 1024 / kPrepGroup;
  __shared__ float3 s_w[kGroups][kPrepGroupWarps];
  __shared__ float4 s_part[kMaxM * kPrepSlices];
  const BatchFrame& f = frames[blockIdx.x];
  unsigned* fl = tile_flags + size_t(f.tile0) * kTileFlagStride;
  const uint32_t flag_words = f.tiles_x * f.tiles_y * kTileFlagStride;
  for (uint32_t i = threadIdx.x; i < flag_words; i += blockDim.x) fl[i] = 0u;
  const uint32_t g = threadIdx.x / kPrepGroup, t = threadIdx.x % kPrepGroup;
  const uint32_t pairs = f.m * kPrepSlices;
  for (uint32_t base = 0; base < pairs; base += kGroups) {  // uniform trip count (barriers inside)
    const uint32_t pr = base + g;
    if (pr < pairs) {
      const float3 v = prep_slice_warp(f.h, f.T, pr / kPrepSlices + 1u, pr % kPrepSlices, f.table, f.two_level != 0, t);
      if ((t & 31u) == 0) s_w[g][t >> 5] = v;
    }
    __syncthreads();
    if (pr < pairs && t == 0) s_part[pr] = prep_slice_total(s_w[g]);
    __syncthreads();
  }
  if (threadIdx.x < 32) prep_final_warp(s_part, f.T, f.m, K, f.hh, f.misc);
}

// Sketched gradient step (Jacobi) of one pixel's K points: reads the state
// (t, a, act), returns the post-step (t, a); inactive points keep t, get a = 0.
// The gradient step of a pixel's two points (K = 2) with the phases and
// residual products of both points in packed FP32 pairs: per harmonic, q_k =
// hhat_l e^{i w_l t_k}, psi = sum_k a_k q_k, r = z_l - psi, the alpha gradient
// sums r . q_k, the depth gradient sums w_l Im(conj(q_k) r) (times a_k at the
// end), and e^{i w_l t_k} advances by one complex rotation. e^{i w_1 t_k}
// comes from the special-function unit: for t in [0, T) the phase in
// revolutions t / T - 1/2 lies in [-1/2, 1/2), where the SFU's sine and
// cosine are accurate to ~4e-7 absolute, and e^{i w_1 t} is the negated pair
// (a shorter dependent chain than the full-precision sincospi).
__device__ __forceinline__ void grad_pixel_pair(const float2* __restrict__ zp, uint32_t cnt, uint32_t T, uint32_t m,
                                                const float2* s_hh, float eta_t, float eta_a, float (&t)[2],
                                                float (&a)[2], const bool (&act)[2]) {
  const float Tf = float(T), invT = 1.f / Tf;
  float s0, c0, s1, c1;
  __sincosf(6.283185307179586f * fmaf(t[0], invT, -0.5f), &s0, &c0);
  __sincosf(6.283185307179586f * fmaf(t[1], invT, -0.5f), &s1, &c1);
  s0 = -s0;
  c0 = -c0;
  s1 = -s1;
  c1 = -c1;
  const float2 e1x = make_float2(c0, c1), e1y = make_float2(s0, s1), ne1y = make_float2(-s0, -s1);
  float2 Ex = e1x, Ey = e1y;
  const float aa0 = act[0] ? a[0] : 0.f, aa1 = act[1] ? a[1] : 0.f;
  float2 ga = make_float2(0.f, 0.f), gt = ga;
  const float wstep = 6.283185307179586f / Tf;
#pragma unroll 4
  for (uint32_t l = 0; l < m; ++l) {
    const float2 hv = s_hh[l];
    const float2 zl = zp[l];
    const float2 hx = make_float2(hv.x, hv.x), hy = make_float2(hv.y, hv.y), nhy = make_float2(-hv.y, -hv.y);
    const float2 qx = ffma2(hx, Ex, fmul2(nhy, Ey));
    const float2 qy = ffma2(hx, Ey, fmul2(hy, Ex));
    const float rx = zl.x - fmaf(aa1, qx.y, aa0 * qx.x);
    const float ry = zl.y - fmaf(aa1, qy.y, aa0 * qy.x);
    ga = ffma2(make_float2(ry, ry), qy, ffma2(make_float2(rx, rx), qx, ga));
    const float w = wstep * float(l + 1);
    const float2 cr = ffma2(make_float2(ry, ry), qx, fmul2(make_float2(-rx, -rx), qy));
    gt = ffma2(make_float2(w, w), cr, gt);
    const float2 nEx = ffma2(Ex, e1x, fmul2(Ey, ne1y));
    Ey = ffma2(Ex, e1y, fmul2(Ey, e1x));
    Ex = nEx;
  }
  const float nn = -2.f * float(cnt);
  const float gtk[2] = {a[0] * gt.x, a[1] * gt.y}, gak[2] = {ga.x, ga.y};
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    if (act[k]) {
      float x = t[k] - eta_t * (nn * gtk[k]);
      x -= floorf(x / Tf) * Tf;
      if (x >= Tf) x -= Tf;
      if (x < 0.f) x += Tf;
      t[k] = x;
      a[k] = fmaxf(a[k] - eta_a * (nn * gak[k]), 0.f);
    } else {
      a[k] = 0.f;
    }
    sum += a[k];
  }
  if (sum > 1.f) {
#pragma unroll
    for (int k = 0; k < 2; ++k) a[k] = a[k] / sum;
  }
}

template <int K>
__device__ __forceinline__ void grad_pixel(const float2* __restrict__ zp, uint32_t cnt, uint32_t T, uint32_t m,
                                           const float2* s_hh, float eta_t, float eta_a, float (&t)[K],
                                           float (&a)[K], const bool (&act)[K]) {
  if constexpr (K == 2) {
    grad_pixel_pair(zp, cnt, T, m, s_hh, eta_t, eta_a, t, a, act);
    return;
  }
  const float Tf = float(T), invT = 1.f / Tf;
  float2 e1[K], E[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float sn, cs;  // e^{i w_1 t} from the SFU as in grad_pixel_pair
    __sincosf(6.283185307179586f * fmaf(t[k], invT, -0.5f), &sn, &cs);
    e1[k] = make_float2(-cs, -sn);
    E[k] = e1[k];
  }
  float gt[K], ga[K];
#pragma unroll
  for (int k = 0; k < K; ++k) gt[k] = ga[k] = 0.f;
  const float wstep = 6.283185307179586f / Tf;
#pragma unroll 4
  for (uint32_t l = 0; l < m; ++l) {
    const float2 hv = s_hh[l];
    const float2 zl = zp[l];
    float2 q[K];
    float2 psi = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      q[k] = cmul(hv, E[k]);
      if (act[k]) {
        psi.x = fmaf(a[k], q[k].x, psi.x);
        psi.y = fmaf(a[k], q[k].y, psi.y);
      }
    }
    const float2 r = make_float2(zl.x - psi.x, zl.y - psi.y);
    const float w = wstep * float(l + 1);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      ga[k] += r.x * q[k].x + r.y * q[k].y;
      gt[k] += w * a[k] * (r.y * q[k].x - r.x * q[k].y);
      E[k] = cmul(E[k], e1[k]);
    }
  }
  const float nn = -2.f * float(cnt);
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (act[k]) {
      float x = t[k] - eta_t * (nn * gt[k]);
      x -= floorf(x / Tf) * Tf;
      if (x >= Tf) x -= Tf;
      if (x < 0.f) x += Tf;
      t[k] = x;
      a[k] = fmaxf(a[k] - eta_a * (nn * ga[k]), 0.f);
    } else {
      a[k] = 0.f;
    }
    sum += a[k];
  }
  if (sum > 1.f) {
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = a[k] / sum;
  }
}

// Ridge added to Sigma_theta before inverting it (Sigma_theta is singular for
// a noise-free point mass).
constexpr float kSigmaRidge = 1e-3f;

// Solves A x = y and A u = g for the Hermitian positive definite Toeplitz
// matrix A_jk = c_{j-k} (c_0 real, c_{-d} = conj(c_d)), size m, by the Levinson
// recursion (O(m^2) operations, O(m) storage): the forward vector f solves
// A_n f = e_1, the backward vector is its conjugate reversal, and each order
// n -> n + 1 updates f, x and u with the new row's residuals.
__device__ __forceinline__ void levinson2(float c0, const float2* c, uint32_t m, const float2* y, const float2* g,
                                          float2* f, float2* x, float2* u) {
  const float inv0 = 1.f / c0;
  f[0] = make_float2(inv0, 0.f);
  x[0] = make_float2(y[0].x * inv0, y[0].y * inv0);
  u[0] = make_float2(g[0].x * inv0, g[0].y * inv0);
  for (uint32_t n = 1; n < m; ++n) {
    // residuals of [f; 0], [x; 0], [u; 0] in the new row: sum_k c_{n-k} v_k
    float2 ef = make_float2(0.f, 0.f), ex = ef, eu = ef;
    for (uint32_t k = 0; k < n; ++k) {
      const float2 cv = c[n - k - 1];  // c_{n-k}
      ef = make_float2(ef.x + cv.x * f[k].x - cv.y * f[k].y, ef.y + cv.x * f[k].y + cv.y * f[k].x);
      ex = make_float2(ex.x + cv.x * x[k].x - cv.y * x[k].y, ex.y + cv.x * x[k].y + cv.y * x[k].x);
      eu = make_float2(eu.x + cv.x * u[k].x - cv.y * u[k].y, eu.y + cv.x * u[k].y + cv.y * u[k].x);
    }
    const float invD = 1.f / (1.f - (ef.x * ef.x + ef.y * ef.y));
    // f' = ([f; 0] - ef [0; b]) / D with b_j = conj(f_{n-1-j}), in place
    // over the pairs (k, n - k)
    f[n] = make_float2(0.f, 0.f);
    for (uint32_t k = 0, j = n; k <= j; ++k, --j) {
      const float2 fk = f[k], fj = f[j];
      const float2 ck = make_float2(fj.x, -fj.y), cj = make_float2(fk.x, -fk.y);  // conj(f_{n-k}), conj(f_{n-j})
      f[k] = make_float2((fk.x - (ef.x * ck.x - ef.y * ck.y)) * invD, (fk.y - (ef.x * ck.y + ef.y * ck.x)) * invD);
      if (j != k)
        f[j] = make_float2((fj.x - (ef.x * cj.x - ef.y * cj.y)) * invD, (fj.y - (ef.x * cj.y + ef.y * cj.x)) * invD);
    }
    // x' = [x; 0] + (y_n - ex) b', b'_j = conj(f'_{n-j}); the same for u
    const float2 mx = make_float2(y[n].x - ex.x, y[n].y - ex.y), mu = make_float2(g[n].x - eu.x, g[n].y - eu.y);
    x[n] = make_float2(0.f, 0.f);
    u[n] = make_float2(0.f, 0.f);
    for (uint32_t j = 0; j <= n; ++j) {
      const float2 b = make_float2(f[n - j].x, -f[n - j].y);
      x[j] = make_float2(x[j].x + mx.x * b.x - mx.y * b.y, x[j].y + mx.x * b.y + mx.y * b.x);
      u[j] = make_float2(u[j].x + mu.x * b.x - mu.y * b.y, u[j].y + mu.x * b.y + mu.y * b.x);
    }
  }
}

// The gradient step of pixelwise mode with W = (Sigma_theta + ridge I)^-1
// (Eq. 6): Sigma_theta = A - psi psi^H with A_jk = Psi(w_j - w_k) (Toeplitz,
// Psi(0) = 1) and psi_l = Psi_l the model at the current state, so v = W r
// comes from the Levinson solves A x = r, A u = psi and Sherman-Morrison,
// v = x + u (psi^H x) / (1 - psi^H u). The gradient is the W = I one with r
// replaced by v; the step sizes are the W = I bounds times alpha_0 + ridge
// (||W|| <= 1 / (alpha_0 + ridge) since Sigma_theta >= alpha_0 I).
template <int K>
__device__ __forceinline__ void grad_pixel_w(const float2* __restrict__ zp, uint32_t cnt, uint32_t T, uint32_t m,
                                             const float2* s_hh, float eta_t, float eta_a, float (&t)[K],
                                             float (&a)[K], const bool (&act)[K]) {
  const float Tf = float(T);
  float2 e1[K], E[K];
  float aa[K];
  float a0 = 1.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float sn, cs;
    sincospif(2.f * t[k] / Tf, &sn, &cs);
    e1[k] = make_float2(cs, sn);
    E[k] = e1[k];
    aa[k] = act[k] ? a[k] : 0.f;
    a0 -= aa[k];
  }
  float2 psi[kMaxM], r[kMaxM], f[kMaxM], x[kMaxM], u[kMaxM];
  for (uint32_t l = 0; l < m; ++l) {
    const float2 hv = s_hh[l];
    float2 ps = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float2 q = cmul(hv, E[k]);
      ps.x = fmaf(aa[k], q.x, ps.x);
      ps.y = fmaf(aa[k], q.y, ps.y);
      E[k] = cmul(E[k], e1[k]);
    }
    psi[l] = ps;
    const float2 zl = zp[l];
    r[l] = make_float2(zl.x - ps.x, zl.y - ps.y);
  }
  levinson2(1.f + kSigmaRidge, psi, m, r, psi, f, x, u);
  float2 px = make_float2(0.f, 0.f);
  float pu = 0.f;
  for (uint32_t l = 0; l < m; ++l) {
    px = make_float2(px.x + psi[l].x * x[l].x + psi[l].y * x[l].y, px.y + psi[l].x * x[l].y - psi[l].y * x[l].x);
    pu += psi[l].x * u[l].x + psi[l].y * u[l].y;
  }
  const float inv = 1.f / (1.f - pu);
  const float2 sm = make_float2(px.x * inv, px.y * inv);
  float gt[K], ga[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    gt[k] = ga[k] = 0.f;
    E[k] = e1[k];
  }
  const float wstep = 6.283185307179586f / Tf;
  for (uint32_t l = 0; l < m; ++l) {
    const float2 v = make_float2(x[l].x + u[l].x * sm.x - u[l].y * sm.y, x[l].y + u[l].x * sm.y + u[l].y * sm.x);
    const float2 hv = s_hh[l];
    const float w = wstep * float(l + 1);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float2 q = cmul(hv, E[k]);
      ga[k] += v.x * q.x + v.y * q.y;
      gt[k] += w * a[k] * (v.y * q.x - v.x * q.y);
      E[k] = cmul(E[k], e1[k]);
    }
  }
  const float scale = fmaxf(a0, 0.f) + kSigmaRidge;
  const float nn = -2.f * float(cnt);
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (act[k]) {
      float xk = t[k] - eta_t * scale * (nn * gt[k]);
      xk -= floorf(xk / Tf) * Tf;
      if (xk >= Tf) xk -= Tf;
      if (xk < 0.f) xk += Tf;
      t[k] = xk;
      a[k] = fmaxf(a[k] - eta_a * scale * (nn * ga[k]), 0.f);
    } else {
      a[k] = 0.f;
    }
    sum += a[k];
  }
  if (sum > 1.f) {
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = a[k] / sum;
  }
}

// Pixelwise iteration (regularize = 0): the gradient step is the new state.
// With `weighted`, W = (Sigma_theta + ridge I)^-1 instead of I.
template <int K, bool WEIGHTED>
__global__ void __launch_bounds__(kBlock) k_grad(const float2* __restrict__ z, const uint32_t* __restrict__ n,
                                                 uint32_t P, uint32_t T, uint32_t m,
                                                 const float2* __restrict__ hh_g, const float* __restrict__ misc,
                                                 float* depth, float* alpha, const uint8_t* active, float* alpha0) {
  __shared__ float2 s_hh[kMaxM];
  if (threadIdx.x < m) s_hh[threadIdx.x] = hh_g[threadIdx.x];
  __syncthreads();
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float nmax = float(max(reinterpret_cast<const unsigned*>(misc)[MISC_NMAX], 1u));
  float t[K], a[K];
  bool act[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    t[k] = depth[size_t(p) * K + k];
    a[k] = alpha[size_t(p) * K + k];
    act[k] = active[size_t(p) * K + k] != 0;
  }
  if (WEIGHTED)
    grad_pixel_w<K>(z + size_t(p) * m, n[p], T, m, s_hh, misc[MISC_ETA_T] / nmax, misc[MISC_ETA_A] / nmax, t, a,
                    act);
  else
    grad_pixel<K>(z + size_t(p) * m, n[p], T, m, s_hh, misc[MISC_ETA_T] / nmax, misc[MISC_ETA_A] / nmax, t, a,
                  act);
  float s2 = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    depth[size_t(p) * K + k] = t[k];
    alpha[size_t(p) * K + k] = a[k];
    s2 += a[k];
  }
  alpha0[p] = 1.f - s2;
}

struct Stencil {
  uint32_t rows, cols, radius;
  float h2, inv_h2, d_max, ds, lambda, prune_alpha;
};

// APSS weight (1 - d^2/h^2)^4 of a neighbour slot at pixel offset (dx, dy)
// and depth offset dt (bins), computed branch-free: 0 (and ok = false) for a
// slot that is not a neighbour (inactive, beyond d_max, or outside the
// support).
__device__ __forceinline__ float slot_weight(const Stencil& st, float dx, float dy, float dt, bool active,
                                             float& dz, bool& ok) {
  dz = dt * st.ds;
  const float d2 = dx * dx + dy * dy + dz * dz;
  const float u = 1.f - d2 * st.inv_h2;
  const float u2 = u * u;
  ok = active && fabsf(dt) <= st.d_max && d2 < st.h2;
  return ok ? u2 * u2 : 0.f;
}

// Unit normal from the weighted plane-fit moments (z = a + b x + c y).
__device__ __forceinline__ float4 plane_normal(int cnt, float Sw, float Sx, float Sy, float Sz, float Sxx, float Sxy,
                                               float Syy, float Sxz, float Syz) {
  const float det = Sw * (Sxx * Syy - Sxy * Sxy) - Sx * (Sx * Syy - Sxy * Sy) + Sy * (Sx * Sxy - Sxx * Sy);
  if (cnt >= 3 && det > 1e-6f * Sw * Sw * Sw) {
    const float db = Sw * (Sxz * Syy - Sxy * Syz) - Sz * (Sx * Syy - Sxy * Sy) + Sy * (Sx * Syz - Sxz * Sy);
    const float dcf = Sw * (Sxx * Syz - Sxz * Sxy) - Sx * (Sx * Syz - Sxz * Sy) + Sz * (Sx * Sxy - Sxx * Sy);
    const float idet = 1.f / det;
    const float b = db * idet, c = dcf * idet;
    const float inv = rsqrtf(b * b + c * c + 1.f);
    return make_float4(-b * inv, -c * inv, inv, 0.f);
  }
  return make_float4(0.f, 0.f, 1.f, 0.f);
}

// Depth after projecting onto the algebraic sphere fitted from the sums
// (Guennebaud & Gross 2007, with normals); tq when the fit is rejected.
__device__ __forceinline__ float sphere_depth(const Stencil& st, float tq, int cnt, float Sw, float Spx, float Spy,
                                              float Spz, float Snx, float Sny, float Snz, float Spn, float Spp) {
  const float iw = 1.f / Sw;  // (one division; the sums are scaled by its reciprocal)
  const float den = Spp - (Spx * Spx + Spy * Spy + Spz * Spz) * iw;
  if (cnt >= 3 && den > 0.f) {
    const float u4 = 0.5f * (Spn - (Spx * Snx + Spy * Sny + Spz * Snz) * iw) / den;
    const float ux = (Snx - 2.f * u4 * Spx) * iw;
    const float uy = (Sny - 2.f * u4 * Spy) * iw;
    const float uz = (Snz - 2.f * u4 * Spz) * iw;
    const float u0 = -(ux * Spx + uy * Spy + uz * Spz + u4 * Spp) * iw;
    const float disc = uz * uz - 4.f * u4 * u0;
    if (disc >= 0.f) {
      const float sq = sqrtf(disc);
      const float qq = -0.5f * (uz + (uz >= 0.f ? sq : -sq));
      if (qq != 0.f) {
        const float zn = u0 / qq;
        const float zf = (u4 != 0.f) ? qq / u4 : INFINITY;
        const float zs = (fabsf(zf) < fabsf(zn)) ? zf : zn;
        if (fabsf(zs) <= st.d_max * st.ds) return tq + zs / st.ds;
      }
    }
  }
  return tq;
}

// Calls f(dr, dc) for every offset of the (2R+1)^2 window, rows outer, as
// compile-time constants (std::integral_constant).
template <int R, typename F, int... I>
__device__ __forceinline__ void static_for_window_impl(F& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I / (2 * R + 1) - R>{}, std::integral_constant<int, I % (2 * R + 1) - R>{}), ...);
}

template <int R, typename F>
__device__ __forceinline__ void static_for_window(F& f) {
  static_for_window_impl<R>(f, std::make_integer_sequence<int, (2 * R + 1) * (2 * R + 1)>{});
}

// Depth stored for an inactive point in the masked copy: its offset to any
// depth in [0, T) exceeds every admissible d_max, so the neighbour test
// rejects it without a separate activity check, and its squared distance
// (depth_scale <= 1e3) stays finite, so a zero weight times it is zero.
constexpr float kMaskedDepth = 1e12f;

// The weights of the two points (K = 2) of one neighbour pixel at offset
// (dc, dr), as a packed pair: the same arithmetic as slot_weight.
template <int DR, int DC>
__device__ __forceinline__ float2 slot_weight_pair(const Stencil& st, float2 tm, float2 tq2, float2& dz, float2& d2,
                                                   int& cnt) {
  constexpr float c = float(DC * DC + DR * DR);
  const float2 dt = fsub2(tm, tq2);
  dz = fmul2(dt, make_float2(st.ds, st.ds));
  d2 = ffma2(dz, dz, make_float2(c, c));
  const float2 u = ffma2(d2, make_float2(-st.inv_h2, -st.inv_h2), make_float2(1.f, 1.f));
  const float2 u2 = fmul2(u, u);
  const float2 w4 = fmul2(u2, u2);
  const bool ok0 = fabsf(dt.x) <= st.d_max && d2.x < st.h2;
  const bool ok1 = fabsf(dt.y) <= st.d_max && d2.y < st.h2;
  cnt += int(ok0) + int(ok1);
  return make_float2(ok0 ? w4.x : 0.f, ok1 ? w4.y : 0.f);
}

// acc + D v for a compile-time integer D (exact for |D| <= 1; an FMA by D
// otherwise, as the scalar w * fx would round).
template <int D>
__device__ __forceinline__ float2 add_scaled(float2 acc, float2 v) {
  if constexpr (D == 0) return acc;
  if constexpr (D == 1) return fadd2(acc, v);
  if constexpr (D == -1) return fsub2(acc, v);
  return ffma2(v, make_float2(float(D), float(D)), acc);
}

// Plane-fit normal of point (lr, lc, k) of a K = 2 region from its
// (2R+1)^2 x 2 neighbour slots, the two points of a neighbour pixel packed.
template <int R>
__device__ __forceinline__ float4 normal_pair(const Stencil& st, const float (*s_tm)[2], int RW, int lr, int lc,
                                              float tq) {
  const float2 tq2 = make_float2(tq, tq);
  float2 Sw = make_float2(0.f, 0.f), Sx = Sw, Sy = Sw, Sz = Sw, Sxx = Sw, Sxy = Sw, Syy = Sw, Sxz = Sw, Syz = Sw;
  int cnt = 0;
  const auto slot = [&](auto dr_c, auto dc_c) {
    constexpr int DR = decltype(dr_c)::value, DC = decltype(dc_c)::value;
    const int q = (lr + DR) * RW + (lc + DC);
    const float2 tm = *reinterpret_cast<const float2*>(&s_tm[q][0]);
    float2 dz, d2;
    const float2 w = slot_weight_pair<DR, DC>(st, tm, tq2, dz, d2, cnt);
    const float2 wz = fmul2(w, dz);
    Sw = fadd2(Sw, w);
    Sz = fadd2(Sz, wz);
    Sx = add_scaled<DC>(Sx, w);
    Sy = add_scaled<DR>(Sy, w);
    Sxx = add_scaled<DC * DC>(Sxx, w);
    Syy = add_scaled<DR * DR>(Syy, w);
    Sxy = add_scaled<DC * DR>(Sxy, w);
    Sxz = add_scaled<DC>(Sxz, wz);
    Syz = add_scaled<DR>(Syz, wz);
  };
  static_for_window<R>(slot);
  return plane_normal(cnt, Sw.x + Sw.y, Sx.x + Sx.y, Sy.x + Sy.y, Sz.x + Sz.y, Sxx.x + Sxx.y, Sxy.x + Sxy.y,
                      Syy.x + Syy.y, Sxz.x + Sxz.y, Syz.x + Syz.y);
}

// Sphere projection and smoothed intensity of point (lr, lc) with depth tq
// and intensity aq of a K = 2 region (the two points of a neighbour pixel
// packed). Returns the new depth; *an = the smoothed intensity.
template <int R>
__device__ __forceinline__ float project_pair(const Stencil& st, const float (*s_tm)[2], const float (*s_a)[2],
                                              const float2* s_nx, const float2* s_ny, const float2* s_nz, int RW,
                                              int NW, int lr, int lc, float tq, float aq, float* an) {
  const float2 tq2 = make_float2(tq, tq);
  float2 Sw = make_float2(0.f, 0.f), Spx = Sw, Spy = Sw, Spz = Sw, Snx = Sw, Sny = Sw, Snz = Sw, Spn = Sw,
         Spp = Sw, Swa = Sw;
  int cnt = 0;
  const auto slot = [&](auto dr_c, auto dc_c) {
    constexpr int DR = decltype(dr_c)::value, DC = decltype(dc_c)::value;
    const int q = (lr + DR) * RW + (lc + DC);
    const int qn = (lr + DR - R) * NW + (lc + DC - R);
    const float2 tm = *reinterpret_cast<const float2*>(&s_tm[q][0]);
    float2 dz, d2;
    const float2 w = slot_weight_pair<DR, DC>(st, tm, tq2, dz, d2, cnt);
    const float2 nx = s_nx[qn], ny = s_ny[qn], nz = s_nz[qn];
    Sw = fadd2(Sw, w);
    Spx = add_scaled<DC>(Spx, w);
    Spy = add_scaled<DR>(Spy, w);
    Spz = ffma2(w, dz, Spz);
    Snx = ffma2(w, nx, Snx);
    Sny = ffma2(w, ny, Sny);
    Snz = ffma2(w, nz, Snz);
    const float2 pn = add_scaled<DR>(add_scaled<DC>(fmul2(dz, nz), nx), ny);
    Spn = ffma2(w, pn, Spn);
    Spp = ffma2(w, d2, Spp);
    Swa = ffma2(w, *reinterpret_cast<const float2*>(&s_a[q][0]), Swa);
  };
  static_for_window<R>(slot);
  const float sw = Sw.x + Sw.y;
  *an = (1.f - st.lambda) * aq + st.lambda * ((Swa.x + Swa.y) / sw);
  return sphere_depth(st, tq, cnt, sw, Spx.x + Spx.y, Spy.x + Spy.y, Spz.x + Spz.y, Snx.x + Snx.y, Sny.x + Sny.y,
                      Snz.x + Snz.y, Spn.x + Spn.y, Spp.x + Spp.y);
}

// One SRT3D iteration on a TW x TH tile, fused: the gradient step on the tile
// plus a 2R halo, plane-fit normals on the tile plus an R halo, then the
// sphere projection, intensity smoothing and pruning on the tile. The
// post-gradient state and the normals stay in shared memory; the state is
// read from and written to global memory once.
constexpr int kTW = 16, kTH = 16;

// One thread per pixel of the post-gradient region (tile + 2R halo), rounded
// up to whole warps, so that every stage runs in a single round.
template <int R>
__host__ __device__ constexpr int iter_threads() {
  return (((kTW + 4 * R) * (kTH + 4 * R) + 31) / 32) * 32;
}

// Threads of the persistent kernel: the halo is loaded, not computed, so a
// CTA needs one thread per pixel of the normals region (tile + R halo) at
// most; at radius 1 that is 288 (16x14 tiles), which lets 3 CTAs share an SM.
template <int R>
__host__ __device__ constexpr int persist_threads() {
  return R == 1 ? 288 : iter_threads<R>();
}

// Block of k_iter_persistent<K, R, MINB>: two points per pixel at radius 1
// with two CTAs per SM take one more warp (the registers allow it), whose
// threads, with those whose first point is inactive, compute the listed
// second points' normals in the first points' round.
template <int K, int R, int MINB>
__host__ __device__ constexpr int persist_block() {
  return (K == 2 && R == 1 && MINB == 2) ? 320 : persist_threads<R>();
}

// Shared memory of one tile: the post-gradient state of the region (tile +
// 2R halo) with a masked depth copy, and the normals of the tile + R halo
// (for K = 2 held as component pairs of the two points in the same storage).
template <int K, int R>
struct TileSmem {
  static constexpr int H = 2 * R;
  static constexpr int RW = kTW + 2 * H, RH = kTH + 2 * H;  // post-gradient region
  static constexpr int NW = kTW + 2 * R, NH = kTH + 2 * R;  // normals region
  alignas(16) float4 n[NH * NW][K];
  alignas(8) float t[RH * RW][K];
  alignas(8) float a[RH * RW][K];
  alignas(8) float tm[RH * RW][K];  // depth, or kMaskedDepth for an inactive point
  uint8_t act[RH * RW][K];
  float2 hh[kMaxM];
  // K = 2: the second points (active in ~13 % of the pixels of a typical
  // frame) are processed from compact lists instead of as a masked second
  // pass of every thread: positions whose second normal is needed, own
  // pixels whose second point is projected, and the projections' results
  int n_list, p_list, n_take;
  uint16_t nlist[NH * NW];
  uint16_t plist[kTW * kTH];
  float2 pres[kTW * kTH];
  __device__ float2* nx() { return reinterpret_cast<float2*>(&n[0][0]); }
  __device__ float2* ny() { return nx() + NH * NW; }
  __device__ float2* nz() { return ny() + NH * NW; }
};

// Empties the second-point lists of the normals and projection stages (one
// thread, before a barrier that precedes stage 2).
template <int K, int R>
__device__ __forceinline__ void reset_lists(TileSmem<K, R>& sm) {
  sm.n_list = 0;
  sm.p_list = 0;
  sm.n_take = 0;
}

// Region index of the j-th halo pixel of a tile th rows high (top band, side
// columns, bottom band).
template <int R>
__device__ __forceinline__ int halo_index(int j, int th) {
  constexpr int H = 2 * R, RW = kTW + 2 * H;
  if (j < H * RW) return j;
  j -= H * RW;
  if (j < th * 2 * H) {
    const int c = j % (2 * H);
    return (H + j / (2 * H)) * RW + (c < H ? c : c + kTW);
  }
  return (H + th) * RW + (j - th * 2 * H);
}

// The state (t, a, act) of pixel p. L2-coherent loads: inside the
// persistent kernel the buffers are rewritten by other CTAs.
template <int K>
__device__ __forceinline__ void load_state(const float* depth, const float* alpha, const uint8_t* active, size_t p,
                                           float (&t)[K], float (&a)[K], bool (&act)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    t[k] = __ldcg(depth + p * K + k);
    a[k] = __ldcg(alpha + p * K + k);
    act[k] = __ldcg(active + p * K + k) != 0;
  }
}

// Gradient step of region pixel i (at array row rr, column cc; `in` = inside
// the array, else inactive) from the state (t, a, act); the post-step state
// goes to shared memory and stays in (t, a, act). The pixel's sketch comes
// from s_z / s_nn (entry zi) when given, else from global memory.
template <int K, int R>
__device__ __forceinline__ void grad_to_smem(TileSmem<K, R>& sm, const Stencil& st, int i, int rr, int cc, bool in,
                                             float (&t)[K], float (&a)[K], bool (&act)[K],
                                             const float2* __restrict__ z, const uint32_t* __restrict__ n, uint32_t T,
                                             uint32_t m, float eta_t, float eta_a, const float2* s_z,
                                             const uint32_t* s_nn, int zi = 0) {
  if (in) {
    if (s_z)
      grad_pixel<K>(s_z + size_t(zi) * m, s_nn[zi], T, m, sm.hh, eta_t, eta_a, t, a, act);
    else {
      const size_t p = size_t(rr) * st.cols + size_t(cc);
      grad_pixel<K>(z + p * m, n[p], T, m, sm.hh, eta_t, eta_a, t, a, act);
    }
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      t[k] = 0.f;
      a[k] = 0.f;
      act[k] = false;
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    sm.t[i][k] = t[k];
    sm.a[i][k] = a[k];
    sm.act[i][k] = act[k] ? 1 : 0;
    sm.tm[i][k] = act[k] ? t[k] : kMaskedDepth;
  }
}

// A region pixel's post-gradient state into shared memory.
template <int K, int R>
__device__ __forceinline__ void put_state(TileSmem<K, R>& sm, int i, const float (&t)[K], const float (&a)[K],
                                          const bool (&act)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    sm.t[i][k] = t[k];
    sm.a[i][k] = a[k];
    sm.act[i][k] = act[k] ? 1 : 0;
    sm.tm[i][k] = act[k] ? t[k] : kMaskedDepth;
  }
}

// Stage 1 for region pixel i, its state read from global memory.
template <int K, int R>
__device__ __forceinline__ void stage1_pixel(TileSmem<K, R>& sm, const Stencil& st, int i, int r0, int c0,
                                             const float2* __restrict__ z, const uint32_t* __restrict__ n, uint32_t T,
                                             uint32_t m, float eta_t, float eta_a, const float* depth_in,
                                             const float* alpha_in, const uint8_t* active_in, const float2* s_z,
                                             const uint32_t* s_nn) {
  constexpr int H = TileSmem<K, R>::H, RW = TileSmem<K, R>::RW;
  const int rr = r0 - H + i / RW, cc = c0 - H + i % RW;
  const bool in = rr >= 0 && rr < int(st.rows) && cc >= 0 && cc < int(st.cols);
  float t[K], a[K];
  bool act[K];
  if (in) load_state<K>(depth_in, alpha_in, active_in, size_t(rr) * st.cols + size_t(cc), t, a, act);
  grad_to_smem<K, R>(sm, st, i, rr, cc, in, t, a, act, z, n, T, m, eta_t, eta_a, s_z, s_nn);
}

// Stage 2: normals of the tile (th rows) plus an R halo, NT threads.
// PRE (K = 2): the second points' positions (sm.nlist) and the tile's own
// second points (sm.plist) were listed before the stage; every thread takes
// list items once its first point is done (threads without a first point,
// or with an inactive one, first), so a short list needs no round of its own.
template <int K, int R, int NT, bool PRE = false>
__device__ __forceinline__ void stage2(TileSmem<K, R>& sm, const Stencil& st, int th) {
  constexpr int RW = TileSmem<K, R>::RW, NW = TileSmem<K, R>::NW;
  const int NH = th + 2 * R;
  const int tid = threadIdx.x;
  if constexpr (K == 2 && PRE) {
    float2* s_nx = sm.nx();
    float2* s_ny = sm.ny();
    float2* s_nz = sm.nz();
    for (int i = tid; i < NH * NW; i += NT) {
      const int lr = i / NW + R, lc = i % NW + R;
      const int q0 = lr * RW + lc;
      const float4 nv = sm.act[q0][0] ? normal_pair<R>(st, sm.tm, RW, lr, lc, sm.t[q0][0])
                                      : make_float4(0.f, 0.f, 1.f, 0.f);
      s_nx[i].x = nv.x;
      s_ny[i].x = nv.y;
      s_nz[i].x = nv.z;
      if (!sm.act[q0][1]) {  // (a listed item writes these words otherwise)
        s_nx[i].y = 0.f;
        s_ny[i].y = 0.f;
        s_nz[i].y = 1.f;
      }
    }
    const int cnt = sm.n_list;
    for (;;) {
      const int j = atomicAdd(&sm.n_take, 1);
      if (j >= cnt) break;
      const int i = sm.nlist[j];
      const int lr = i / NW + R, lc = i % NW + R;
      const float4 nv = normal_pair<R>(st, sm.tm, RW, lr, lc, sm.t[lr * RW + lc][1]);
      s_nx[i].y = nv.x;
      s_ny[i].y = nv.y;
      s_nz[i].y = nv.z;
    }
  } else if constexpr (K == 2) {
    float2* s_nx = sm.nx();
    float2* s_ny = sm.ny();
    float2* s_nz = sm.nz();
    // first points by every thread, second points from a compact list
    // (sm.n_list was zeroed before the barrier that precedes this stage);
    // the tile's own second points are listed for stage 3 as well
    constexpr int H = TileSmem<K, R>::H;
    for (int i = tid; i < NH * NW; i += NT) {
      const int lr = i / NW + R, lc = i % NW + R;
      const int q0 = lr * RW + lc;
      const float4 nv = sm.act[q0][0] ? normal_pair<R>(st, sm.tm, RW, lr, lc, sm.t[q0][0])
                                      : make_float4(0.f, 0.f, 1.f, 0.f);
      s_nx[i] = make_float2(nv.x, 0.f);
      s_ny[i] = make_float2(nv.y, 0.f);
      s_nz[i] = make_float2(nv.z, 1.f);
      if (sm.act[q0][1]) {
        sm.nlist[atomicAdd(&sm.n_list, 1)] = uint16_t(i);
        if (lr >= H && lr < H + th && lc >= H && lc < H + kTW)
          sm.plist[atomicAdd(&sm.p_list, 1)] = uint16_t((lr - H) * kTW + (lc - H));
      }
    }
    __syncthreads();
    const int cnt = sm.n_list;
    for (int j = tid; j < cnt; j += NT) {
      const int i = sm.nlist[j];
      const int lr = i / NW + R, lc = i % NW + R;
      const float4 nv = normal_pair<R>(st, sm.tm, RW, lr, lc, sm.t[lr * RW + lc][1]);
      s_nx[i].y = nv.x;
      s_ny[i].y = nv.y;
      s_nz[i].y = nv.z;
    }
  } else {
    for (int i = tid; i < NH * NW; i += NT) {
      const int lr = i / NW + R, lc = i % NW + R;  // region coordinates
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float4 nv = make_float4(0.f, 0.f, 1.f, 0.f);
        const int q0 = lr * RW + lc;
        if (sm.act[q0][k]) {
          const float tq = sm.t[q0][k];
          float Sw = 0, Sx = 0, Sy = 0, Sz = 0, Sxx = 0, Sxy = 0, Syy = 0, Sxz = 0, Syz = 0;
          int cnt = 0;
          // branch-free: every slot is loaded and weighted (0 for non-neighbours),
          // which leaves the sums exactly as if the slot were skipped
#pragma unroll(K <= 2 ? 2 * R + 1 : 1)
          for (int dr = -R; dr <= R; ++dr)
#pragma unroll
            for (int dc = -R; dc <= R; ++dc) {
              const int q = (lr + dr) * RW + (lc + dc);
#pragma unroll
              for (int k2 = 0; k2 < K; ++k2) {
                const float fx = float(dc), fy = float(dr);
                float dz;
                bool ok;
                const float w = slot_weight(st, fx, fy, sm.t[q][k2] - tq, sm.act[q][k2] != 0, dz, ok);
                cnt += ok ? 1 : 0;
                Sw += w;
                Sx += w * fx;
                Sy += w * fy;
                Sz += w * dz;
                Sxx += w * fx * fx;
                Sxy += w * fx * fy;
                Syy += w * fy * fy;
                Sxz += w * fx * dz;
                Syz += w * fy * dz;
              }
            }
          nv = plane_normal(cnt, Sw, Sx, Sy, Sz, Sxx, Sxy, Syy, Sxz, Syz);
        }
        sm.n[i][k] = nv;
      }
    }
  }
}

// Stage 3: sphere projection, smoothing and pruning of tile pixel tid (tile
// origin r0, c0, th rows). Returns whether the thread owns an in-array tile
// pixel; its new state is then in (tout, aout, aact) and written to global
// memory.
// Must be called by every thread of the CTA (for K = 2 it passes barriers).
template <int K, int R>
__device__ __forceinline__ bool stage3(TileSmem<K, R>& sm, const Stencil& st, int r0, int c0, int th, float* depth,
                                       float* alpha, uint8_t* active, float* alpha0, float (&tout)[K],
                                       float (&aout)[K], bool (&aact)[K], bool store = true) {
  constexpr int H = TileSmem<K, R>::H, RW = TileSmem<K, R>::RW, NW = TileSmem<K, R>::NW;
  const int tid = threadIdx.x;
  const int ty = tid / kTW, tx = tid % kTW;
  const int rr = r0 + ty, cc = c0 + tx;
  const bool own = tid < kTW * th && rr < int(st.rows) && cc < int(st.cols);
  const int lr = ty + H, lc = tx + H;
  const int q0 = lr * RW + lc;
  if constexpr (K == 2) {
    // first points by their owners; in the same round the second points that
    // stage 2 listed, by the threads without a tile pixel (all threads, in a
    // round of their own, if the block has none)
    const auto second = [&](int j) {
      const int o = sm.plist[j];
      const int olr = o / kTW + H, olc = o % kTW + H, oq = olr * RW + olc;
      float an;
      const float tn = project_pair<R>(st, sm.tm, sm.a, sm.nx(), sm.ny(), sm.nz(), RW, NW, olr, olc, sm.t[oq][1],
                                       sm.a[oq][1], &an);
      sm.pres[o] = make_float2(tn, an);
    };
    const int cnt = sm.p_list;
    const int npx = kTW * th, spare = int(blockDim.x) - npx;
    if (own) {
      const float tq = sm.t[q0][0];
      tout[0] = tq;
      aout[0] = 0.f;
      aact[0] = false;
      if (sm.act[q0][0]) {
        float an;
        tout[0] = project_pair<R>(st, sm.tm, sm.a, sm.nx(), sm.ny(), sm.nz(), RW, NW, lr, lc, tq, sm.a[q0][0],
                                  &an);
        aact[0] = an >= st.prune_alpha;
        aout[0] = aact[0] ? an : 0.f;
      }
    }
    if (spare > 0) {
      if (tid >= npx)
        for (int j = tid - npx; j < cnt; j += spare) second(j);
    } else {
      __syncthreads();
      for (int j = tid; j < cnt; j += blockDim.x) second(j);
    }
    __syncthreads();
    if (!own) return false;
    tout[1] = sm.t[q0][1];
    aout[1] = 0.f;
    aact[1] = false;
    if (sm.act[q0][1]) {
      const float2 res = sm.pres[tid];
      tout[1] = res.x;
      aact[1] = res.y >= st.prune_alpha;
      aout[1] = aact[1] ? res.y : 0.f;
    }
  } else {
    if (!own) return false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float tq = sm.t[q0][k];
      tout[k] = tq;
      aout[k] = 0.f;
      aact[k] = false;
      if (!sm.act[q0][k]) continue;
      float Sw = 0, Spx = 0, Spy = 0, Spz = 0, Snx = 0, Sny = 0, Snz = 0, Spn = 0, Spp = 0, Swa = 0;
      int cnt = 0;
#pragma unroll(K <= 2 ? 2 * R + 1 : 1)
      for (int dr = -R; dr <= R; ++dr)
#pragma unroll
        for (int dc = -R; dc <= R; ++dc) {
          const int q = (lr + dr) * RW + (lc + dc);
          const int qn = (lr + dr - R) * NW + (lc + dc - R);
#pragma unroll
          for (int k2 = 0; k2 < K; ++k2) {
            const float fx = float(dc), fy = float(dr);
            float dz;
            bool ok;
            const float w = slot_weight(st, fx, fy, sm.t[q][k2] - tq, sm.act[q][k2] != 0, dz, ok);
            cnt += ok ? 1 : 0;
            const float4 nv = sm.n[qn][k2];
            Sw += w;
            Spx += w * fx;
            Spy += w * fy;
            Spz += w * dz;
            Snx += w * nv.x;
            Sny += w * nv.y;
            Snz += w * nv.z;
            Spn += w * (fx * nv.x + fy * nv.y + dz * nv.z);
            Spp += w * (fx * fx + fy * fy + dz * dz);
            Swa += w * sm.a[q][k2];
          }
        }
      tout[k] = sphere_depth(st, tq, cnt, Sw, Spx, Spy, Spz, Snx, Sny, Snz, Spn, Spp);
      const float an = (1.f - st.lambda) * sm.a[q0][k] + st.lambda * (Swa / Sw);
      aact[k] = an >= st.prune_alpha;
      aout[k] = aact[k] ? an : 0.f;
    }
  }
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) sum += aout[k];
  if (sum > 1.f) {
#pragma unroll
    for (int k = 0; k < K; ++k) aout[k] = aout[k] / sum;
    sum = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) sum += aout[k];
  }
  if (store) {
    const size_t p = size_t(rr) * st.cols + size_t(cc);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      depth[p * K + k] = tout[k];
      alpha[p * K + k] = aout[k];
      active[p * K + k] = aact[k] ? 1 : 0;
    }
    alpha0[p] = 1.f - sum;
  }
  return true;
}

template <int K, int R>
__device__ __forceinline__ void iter_tile(const Stencil st, uint32_t tile_x, uint32_t tile_y,
                                          const float2* __restrict__ z, const uint32_t* __restrict__ n, uint32_t T,
                                          uint32_t m, const float2* __restrict__ hh_g,
                                          const float* __restrict__ misc, const float* depth_in,
                                          const float* alpha_in, const uint8_t* active_in, float* depth,
                                          float* alpha, uint8_t* active, float* alpha0) {
  __shared__ TileSmem<K, R> sm;
  constexpr int NT = iter_threads<R>();
  constexpr int RW = TileSmem<K, R>::RW, RH = TileSmem<K, R>::RH;
  const int tid = threadIdx.x;
  if (tid < int(m)) sm.hh[tid] = hh_g[tid];
  __syncthreads();
  const int r0 = int(tile_y) * kTH, c0 = int(tile_x) * kTW;
  const float nmax = float(max(reinterpret_cast<const unsigned*>(misc)[MISC_NMAX], 1u));
  const float eta_t = misc[MISC_ETA_T] / nmax, eta_a = misc[MISC_ETA_A] / nmax;
  // 1) gradient step on the region (pixels outside the array are inactive)
  for (int i = tid; i < RH * RW; i += NT)
    stage1_pixel<K, R>(sm, st, i, r0, c0, z, n, T, m, eta_t, eta_a, depth_in, alpha_in, active_in, nullptr,
                       nullptr);
  if (tid == 0) reset_lists(sm);
  __syncthreads();
  // 2) normals on the tile plus an R halo
  stage2<K, R, NT>(sm, st, kTH);
  __syncthreads();
  // 3) sphere projection, smoothing and pruning on the tile
  float tout[K], aout[K];
  bool aact[K];
  stage3<K, R>(sm, st, r0, c0, kTH, depth, alpha, active, alpha0, tout, aout, aact);
}

// The state is read from (depth_in, alpha_in, active_in) and written to
// (depth, alpha, active): distinct buffers, since neighbouring tiles read
// each other's state as their halo within the same launch.
template <int K, int R>
__global__ void __launch_bounds__(iter_threads<R>()) k_iter(Stencil st, const float2* __restrict__ z,
                                                            const uint32_t* __restrict__ n, uint32_t T, uint32_t m,
                                                            const float2* __restrict__ hh_g,
                                                            const float* __restrict__ misc,
                                                            const float* __restrict__ depth_in,
                                                            const float* __restrict__ alpha_in,
                                                            const uint8_t* __restrict__ active_in, float* depth,
                                                            float* alpha, uint8_t* active, float* alpha0) {
  iter_tile<K, R>(st, blockIdx.x, blockIdx.y, z, n, T, m, hh_g, misc, depth_in, alpha_in, active_in, depth, alpha,
                  active, alpha0);
}

constexpr long long kGridWaitCycles = 2000000000ll;  // ~1 s at 2 GHz
constexpr long long kInjectedWaitCycles = 100000ll;  // ~50 us: fault injection only

// Neighbour synchronisation of the persistent kernel. Each tile has a
// progress flag in global memory (zeroed by k_prep; one 32-byte sector per
// flag, see kTileFlagStride): after the CTA has
// published its post-gradient state of iteration it, it stores it + 1 to its
// flag (release); before it reads its halo of iteration it, it waits until
// the flag of every tile its halo touches is >= it + 1 (acquire). Only the
// tiles within reach are waited for, not the whole grid, and the lanes of
// warp 0 poll them in parallel (one L2 round trip per poll round). The wait is
// bounded like the grid barrier's.
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Tagged exchange words: a 32-bit value in the low half and the iteration's
// tag in the high half of one aligned 64-bit word, which is written and read
// as a single access (single-copy atomic), so a reader that sees the tag sees
// the value written with it: no flag and no fence between the data and its
// readiness. A point (p, k) takes two words, its post-gradient depth and its
// intensity (-1 for an inactive point). Reuse of a buffer needs no fence
// either: a CTA rewrites the buffer of parity it & 1 at iteration it + 2 only
// after its halo loads of iteration it + 1 returned every neighbour's words
// of it + 1, which each neighbour issues after the barrier that follows its
// own halo loads of iteration it; those loads had returned (their values are
// in shared memory) before that barrier, so none can see the rewrite. (Fences
// on both sides cost 11 % of the iteration launch; they are not needed for
// this order.)
__device__ __forceinline__ void st_tagged2(unsigned long long* w, float t, float a, unsigned tag) {
  const unsigned long long hi = static_cast<unsigned long long>(tag) << 32;
  const unsigned long long w0 = hi | __float_as_uint(t), w1 = hi | __float_as_uint(a);
  asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(w), "l"(w0), "l"(w1) : "memory");
}

__device__ __forceinline__ void ld_tagged2(const unsigned long long* w, unsigned long long& w0,
                                           unsigned long long& w1) {
  asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(w0), "=l"(w1) : "l"(w) : "memory");
}

// The state of halo pixel p from the tagged buffer once both words of each
// of its K points carry `tag`. Returns false when that takes longer than
// `limit` cycles (the pixel's state is then left inactive).
template <int K>
__device__ __forceinline__ bool load_state_tagged(const unsigned long long* xt, size_t p, unsigned tag,
                                                  long long limit, float (&t)[K], float (&a)[K], bool (&act)[K]) {
  unsigned long long w[K][2];
  const long long t0 = clock64();
  for (;;) {
    bool ready = true;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      ld_tagged2(xt + (p * K + k) * 2, w[k][0], w[k][1]);
      ready = ready && unsigned(w[k][0] >> 32) == tag && unsigned(w[k][1] >> 32) == tag;
    }
    if (ready) break;
    if (clock64() - t0 > limit) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        t[k] = 0.f;
        a[k] = 0.f;
        act[k] = false;
      }
      return false;
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    t[k] = __uint_as_float(unsigned(w[k][0]));
    const float ae = __uint_as_float(unsigned(w[k][1]));
    act[k] = ae >= 0.f;
    a[k] = act[k] ? ae : 0.f;
  }
  return true;
}

__device__ __forceinline__ void tile_publish(unsigned* flags, uint32_t tile, unsigned value) {
  __syncthreads();  // every thread's state of this iteration is written
  // The barrier orders the CTA's writes before thread 0's release store, and
  // release is cumulative at gpu scope: a CTA whose acquire load reads the
  // flag sees them (no separate fence; 2 % faster per launch).
  if (threadIdx.x == 0) st_release(flags + tile * kTileFlagStride, value);
}

// Waits for the tiles (tx + dx, ty + dy), |dx| <= 1, |dy| <= reach_y, to reach
// `target`. Returns false (after latching FLAG_DEVICE_TIMEOUT) when a wait
// exceeds `limit` cycles.
__device__ __forceinline__ bool tile_wait(const unsigned* flags, int tx, int ty, int tiles_x, int tiles_y,
                                          int reach_y, unsigned target, uint32_t* err, int* s_abort,
                                          long long limit) {
  if (threadIdx.x < 32) {
    const int lane = int(threadIdx.x);
    const int dy = lane / 3 - reach_y, dx = lane % 3 - 1;
    const int x = tx + dx, y = ty + dy;
    const bool mine = lane < 3 * (2 * reach_y + 1) && x >= 0 && x < tiles_x && y >= 0 && y < tiles_y;
    bool ok = true;
    if (mine) {
      const unsigned* f = flags + (y * tiles_x + x) * int(kTileFlagStride);
      const long long t0 = clock64();
      while (ld_acquire(f) < target) {
        if (clock64() - t0 > limit) {
          ok = false;
          break;
        }
        __nanosleep(32);
      }
    }
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0 && !ok) {
      *s_abort = 1;
      atomicOr(err, FLAG_DEVICE_TIMEOUT);
    }
  }
  __syncthreads();
  return *s_abort == 0;
}

// Diagnostic: the persistent kernel's bounded wait on a progress flag that
// nothing raises, with a short limit (see srt3d_selftest_wait_timeout).
__device__ unsigned g_selftest_flag = 0u;

__global__ void k_selftest_wait(uint32_t* flags, long long limit) {
  __shared__ int s_abort;
  if (threadIdx.x == 0) s_abort = 0;
  __syncthreads();
  tile_wait(&g_selftest_flag, 0, 0, 1, 1, 0, 1u, flags, &s_abort, limit);
}

// Post-gradient state of every point, exchanged between the CTAs of the
// persistent kernel (structure of arrays, [P][K]).
struct XBuf {
  float* t;
  float* a;
  uint8_t* c;
};

// All iterations in one cooperative launch, one CTA per kTW x th tile (th <=
// kTH, chosen by the launcher to balance the tiles over the SMs); the tile's
// sketches and counts are loaded into shared memory once. Per iteration a
// CTA takes the gradient step of its own pixels (pixelwise, from the state it
// produced last iteration or the initial state), publishes the post-gradient
// state to one of two exchange buffers, reads the halo's post-gradient state
// from the buffer once it is there, and runs the normals and the projection
// stages. With `xtag` (the scratch block holds the tagged buffers) every word
// carries its iteration's tag and the halo loads themselves wait for it (a
// reader waits only for the words it needs, and no flag, fence or extra
// barrier sits between a neighbour's store and the load: 13 % faster than
// flags); without, the tile raises a progress flag (release store, one flag
// per 32-byte sector) and waits for the flags of the tiles its halo touches
// before loading. (Overlapping the interior's stages with the wait was
// slower, since splitting a latency-bound stage in two doubles its latency.)
// The buffers alternate by iteration: a tile rewrites buffer it & 1 at
// iteration it + 2 only after its halo of iteration it + 1 was complete,
// i.e. after every tile within reach published iteration it + 1, which each
// does only after reading its halo of iteration it from that buffer. The
// final state goes to the caller's buffers during the last iteration.
// MINB: co-resident CTAs per SM the registers are held to. At radius 1 the
// kernel exists for 3 (more tiles fit at once) and for 2 (more registers, no
// spills: used when the frame's tiles fit two per SM).
template <int K, int R, int MINB>
__global__ void __launch_bounds__(persist_block<K, R, MINB>(), MINB) k_iter_persistent(
    Stencil st, const float2* __restrict__ z, const uint32_t* __restrict__ n, uint32_t T, uint32_t m,
    const float2* __restrict__ hh_g, float* __restrict__ misc, float* depth, float* alpha, uint8_t* active,
    float* alpha0, XBuf x0, XBuf x1, uint32_t iters, uint32_t tiles_x, uint32_t th_u, uint32_t* __restrict__ flags,
    unsigned* tile_flags, uint32_t flag_base, uint32_t bar_skew, long long wait_limit,
    unsigned long long* __restrict__ xtag) {
  using S = TileSmem<K, R>;
  constexpr int H = S::H, RW = S::RW, NW = S::NW;
  constexpr int NT = persist_block<K, R, MINB>();
  constexpr bool PRE = K == 2;  // second points listed before the normals stage
  const int th = int(th_u), RH = th + 2 * H, halo = RH * RW - kTW * th, npx = kTW * th;
  __shared__ S sm;
  __shared__ int s_abort;
  extern __shared__ float2 s_z[];  // [kTW * kTH][m] sketches of the tile's pixels, then [kTW * kTH] counts
  uint32_t* s_nn = reinterpret_cast<uint32_t*>(s_z + size_t(kTW) * kTH * m);
  const int tid = threadIdx.x;
  const uint32_t tile_x = blockIdx.x % tiles_x, tile_y = blockIdx.x / tiles_x;
  const int r0 = int(tile_y) * th, c0 = int(tile_x) * kTW;
  for (uint32_t i = tid; i < uint32_t(npx) * m; i += NT) {
    const uint32_t q = i / m, l = i - q * m;
    const int rr = r0 + int(q) / kTW, cc = c0 + int(q) % kTW;
    const bool in = rr < int(st.rows) && cc < int(st.cols);
    s_z[i] = in ? z[(size_t(rr) * st.cols + size_t(cc)) * m + l] : make_float2(0.f, 0.f);
  }
  for (int q = tid; q < npx; q += NT) {
    const int rr = r0 + q / kTW, cc = c0 + q % kTW;
    s_nn[q] = rr < int(st.rows) && cc < int(st.cols) ? n[size_t(rr) * st.cols + size_t(cc)] : 0u;
  }
  if (tid < int(m)) sm.hh[tid] = hh_g[tid];
  if (tid == 0) {
    s_abort = 0;
    reset_lists(sm);
  }
  __syncthreads();
  const float nmax = float(max(reinterpret_cast<const unsigned*>(misc)[MISC_NMAX], 1u));
  const float eta_t = misc[MISC_ETA_T] / nmax, eta_a = misc[MISC_ETA_A] / nmax;
  const int tiles_y = int(gridDim.x / tiles_x);
  const int reach_y = (H + th - 1) / th;  // tile rows the 2R halo reaches
  // the thread's own pixel (tid < npx) and its state between iterations
  const int ty = tid / kTW, tx = tid % kTW;
  const int rr = r0 + ty, cc = c0 + tx;
  const bool mine = tid < npx;
  const bool in = mine && rr < int(st.rows) && cc < int(st.cols);
  const size_t p = in ? size_t(rr) * st.cols + size_t(cc) : 0;
  float t[K], a[K];
  bool act[K];
  if (in) load_state<K>(depth, alpha, active, p, t, a, act);
  const size_t xwords = size_t(st.rows) * st.cols * K * 2;  // one tagged buffer
  for (uint32_t it = 0; it < iters; ++it) {
    const XBuf xb = (it & 1u) ? x1 : x0;
    unsigned long long* xt = xtag ? xtag + (it & 1u) * xwords : nullptr;
    const unsigned tag = flag_base + it + 1u;
    const bool last = it + 1u == iters;
    // 1) gradient step of the own pixel, published for the neighbours
    if (mine) {
      grad_to_smem<K, R>(sm, st, (ty + H) * RW + (tx + H), rr, cc, in, t, a, act, z, n, T, m, eta_t, eta_a, s_z,
                         s_nn, tid);
      if constexpr (PRE) {
        if (act[K - 1]) {
          sm.nlist[atomicAdd(&sm.n_list, 1)] = uint16_t((ty + R) * NW + tx + R);
          sm.plist[atomicAdd(&sm.p_list, 1)] = uint16_t(tid);
        }
      }
      if (in) {
        if (xt) {
#pragma unroll
          for (int k = 0; k < K; ++k) st_tagged2(xt + (p * K + k) * 2, t[k], act[k] ? a[k] : -1.f, tag);
        } else {
#pragma unroll
          for (int k = 0; k < K; ++k) {
            xb.t[p * K + k] = t[k];
            xb.a[p * K + k] = a[k];
            xb.c[p * K + k] = act[k] ? 1 : 0;
          }
        }
      }
    }
    if (!xt) {
      tile_publish(tile_flags, blockIdx.x, flag_base + it + 1u);
      if (!tile_wait(tile_flags, int(tile_x), int(tile_y), int(tiles_x), tiles_y, reach_y,
                     flag_base + it + 1u + bar_skew, flags, &s_abort, wait_limit))
        break;
    }
    // 2) the halo's post-gradient state (tagged: each word read once it
    // carries this iteration's tag)
    for (int j = tid; j < halo; j += NT) {
      const int i = halo_index<R>(j, th);
      const int hr = r0 - H + i / RW, hc = c0 - H + i % RW;
      float ht[K], ha[K];
      bool hact[K];
      if (hr >= 0 && hr < int(st.rows) && hc >= 0 && hc < int(st.cols)) {
        const size_t hp = size_t(hr) * st.cols + size_t(hc);
        if (xt) {
          if (!load_state_tagged<K>(xt, hp, tag + bar_skew, wait_limit, ht, ha, hact)) {
            s_abort = 1;
            atomicOr(flags, FLAG_DEVICE_TIMEOUT);
          }
        } else {
          load_state<K>(xb.t, xb.a, xb.c, hp, ht, ha, hact);
        }
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          ht[k] = 0.f;
          ha[k] = 0.f;
          hact[k] = false;
        }
      }
      put_state<K, R>(sm, i, ht, ha, hact);
      if constexpr (PRE) {
        const int lr = i / RW, lc = i % RW;  // listed when in the normals region
        if (hact[K - 1] && lr >= R && lr < th + 3 * R && lc >= R && lc < kTW + 3 * R)
          sm.nlist[atomicAdd(&sm.n_list, 1)] = uint16_t((lr - R) * NW + lc - R);
      }
    }
    if (!PRE && tid == 0) reset_lists(sm);
    __syncthreads();
    if (s_abort) break;
    // 3) normals, 4) projection, smoothing and pruning
    stage2<K, R, NT, PRE>(sm, st, th);
    __syncthreads();
    float tout[K], aout[K];
    bool aact[K];
    if (stage3<K, R>(sm, st, r0, c0, th, depth, alpha, active, alpha0, tout, aout, aact, last)) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        t[k] = tout[k];
        a[k] = aout[k];
        act[k] = aact[k];
      }
    }
    if (PRE && tid == 0) reset_lists(sm);  // read above, before stage 3's barrier
    __syncthreads();  // the next gradient step rewrites the tile's shared state (and lists)
  }
}

// All iterations of every frame of a batch in one cooperative launch. The
// batch's tiles (16 x th pixels of any frame, numbered frame after frame) are
// shared out round-robin over the CTAs, so a CTA owns many tiles and keeps
// their state in global memory: the frames' own depth/alpha/active buffers,
// updated in place. Per iteration, phase 1 takes the gradient step of every
// own tile and publishes its post-gradient state to the frame's exchange
// words of this iteration's parity, tagged with the iteration (as in
// k_iter_persistent); phase 2, for every own tile, loads the post-gradient
// state of tile + halo, each load waiting (bounded) for its words' tag, and
// runs the normals and the projection stages, writing the tile's new state.
// Phase 1 never waits, and a phase-2 wait is on tiles' phase 1 of the same
// iteration, which the CTA that is furthest behind can always complete, so
// the launch cannot deadlock. A tile rewrites the words of parity it & 1 in
// phase 1 of it + 2 only after its phase-2 loads of it + 1 returned every
// tile within reach past phase 1 of it + 1, i.e. past its phase-2 reads of
// iteration it. The words are zeroed before the launch (tag 0 is no
// iteration's).
template <int K, int R>
__global__ void __launch_bounds__(persist_threads<R>(), R == 1 ? 3 : 1) k_iter_batch_persistent(
    Stencil base, const BatchFrame* __restrict__ frames, uint32_t nframes, uint32_t total_tiles, uint32_t th_u,
    uint32_t iters, unsigned* tile_flags, uint32_t* __restrict__ err) {
  using S = TileSmem<K, R>;
  constexpr int H = S::H, RW = S::RW;
  constexpr int NT = persist_threads<R>();
  const int th = int(th_u), RH = th + 2 * H, npx = kTW * th;
  (void)tile_flags;  // (the exchange words carry their own tags)
  __shared__ S sm;
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  if (tid == 0) s_abort = 0;
  const int ty = tid / kTW, tx = tid % kTW;
  uint32_t cur = 0xffffffffu;  // frame whose hhat is in shared memory
  for (uint32_t it = 0; it < iters; ++it) {
    // phase 1: gradient steps, published
    for (uint32_t tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
      uint32_t lo = 0, hi = nframes - 1;
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) / 2;
        if (frames[mid].tile0 <= tile)
          lo = mid;
        else
          hi = mid - 1;
      }
      const BatchFrame& f = frames[lo];
      if (lo != cur) {
        __syncthreads();
        if (tid < int(f.m)) sm.hh[tid] = f.hh[tid];
        __syncthreads();
        cur = lo;
      }
      const uint32_t t = tile - f.tile0;
      const int rr = int(t / f.tiles_x) * th + ty, cc = int(t % f.tiles_x) * kTW + tx;
      if (tid < npx && rr < int(f.rows) && cc < int(f.cols)) {
        const size_t p = size_t(rr) * f.cols + size_t(cc);
        float tq[K], aq[K];
        bool cq[K];
        load_state<K>(f.depth, f.alpha, f.active, p, tq, aq, cq);
        const float nmax = float(max(reinterpret_cast<const unsigned*>(f.misc)[MISC_NMAX], 1u));
        grad_pixel<K>(f.S + p * f.m, f.n[p], f.T, f.m, sm.hh, f.misc[MISC_ETA_T] / nmax, f.misc[MISC_ETA_A] / nmax,
                      tq, aq, cq);
        unsigned long long* xt = f.xtag + (it & 1u) * (size_t(f.P) * K * 2);
#pragma unroll
        for (int k = 0; k < K; ++k) st_tagged2(xt + (p * K + k) * 2, tq[k], cq[k] ? aq[k] : -1.f, it + 1u);
      }
    }
    // phase 2: normals, projection, smoothing and pruning
    for (uint32_t tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
      uint32_t lo = 0, hi = nframes - 1;
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) / 2;
        if (frames[mid].tile0 <= tile)
          lo = mid;
        else
          hi = mid - 1;
      }
      const BatchFrame& f = frames[lo];
      Stencil st = base;
      st.rows = f.rows;
      st.cols = f.cols;
      const uint32_t t = tile - f.tile0;
      const int tyy = int(t / f.tiles_x), txx = int(t % f.tiles_x);
      const int r0 = tyy * th, c0 = txx * kTW;
      const unsigned long long* xt = f.xtag + (it & 1u) * (size_t(f.P) * K * 2);
      for (int i = tid; i < RH * RW; i += NT) {
        const int hr = r0 - H + i / RW, hc = c0 - H + i % RW;
        float ht[K], ha[K];
        bool hact[K];
        if (hr >= 0 && hr < int(f.rows) && hc >= 0 && hc < int(f.cols)) {
          if (!load_state_tagged<K>(xt, size_t(hr) * f.cols + size_t(hc), it + 1u, kGridWaitCycles, ht, ha, hact)) {
            s_abort = 1;
            atomicOr(err, FLAG_DEVICE_TIMEOUT);
          }
        } else {
#pragma unroll
          for (int k = 0; k < K; ++k) {
            ht[k] = 0.f;
            ha[k] = 0.f;
            hact[k] = false;
          }
        }
        put_state<K, R>(sm, i, ht, ha, hact);
      }
      if (tid == 0) reset_lists(sm);
      __syncthreads();
      if (s_abort) return;  // uniform: read after the barrier
      stage2<K, R, NT>(sm, st, th);
      __syncthreads();
      float tout[K], aout[K];
      bool aact[K];
      stage3<K, R>(sm, st, r0, c0, th, f.depth, f.alpha, f.active, f.alpha0, tout, aout, aact, true);
      __syncthreads();  // the next tile's region load rewrites shared memory
    }
  }
}

template <int K>
__global__ void k_alpha0(uint32_t P, const float* __restrict__ alpha, const uint8_t* __restrict__ active,
                         float* __restrict__ alpha0, const uint32_t* __restrict__ n, float* __restrict__ misc) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t nm = p < P ? n[p] : 0u;
  for (int off = 16; off; off >>= 1) nm = max(nm, __shfl_xor_sync(0xffffffffu, nm, off));
  if ((threadIdx.x & 31u) == 0u) atomicMax(reinterpret_cast<unsigned*>(misc) + MISC_NMAX, nm);
  if (p >= P) return;
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) s += active[size_t(p) * K + k] ? alpha[size_t(p) * K + k] : 0.f;
  alpha0[p] = 1.f - s;
}

// Tile height for the persistent kernel: the th in [4, kTH] whose tiles all
// fit on the device at once (bps CTAs per SM) and minimise the work of the
// busiest SM, ceil(tiles / SMs) x the per-tile work (the tile's gradient
// steps + the normals region + 2 x tile for the projection, + the halo
// loads). 0 if no th fits.
template <int R>
uint32_t persistent_tile_height(uint32_t rows, uint32_t cols, int num_sms, int bps) {
  constexpr int H = 2 * R;
  const uint64_t tiles_x = (cols + kTW - 1) / kTW;
  uint32_t best = 0;
  uint64_t best_cost = ~uint64_t(0);
  for (uint32_t th = kTH; th >= 4; --th) {
    const uint64_t ntiles = tiles_x * ((rows + th - 1) / th);
    if (ntiles > uint64_t(num_sms) * uint64_t(bps)) continue;
    const uint64_t halo = uint64_t(th + 2 * H) * (kTW + 2 * H) - uint64_t(kTW) * th;
    const uint64_t per_tile = uint64_t(kTW) * th + uint64_t(th + 2 * R) * (kTW + 2 * R) + 2ull * kTW * th + halo / 4;
    const uint64_t cost = (ntiles + num_sms - 1) / num_sms * per_tile;
    if (cost < best_cost) {
      best_cost = cost;
      best = th;
    }
  }
  return best;
}

// Cooperative launch of k_iter_persistent; SRT3D_EAGAIN when the tiles do
// not all fit on the device at once (the caller then launches per iteration).
template <int K, int R>
srt3d_status launch_iter_persistent(srt3d_ctx* ctx, const Stencil& st, const float2* z, const uint32_t* n,
                                    uint32_t T, uint32_t m, const Scratch& sc, float* depth, float* alpha,
                                    uint8_t* active, float* alpha0, uint32_t iters, uint32_t flag_base,
                                    uint32_t* flags, bool inject_barrier_timeout, cudaStream_t stream) {
  if constexpr (K > 2 && R > 1) {
    // three or four points per pixel at radius > 1 do not fit two CTAs per SM:
    // the caller launches per iteration
    return SRT3D_EAGAIN;
  } else {
  const size_t zsmem = size_t(kTW) * kTH * (size_t(m) * sizeof(float2) + sizeof(uint32_t));
  auto fn = k_iter_persistent<K, R, R == 1 ? 3 : 1>;
  cudaFuncAttributes fa;
  SRT3D_CUDA_TRY(ctx, cudaFuncGetAttributes(&fa, fn));
  if (fa.sharedSizeBytes + zsmem > ctx->smem_optin) return SRT3D_EAGAIN;
  // static + dynamic shared memory may exceed the 48 KB default
  SRT3D_CUDA_TRY(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(zsmem)));
  int bps = 0;
  SRT3D_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, persist_block<K, R, R == 1 ? 3 : 1>(),
                                                                    zsmem));
  int block = persist_block<K, R, R == 1 ? 3 : 1>();
  const uint32_t th = persistent_tile_height<R>(st.rows, st.cols, ctx->num_sms, bps);
  if (th == 0) return SRT3D_EAGAIN;
  const uint32_t tiles_x = (st.cols + kTW - 1) / kTW;
  const uint32_t ntiles = tiles_x * ((st.rows + th - 1) / th);
  if constexpr (R == 1) {
    // tiles that fit two per SM: the variant with more registers per thread
    if (ntiles <= 2u * uint32_t(ctx->num_sms)) {
      auto fn2 = k_iter_persistent<K, R, 2>;
      SRT3D_CUDA_TRY(ctx, cudaFuncSetAttribute(fn2, cudaFuncAttributeMaxDynamicSharedMemorySize, int(zsmem)));
      int bps2 = 0;
      SRT3D_CUDA_TRY(ctx,
                     cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps2, fn2, persist_block<K, R, 2>(), zsmem));
      if (bps2 >= 2) {
        fn = fn2;
        block = persist_block<K, R, 2>();
      }
    }
  }
  if (ntiles * kTileFlagStride > kMaxTileFlags) return SRT3D_EAGAIN;
  // exchange buffers: the scratch block's spare region and its alternate state
  const size_t pk = size_t(st.rows) * st.cols * K;
  XBuf x0{sc.xch, sc.xch + pk, reinterpret_cast<uint8_t*>(sc.xch + 2 * pk)};
  XBuf x1{sc.t1, sc.a1, sc.act1};
  Stencil stv = st;
  const float2* zz = z;
  const uint32_t* nn = n;
  uint32_t TT = T, mm = m, it = iters, tx = tiles_x, thv = th;
  const float2* hh = sc.hh;
  float* misc = sc.misc;
  float *d = depth, *a = alpha, *a0 = alpha0;
  uint8_t* c = active;
  uint32_t* fl = flags;
  // fault injection (tests): a neighbour-flag target one iteration beyond
  // what the tiles publish, with a ~50 us limit, so every CTA's wait gives up
  uint32_t skew = inject_barrier_timeout ? 1u : 0u, fbase = flag_base;
  long long limit = inject_barrier_timeout ? kInjectedWaitCycles : kGridWaitCycles;
  unsigned* tflags = sc.tile_flags;
  // tagged exchange when the scratch block holds its buffers (zeroed by the
  // init of this reconstruction: tag 0 never matches an iteration's tag)
  unsigned long long* xt = uint64_t(flag_base) + iters + 2u < (1ull << 32) ? sc.xtag : nullptr;
  void* args[] = {&stv, &zz, &nn, &TT, &mm, &hh, &misc, &d, &a, &c, &a0, &x0, &x1, &it, &tx, &thv, &fl, &tflags,
                  &fbase, &skew, &limit, &xt};
  const ProfMark mk = prof_begin(ctx, KID_ITER_ALL, stream);
  const srt3d_status ls = launch_cooperative_chained(ctx, reinterpret_cast<const void*>(fn), dim3(ntiles),
                                                     dim3(block), args, zsmem, stream);
  prof_end(ctx, KID_ITER_ALL, mk, stream);
  return ls;
  }
}

template <int K>
srt3d_status run(srt3d_ctx* ctx, const float2* z, const uint32_t* n, uint32_t rows, uint32_t cols, uint32_t T,
                 uint32_t m, const float* h, const srt3d_params& prm, float* depth, float* alpha, uint8_t* active,
                 float* alpha0, const Scratch& sc, const PhaseTable& tab, uint32_t* flags, bool inject_barrier_timeout,
                 cudaStream_t stream) {
  const uint32_t P = rows * cols;
  const int tl = tab.two_level ? 1 : 0;
  {
    const ProfMark mk = prof_begin(ctx, KID_PREP, stream);
    k_prep_part<<<dim3(kPrepSlices, m), kPrepGroup, 0, stream>>>(h, T, tab.dev, tl, sc.part);
    k_prep_final<<<1, 1024, 0, stream>>>(sc.part, T, m, K, sc.hh, sc.misc, sc.tile_flags);
    prof_end(ctx, KID_PREP, mk, stream, 2);
  }
  SRT3D_CUDA_TRY(ctx, cudaGetLastError());
  if (prm.init_mode == SRT3D_INIT_MATCHED) {
    const srt3d_status st = launch_init(ctx, z, n, P, T, m, K, tab, sc.hh, sc.misc, prm, depth, alpha, active,
                                        alpha0, stream);
    if (st != SRT3D_OK) return st;
  } else {
    {
      const ProfMark mk = prof_begin(ctx, KID_ALPHA0, stream);
      k_alpha0<K><<<(P + kBlock - 1) / kBlock, kBlock, 0, stream>>>(P, alpha, active, alpha0, n, sc.misc);
      prof_end(ctx, KID_ALPHA0, mk, stream);
    }
    SRT3D_CUDA_TRY(ctx, cudaGetLastError());
  }
  const uint32_t grid = (P + kBlock - 1) / kBlock;
  Stencil st;
  st.rows = rows;
  st.cols = cols;
  st.radius = prm.radius;
  st.h2 = prm.apss_h * prm.apss_h;
  st.inv_h2 = 1.f / st.h2;
  st.d_max = prm.d_max;
  st.ds = prm.depth_scale;
  st.lambda = prm.smooth_lambda;
  st.prune_alpha = prm.prune_alpha;
  const dim3 tiles((cols + kTW - 1) / kTW, (rows + kTH - 1) / kTH);
  const char* env = std::getenv("SRT3D_ITER_PERSISTENT");
  const bool allow_persistent = !(env && env[0] == '0');
  // `count` iterations from the caller's state to the caller's state, after
  // `done` iterations of this reconstruction (the persistent kernel's progress
  // flags continue from there).
  const auto iterate_span = [&](uint32_t count, uint32_t done) -> srt3d_status {
    // All iterations in one cooperative launch when every tile's CTA fits on
    // the device at once (SRT3D_ITER_PERSISTENT=0 forces one launch per iteration).
    if (prm.regularize && count > 0 && allow_persistent) {
      srt3d_status pst;
      if (prm.radius == 1)
        pst = launch_iter_persistent<K, 1>(ctx, st, z, n, T, m, sc, depth, alpha, active, alpha0, count, done,
                                           flags, inject_barrier_timeout, stream);
      else if (prm.radius == 2)
        pst = launch_iter_persistent<K, 2>(ctx, st, z, n, T, m, sc, depth, alpha, active, alpha0, count, done,
                                           flags, inject_barrier_timeout, stream);
      else
        pst = launch_iter_persistent<K, 3>(ctx, st, z, n, T, m, sc, depth, alpha, active, alpha0, count, done,
                                           flags, inject_barrier_timeout, stream);
      if (pst != SRT3D_EAGAIN) return pst;  // launched (or failed)
    }
    // One launch per iteration: ping-pong between the caller's state and the
    // scratch copy (t1, a1, act1); with an odd count the state is first copied
    // to scratch, so that the last iteration writes the caller's buffers.
    const size_t pk = size_t(P) * K;
    if (prm.regularize && (count & 1u)) {
      SRT3D_CUDA_TRY(ctx, cudaMemcpyAsync(sc.t1, depth, pk * sizeof(float), cudaMemcpyDeviceToDevice, stream));
      SRT3D_CUDA_TRY(ctx, cudaMemcpyAsync(sc.a1, alpha, pk * sizeof(float), cudaMemcpyDeviceToDevice, stream));
      SRT3D_CUDA_TRY(ctx, cudaMemcpyAsync(sc.act1, active, pk, cudaMemcpyDeviceToDevice, stream));
    }
    for (uint32_t it = 0; it < count; ++it) {
      const ProfMark mk = prof_begin(ctx, prm.regularize ? KID_ITER : KID_GRAD, stream);
      const bool from_scratch = ((count - it) & 1u) != 0;  // the last iteration reads scratch
      const float* din = from_scratch ? sc.t1 : depth;
      const float* ain = from_scratch ? sc.a1 : alpha;
      const uint8_t* cin = from_scratch ? sc.act1 : active;
      float* dout = from_scratch ? depth : sc.t1;
      float* aout = from_scratch ? alpha : sc.a1;
      uint8_t* cout = from_scratch ? active : sc.act1;
      if (!prm.regularize) {
        if (prm.weighting)
          k_grad<K, true><<<grid, kBlock, 0, stream>>>(z, n, P, T, m, sc.hh, sc.misc, depth, alpha, active, alpha0);
        else
          k_grad<K, false><<<grid, kBlock, 0, stream>>>(z, n, P, T, m, sc.hh, sc.misc, depth, alpha, active, alpha0);
      } else if (prm.radius == 1) {
        k_iter<K, 1><<<tiles, iter_threads<1>(), 0, stream>>>(st, z, n, T, m, sc.hh, sc.misc, din, ain, cin, dout,
                                                             aout, cout, alpha0);
      } else if (prm.radius == 2) {
        k_iter<K, 2><<<tiles, iter_threads<2>(), 0, stream>>>(st, z, n, T, m, sc.hh, sc.misc, din, ain, cin, dout,
                                                             aout, cout, alpha0);
      } else {
        k_iter<K, 3><<<tiles, iter_threads<3>(), 0, stream>>>(st, z, n, T, m, sc.hh, sc.misc, din, ain, cin, dout,
                                                             aout, cout, alpha0);
      }
      prof_end(ctx, prm.regularize ? KID_ITER : KID_GRAD, mk, stream);
      SRT3D_CUDA_TRY(ctx, cudaGetLastError());
    }
    return SRT3D_OK;
  };
  // the persistent kernel's tagged exchange words start at tag 0, which no
  // iteration uses: words a previous reconstruction left never match
  if (sc.xtag && prm.regularize && prm.iters > 0 && allow_persistent)
    SRT3D_CUDA_TRY(ctx, cudaMemsetAsync(sc.xtag, 0, scratch_xtag_bytes(P, K), stream));
  if (prm.birth_every == 0) return iterate_span(prm.iters, 0);
  // birth moves every birth_every iterations, not after the last one
  uint32_t done = 0;
  while (done < prm.iters) {
    const uint32_t span = std::min(prm.birth_every, prm.iters - done);
    srt3d_status s2 = iterate_span(span, done);
    if (s2 != SRT3D_OK) return s2;
    done += span;
    if (done < prm.iters) {
      s2 = launch_birth(ctx, z, n, P, T, m, K, tab, sc.hh, sc.misc, prm, depth, alpha, active, alpha0, stream);
      if (s2 != SRT3D_OK) return s2;
    }
  }
  return SRT3D_OK;
}

Stencil batch_stencil(const srt3d_params& prm) {
  Stencil st;
  st.rows = 0;
  st.cols = 0;
  st.radius = prm.radius;
  st.h2 = prm.apss_h * prm.apss_h;
  st.inv_h2 = 1.f / st.h2;
  st.d_max = prm.d_max;
  st.ds = prm.depth_scale;
  st.lambda = prm.smooth_lambda;
  st.prune_alpha = prm.prune_alpha;
  return st;
}

template <int K, int R>
srt3d_status iterations_batch(srt3d_ctx* ctx, const BatchFrame* d_frames, uint32_t nframes, uint32_t total_tiles,
                              uint32_t th, unsigned* tile_flags, uint32_t iters, const srt3d_params& prm,
                              cudaStream_t stream) {
  if (iters == 0 || total_tiles == 0) return SRT3D_OK;
  auto fn = k_iter_batch_persistent<K, R>;
  int bps = 0;
  SRT3D_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, persist_threads<R>(), 0));
  if (bps < 1) return set_error(ctx, SRT3D_ECUDA, "batched iteration kernel does not fit on an SM");
  const uint32_t grid = std::min<uint32_t>(total_tiles, uint32_t(ctx->num_sms) * uint32_t(bps));
  Stencil st = batch_stencil(prm);
  const BatchFrame* fr = d_frames;
  uint32_t nf = nframes, tt = total_tiles, thv = th, it = iters;
  unsigned* fl = tile_flags;
  uint32_t* err = ctx->d_flags;
  void* args[] = {&st, &fr, &nf, &tt, &thv, &it, &fl, &err};
  const ProfMark mk = prof_begin(ctx, KID_ITER_ALL, stream);
  const srt3d_status ls = launch_cooperative_chained(ctx, reinterpret_cast<const void*>(fn), dim3(grid),
                                                     dim3(persist_threads<R>()), args, 0, stream);
  prof_end(ctx, KID_ITER_ALL, mk, stream);
  return ls;
}

template <int K>
srt3d_status iterations_batch_r(srt3d_ctx* ctx, const BatchFrame* d_frames, uint32_t nframes, uint32_t total_tiles,
                                uint32_t th, unsigned* tile_flags, uint32_t iters, const srt3d_params& prm,
                                cudaStream_t stream) {
  if (prm.radius == 1)
    return iterations_batch<K, 1>(ctx, d_frames, nframes, total_tiles, th, tile_flags, iters, prm, stream);
  if (prm.radius == 2)
    return iterations_batch<K, 2>(ctx, d_frames, nframes, total_tiles, th, tile_flags, iters, prm, stream);
  return iterations_batch<K, 3>(ctx, d_frames, nframes, total_tiles, th, tile_flags, iters, prm, stream);
}

template <int K>
srt3d_status run_batch(srt3d_ctx* ctx, const BatchFrame* d_frames, uint32_t nframes, const InitGroup* groups,
                       uint32_t num_groups, uint32_t total_tiles, uint32_t th, unsigned* tile_flags,
                       uint32_t max_entries, uint32_t max_G, const srt3d_params& prm, cudaStream_t stream) {
  {
    const ProfMark mk = prof_begin(ctx, KID_PREP, stream);
    k_prep_batch<<<nframes, 1024, 0, stream>>>(d_frames, K, tile_flags);
    prof_end(ctx, KID_PREP, mk, stream);
  }
  SRT3D_CUDA_TRY(ctx, cudaGetLastError());
  for (uint32_t g = 0; g < num_groups; ++g) {
    const srt3d_status st = launch_init_batch(ctx, d_frames, groups[g].items, groups[g].count, K, groups[g].M,
                                              max_entries, max_G, prm, stream);
    if (st != SRT3D_OK) return st;
  }
  return iterations_batch_r<K>(ctx, d_frames, nframes, total_tiles, th, tile_flags, prm.iters, prm, stream);
}

}  // namespace

uint32_t tile_flag_stride() { return kTileFlagStride; }
uint32_t max_tile_height() { return kTH; }

srt3d_status launch_reconstruct_batch(srt3d_ctx* ctx, const BatchFrame* d_frames, uint32_t nframes,
                                      const InitGroup* init_groups, uint32_t num_groups, uint32_t total_tiles,
                                      uint32_t th, unsigned* tile_flags, uint32_t max_tab_entries, uint32_t max_G,
                                      const srt3d_params& prm, cudaStream_t stream) {
  switch (prm.k_max) {
    case 1:
      return run_batch<1>(ctx, d_frames, nframes, init_groups, num_groups, total_tiles, th, tile_flags,
                          max_tab_entries, max_G, prm, stream);
    case 2:
      return run_batch<2>(ctx, d_frames, nframes, init_groups, num_groups, total_tiles, th, tile_flags,
                          max_tab_entries, max_G, prm, stream);
    case 3:
      return run_batch<3>(ctx, d_frames, nframes, init_groups, num_groups, total_tiles, th, tile_flags,
                          max_tab_entries, max_G, prm, stream);
    default:
      return run_batch<4>(ctx, d_frames, nframes, init_groups, num_groups, total_tiles, th, tile_flags,
                          max_tab_entries, max_G, prm, stream);
  }
}

srt3d_status launch_iterations_batch(srt3d_ctx* ctx, const BatchFrame* d_frames, uint32_t nframes,
                                     uint32_t total_tiles, uint32_t th, unsigned* tile_flags, uint32_t iters,
                                     const srt3d_params& prm, cudaStream_t stream) {
  switch (prm.k_max) {
    case 1: return iterations_batch_r<1>(ctx, d_frames, nframes, total_tiles, th, tile_flags, iters, prm, stream);
    case 2: return iterations_batch_r<2>(ctx, d_frames, nframes, total_tiles, th, tile_flags, iters, prm, stream);
    case 3: return iterations_batch_r<3>(ctx, d_frames, nframes, total_tiles, th, tile_flags, iters, prm, stream);
    default: return iterations_batch_r<4>(ctx, d_frames, nframes, total_tiles, th, tile_flags, iters, prm, stream);
  }
}

// Cooperative grids of this library never run concurrently on one device.
// A cooperative launch is sized so that all its CTAs fit on an otherwise idle
// device; two such grids issued from different streams (serving slots, or
// callers' streams) could each become partly resident, every resident CTA
// spinning in the grid barrier on CTAs that wait for the other grid's SMs,
// until the bounded wait gives up. Chaining them through one event per device
// (each launch waits on the event the previous launch recorded) leaves at most
// one cooperative grid on the device; the other kernels of the library never
// wait on anything, so the SMs they hold free up in bounded time and every CTA
// of the cooperative grid becomes resident. Not chained while the stream is
// being captured into a graph (an event of another stream cannot be waited on
// there): the batch graph's cooperative node runs on the stream the caller
// launches the graph on, serialised with that stream's work only.
namespace {
constexpr int kCoopMaxDevices = 64;
std::mutex g_coop_mu;
cudaEvent_t g_coop_ev[kCoopMaxDevices];
}  // namespace

srt3d_status coop_chain_init(srt3d_ctx* ctx) {
  if (ctx->device < 0 || ctx->device >= kCoopMaxDevices) return SRT3D_OK;  // launches are then not chained
  std::lock_guard<std::mutex> lock(g_coop_mu);
  if (!g_coop_ev[ctx->device])
    SRT3D_CUDA_TRY(ctx, cudaEventCreateWithFlags(&g_coop_ev[ctx->device], cudaEventDisableTiming));
  return SRT3D_OK;
}

srt3d_status launch_cooperative_chained(srt3d_ctx* ctx, const void* fn, dim3 grid, dim3 block, void** args,
                                        size_t smem, cudaStream_t stream) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  SRT3D_CUDA_TRY(ctx, cudaStreamIsCapturing(stream, &cap));
  cudaEvent_t ev = nullptr;
  if (cap == cudaStreamCaptureStatusNone && ctx->device >= 0 && ctx->device < kCoopMaxDevices) {
    std::lock_guard<std::mutex> lock(g_coop_mu);
    ev = g_coop_ev[ctx->device];
    if (ev) {
      SRT3D_CUDA_TRY(ctx, cudaStreamWaitEvent(stream, ev, 0));
      SRT3D_CUDA_TRY(ctx, cudaLaunchCooperativeKernel(fn, grid, block, args, smem, stream));
      SRT3D_CUDA_TRY(ctx, cudaEventRecord(ev, stream));
      return SRT3D_OK;
    }
  }
  SRT3D_CUDA_TRY(ctx, cudaLaunchCooperativeKernel(fn, grid, block, args, smem, stream));
  return SRT3D_OK;
}

uint32_t plan_tile_height(uint32_t k_max, uint32_t radius, uint32_t rows, uint32_t cols, int num_sms, int bps) {
  if (k_max > 2 && radius > 1) return 0;  // such launches go one iteration at a time
  switch (radius) {
    case 1: return persistent_tile_height<1>(rows, cols, num_sms, bps);
    case 2: return persistent_tile_height<2>(rows, cols, num_sms, bps);
    default: return persistent_tile_height<3>(rows, cols, num_sms, bps);
  }
}

size_t reconstruct_scratch_bytes(uint32_t P, uint32_t k_max, uint32_t m) {
  (void)m;
  return scratch_min_bytes(P, k_max) + scratch_xtag_bytes(P, k_max);
}

srt3d_status reconstruct_impl(srt3d_ctx* ctx, const float2* z, const uint32_t* n, uint32_t rows, uint32_t cols,
                              uint32_t T, uint32_t m, const float* h, const srt3d_params& prm, float* depth,
                              float* alpha, uint8_t* active, float* alpha0, void* scratch, size_t scratch_bytes,
                              cudaStream_t stream, uint32_t* flags, bool inject_barrier_timeout) {
  const uint32_t P = rows * cols;
  if (!flags) flags = ctx->d_flags;
  if (scratch_bytes < scratch_min_bytes(P, prm.k_max))
    return set_error(ctx, SRT3D_EINVAL, "reconstruction scratch too small");
  PhaseTable tab;
  srt3d_status st = get_phase_table(ctx, T, &tab);
  if (st != SRT3D_OK) return st;
  const Scratch sc = carve(scratch, scratch_bytes, P, prm.k_max);
  switch (prm.k_max) {
    case 1: return run<1>(ctx, z, n, rows, cols, T, m, h, prm, depth, alpha, active, alpha0, sc, tab, flags,
                            inject_barrier_timeout, stream);
    case 2: return run<2>(ctx, z, n, rows, cols, T, m, h, prm, depth, alpha, active, alpha0, sc, tab, flags,
                            inject_barrier_timeout, stream);
    case 3: return run<3>(ctx, z, n, rows, cols, T, m, h, prm, depth, alpha, active, alpha0, sc, tab, flags,
                            inject_barrier_timeout, stream);
    default: return run<4>(ctx, z, n, rows, cols, T, m, h, prm, depth, alpha, active, alpha0, sc, tab, flags,
                           inject_barrier_timeout, stream);
  }
}

}  // namespace srt3d

using namespace srt3d;

extern "C" srt3d_status srt3d_reconstruct(srt3d_ctx* ctx, const float* z, const uint32_t* n, uint32_t rows,
                                          uint32_t cols, uint32_t T, uint32_t m, const float* h,
                                          const srt3d_params* params, float* depth, float* alpha, uint8_t* active,
                                          float* alpha0, void* stream) {
  if (!ctx) return SRT3D_EINVAL;
  srt3d_status st = validate_params(ctx, rows, cols, T, m, params);
  if (st != SRT3D_OK) return st;
  if (!z || !n || !h || !depth || !alpha || !active || !alpha0) return set_error(ctx, SRT3D_EINVAL, "NULL pointer");
  if (reinterpret_cast<uintptr_t>(z) % 8) return set_error(ctx, SRT3D_EINVAL, "z must be 8-byte aligned");
  const uint32_t P = rows * cols;
  const size_t need = reconstruct_scratch_bytes(P, params->k_max, m);
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    st = grow(ctx, &ctx->rc_scratch, need);
  }
  if (st != SRT3D_OK) return st;
  return reconstruct_impl(ctx, reinterpret_cast<const float2*>(z), n, rows, cols, T, m, h, *params, depth, alpha,
                          active, alpha0, ctx->rc_scratch.ptr, ctx->rc_scratch.bytes,
                          static_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------------------
// Allocation-free variant of srt3d_reconstruct.
//
// Some callers cannot allocate device memory at the moment they reconstruct a
// frame: a lidar front-end that runs the reconstruction inside a hard
// real-time loop (cudaMalloc / cudaFree may synchronise the whole device and
// take unbounded time), or a process whose device memory is entirely reserved
// by another allocator. srt3d_reconstruct_noalloc serves them: its scratch
// (post-gradient state, normals, hhat, step sizes) and its phase table live in
// one file-scope __device__ array of fixed size that every GPU loading this
// library holds until exit. The launches are the ones srt3d_reconstruct uses.
namespace srt3d {
namespace {

constexpr size_t kNoAllocBytes = size_t(16) << 20;                   // whole array: 16 MiB
constexpr size_t kNoAllocTableBytes = size_t(kDirectTableMax) * sizeof(float2);  // 64 KiB
constexpr size_t kNoAllocScratchMax = kNoAllocBytes - kNoAllocTableBytes;
constexpr int kNoAllocMaxDevices = 64;
constexpr uint64_t kNoAllocMaxPoints = 655360;  // rows * cols * k_max

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices];  // device address of the array, per device

// The phase table reaches the array through kernel parameters: each launch
// carries up to kNoAllocTableChunk entries (24 KiB of its 32 KiB parameter
// space) built on the host by phase_table_host, the same values the
// allocating path uploads, so the two entry points compute bit for bit the
// same result. No host staging, no copy from pageable memory, no device FP64.
constexpr uint32_t kNoAllocTableChunk = 3072;
struct TableChunk {
  float2 v[kNoAllocTableChunk];
};
float2 g_noalloc_host_table[kDirectTableMax];  // guarded by g_noalloc_mu

__global__ void k_noalloc_put_table(const TableChunk chunk, uint32_t first, uint32_t count, float2* __restrict__ tab) {
  for (uint32_t i = threadIdx.x; i < count; i += blockDim.x) tab[first + i] = chunk.v[i];
}

}  // namespace

void noalloc_forget_device(int device) {
  if (device < 0 || device >= kNoAllocMaxDevices) return;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  g_noalloc_addr[device] = nullptr;
}

}  // namespace srt3d

static __device__ __align__(256) unsigned char g_noalloc_scratch[srt3d::kNoAllocBytes];

extern "C" srt3d_status srt3d_reconstruct_noalloc(srt3d_ctx* ctx, const float* z, const uint32_t* n, uint32_t rows,
                                                  uint32_t cols, uint32_t T, uint32_t m, const float* h,
                                                  const srt3d_params* params, float* depth, float* alpha,
                                                  uint8_t* active, float* alpha0, void* stream) {
  using namespace srt3d;
  if (!ctx) return SRT3D_EINVAL;
  srt3d_status st = validate_params(ctx, rows, cols, T, m, params);
  if (st != SRT3D_OK) return st;
  if (!z || !n || !h || !depth || !alpha || !active || !alpha0) return set_error(ctx, SRT3D_EINVAL, "NULL pointer");
  if (reinterpret_cast<uintptr_t>(z) % 8) return set_error(ctx, SRT3D_EINVAL, "z must be 8-byte aligned");
  if (ctx->prof.enabled)
    return set_error(ctx, SRT3D_EINVAL, "srt3d_reconstruct_noalloc: disable profiling (it creates CUDA events)");
  const uint32_t P = rows * cols;
  // (the tagged exchange buffers are used when they fit too; without them
  // the iterations exchange state through progress flags, same results)
  const size_t need = scratch_min_bytes(P, params->k_max);
  if (uint64_t(P) * params->k_max > kNoAllocMaxPoints || need > kNoAllocScratchMax)
    return set_error(ctx, SRT3D_EINVAL,
                     "srt3d_reconstruct_noalloc: frame too large for the static scratch (rows*cols*k_max must be "
                     "<= 655360 points)");
  if (ctx->device < 0 || ctx->device >= kNoAllocMaxDevices)
    return set_error(ctx, SRT3D_EINVAL, "srt3d_reconstruct_noalloc: device index out of range");
  // Set-up once per device, with that device current: the array's device address.
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[ctx->device]) {
      int cur = -1;
      SRT3D_CUDA_TRY(ctx, cudaGetDevice(&cur));
      if (cur != ctx->device) SRT3D_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (cur != ctx->device) cudaSetDevice(cur);
      if (e != cudaSuccess) return cuda_error(ctx, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
      g_noalloc_addr[ctx->device] = p;
    }
    base = g_noalloc_addr[ctx->device];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Phase table at the end of the array, rewritten on every call (every word
  // of the array is written before it is read within a call; nothing needs
  // clearing). The launches copy their parameters when they are issued, so
  // the host table is free again when they return.
  PhaseTable tab;
  tab.dev = reinterpret_cast<float2*>(static_cast<char*>(base) + kNoAllocScratchMax);
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    tab.entries = phase_table_host(T, g_noalloc_host_table, &tab.two_level);
    for (uint32_t first = 0; first < tab.entries; first += kNoAllocTableChunk) {
      const uint32_t count = std::min(kNoAllocTableChunk, tab.entries - first);
      TableChunk c;
      std::memcpy(c.v, g_noalloc_host_table + first, size_t(count) * sizeof(float2));
      k_noalloc_put_table<<<1, 256, 0, s>>>(c, first, count, tab.dev);
      SRT3D_CUDA_TRY(ctx, cudaGetLastError());
    }
  }
  const Scratch sc = carve(base, kNoAllocScratchMax, P, params->k_max);
  const float2* zz = reinterpret_cast<const float2*>(z);
  switch (params->k_max) {
    case 1: return run<1>(ctx, zz, n, rows, cols, T, m, h, *params, depth, alpha, active, alpha0, sc, tab,
                            ctx->d_flags, false, s);
    case 2: return run<2>(ctx, zz, n, rows, cols, T, m, h, *params, depth, alpha, active, alpha0, sc, tab,
                            ctx->d_flags, false, s);
    case 3: return run<3>(ctx, zz, n, rows, cols, T, m, h, *params, depth, alpha, active, alpha0, sc, tab,
                            ctx->d_flags, false, s);
    default: return run<4>(ctx, zz, n, rows, cols, T, m, h, *params, depth, alpha, active, alpha0, sc, tab,
                           ctx->d_flags, false, s);
  }
}

extern "C" srt3d_status srt3d_selftest_wait_timeout(srt3d_ctx* ctx, uint64_t wait_cycles, void* stream) {
  if (!ctx) return SRT3D_EINVAL;
  if (wait_cycles == 0 || wait_cycles > 4000000000ull)
    return set_error(ctx, SRT3D_EINVAL, "wait_cycles must be in [1, 4e9]");
  k_selftest_wait<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(ctx->d_flags, static_cast<long long>(wait_cycles));
  SRT3D_CUDA_TRY(ctx, cudaGetLastError());
  return SRT3D_OK;
}
