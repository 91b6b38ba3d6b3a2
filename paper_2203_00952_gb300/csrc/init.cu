// Sketched matched-filter initialisation (Sec. 3): for each pixel, the first
// point is the integer t maximising
//   s(t) = Re sum_{l=1}^{m} c_l e^{-i w_l t},   c_l = conj(hhat_l) z_l,
// with alpha = s / sum_l |hhat_l|^2; point k = 2..K maximises the same score of
// the residual z - sum_{i<k} f_i hhat e^{i w t_i} (f_i = alpha_i if it reaches
// prune_alpha, else 0) at least min_sep bins (circularly) from every earlier
// t_i (greedy passes; K <= 4).
//
// One warp per pixel. The coefficients c_l live in registers, zero-padded to
// the kernel's harmonic count M (Horner with leading zero coefficients gives
// the same FP32 value bit for bit). Scores are evaluated by complex Horner in
// w = e^{-i 2 pi t / T}; grid points are evaluated two per lane with packed
// FP32 pairs whose operations round exactly like the scalar evaluation, so
// every candidate's score is the same FP32 number whichever way it is
// computed. The argmax is exact (see warp_argmax_scores).
#include <cfloat>
#include <cmath>

#include "device_util.cuh"
#include "internal.h"

namespace srt3d {
namespace {

constexpr int kBlock = 256;
constexpr int kMaxM = 32;

// Harmonic counts with their own instantiation; other m are zero-padded to
// the next one up.
constexpr int kInitM[] = {2, 4, 6, 8, 10, 12, 16, 20, 24, 32};

// The coefficients are held as duplicated pairs (c, c) so that the packed
// evaluation below can use them directly.
// s(t) for one t; `we` = e^{+i 2 pi t / T}, so w = conj(we).
template <int M>
__device__ __forceinline__ float mf_score(const float2 (&cx)[M], const float2 (&cy)[M], float2 we) {
  const float wx = we.x, wy = -we.y;
  float ax = cx[M - 1].x, ay = cy[M - 1].x;
#pragma unroll
  for (int l = M - 2; l >= 0; --l) {
    const float nx = fmaf(ax, wx, fmaf(ay, -wy, cx[l].x));
    const float ny = fmaf(ax, wy, fmaf(ay, wx, cy[l].x));
    ax = nx;
    ay = ny;
  }
  return fmaf(ax, wx, ay * -wy);
}

// s(t) at two points at once, each component rounded exactly as mf_score.
template <int M>
__device__ __forceinline__ float2 mf_score2(const float2 (&cx)[M], const float2 (&cy)[M], float2 weA,
                                            float2 weB) {
  const float2 wx = make_float2(weA.x, weB.x);
  const float2 wy = make_float2(-weA.y, -weB.y);
  const float2 nwy = make_float2(weA.y, weB.y);
  float2 ax = cx[M - 1], ay = cy[M - 1];
#pragma unroll
  for (int l = M - 2; l >= 0; --l) {
    const float2 nx = ffma2(ax, wx, ffma2(ay, nwy, cx[l]));
    const float2 ny = ffma2(ax, wy, ffma2(ay, wx, cy[l]));
    ax = nx;
    ay = ny;
  }
  return ffma2(ax, wx, fmul2(ay, nwy));
}

// Exclusion zones of a later pass: the first `used` (<= NX) of the earlier
// depths, and the least circular distance min_sep a candidate keeps from each.
template <int NX>
struct Excl {
  uint32_t t[NX > 0 ? NX : 1];
  float min_sep;
  int used;
};

template <int NX>
__device__ __forceinline__ bool mf_allowed(uint32_t t, const Excl<NX>& ex, uint32_t T) {
  bool ok = true;
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    const uint32_t d0 = t > ex.t[i] ? t - ex.t[i] : ex.t[i] - t;
    ok = ok && (i >= ex.used || float(min(d0, T - d0)) >= ex.min_sep);
  }
  return ok;
}

__device__ __forceinline__ void mf_take(float s, uint32_t t, float& bs, uint32_t& bt) {
  if (s > bs || (s == bs && t < bt)) {
    bs = s;
    bt = t;
  }
}

// Grid spacing of the branch and bound for a frame: the largest power of two
// D <= 64 with w_m^2 D^2 / 8 <= 0.08, so that for every pixel the curvature
// term M2 D^2 / 8 stays below 8% of M0 (M2 <= w_m^2 M0). G = ceil(T / D) is
// then at most 1024 (T <= 65536 gives D = 64 for every m <= 32). D only
// trades grid points against point-wise work in the surviving intervals
// (about 2.3 per pass on sketches of 10 to 5000 photons per pixel, whatever
// D up to 32); the result does not depend on it.
uint32_t mf_grid_spacing_impl(uint32_t T, uint32_t m) {
  const double w = 2.0 * M_PI * double(m) / double(T);
  uint32_t D = 64u;
  while (D > 1u && w * w * double(D) * double(D) / 8.0 > 0.08) D >>= 1;
  return D;
}

// Exact argmax over integer t in [0, T) (smallest t on ties) of the FP32
// scores, one warp per pixel, by branch and bound: s is a trigonometric
// polynomial with |s''| <= M2 = sum_l |c_l| w_l^2, so on an interval of length
// L between grid points s <= max(endpoints) + M2 L^2 / 8. Scores are evaluated
// on the grid t = g D (phases from the conflict-free coarse table s_wg, scores
// kept in s_grid), and only intervals whose bound (plus a margin covering the
// FP32 evaluation error of both ends) reaches the best grid score are
// evaluated point by point: their interior points are packed D to a slot
// across the warp's lanes. Every t whose FP32 score can be the maximum is
// evaluated with the same arithmetic as an exhaustive scan, so the result
// equals the exhaustive FP32 argmax.
template <int M, int NX>
__device__ __forceinline__ void warp_argmax_scores(float2 mine, const float2 (&cx)[M], const float2 (&cy)[M],
                                                   uint32_t T, const float2* s_tab, bool tl, const float2* s_wg,
                                                   float* s_grid, uint32_t D, uint32_t G, const Excl<NX>& ex,
                                                   float* best_s, uint32_t* best_t) {
  const uint32_t lane = threadIdx.x & 31u;
  // M0 = sum |c_l|, M2 = sum |c_l| w_l^2 (lane l holds c_{l+1}, zero beyond m)
  float m0 = sqrtf(mine.x * mine.x + mine.y * mine.y);
  const float wl = 6.283185307179586f * float(lane + 1u) / float(T);
  float m2 = m0 * wl * wl;
  for (int off = 16; off; off >>= 1) {
    m0 += __shfl_xor_sync(0xffffffffu, m0, off);
    m2 += __shfl_xor_sync(0xffffffffu, m2, off);
  }
  if (m0 == 0.f) {  // all scores are exactly 0: the smallest allowed t wins
    for (uint32_t t0 = 0; t0 < T; t0 += 32u) {
      const uint32_t t = t0 + lane;
      const unsigned ok = __ballot_sync(0xffffffffu, t < T && mf_allowed<NX>(t, ex, T));
      if (ok) {
        *best_s = 0.f;
        *best_t = t0 + uint32_t(__ffs(ok)) - 1u;
        return;
      }
    }
    *best_s = -FLT_MAX;
    *best_t = 0xffffffffu;
    return;
  }
  m2 *= 1.01f;
  const float margin = 4e-5f * m0 + 1e-30f;
  float bs = -FLT_MAX;
  uint32_t bt = 0xffffffffu;
  // grid points, two per lane (every score kept: the interval bounds need them)
  for (uint32_t g = lane; g < G; g += 64u) {
    const uint32_t g2 = g + 32u;
    const bool two = g2 < G;
    const float2 sg = mf_score2<M>(cx, cy, s_wg[g], s_wg[two ? g2 : g]);
    s_grid[g] = sg.x;
    if (mf_allowed<NX>(g * D, ex, T)) mf_take(sg.x, g * D, bs, bt);
    if (two) {
      s_grid[g2] = sg.y;
      if (mf_allowed<NX>(g2 * D, ex, T)) mf_take(sg.y, g2 * D, bs, bt);
    }
  }
  __syncwarp();
  float best_grid = bs;
  for (int off = 16; off; off >>= 1) best_grid = fmaxf(best_grid, __shfl_xor_sync(0xffffffffu, best_grid, off));
  // intervals whose bound reaches the best grid score
  if (D > 1u) {
    const uint32_t log2D = uint32_t(__ffs(int(D))) - 1u;
    for (uint32_t base = 0; base < G; base += 32u) {
      const uint32_t i = base + lane;
      bool surv = false;
      if (i < G) {
        const uint32_t len = min(D, T - i * D);
        if (len > 1u) {
          const float sa = s_grid[i], sb = s_grid[i + 1u < G ? i + 1u : 0u];
          surv = fmaxf(sa, sb) + m2 * float(len * len) * 0.125f + margin >= best_grid;
        }
      }
      const unsigned mask = __ballot_sync(0xffffffffu, surv);
      const uint32_t slots = uint32_t(__popc(mask)) << log2D;
      // slot f: surviving interval k = f / D (k-th set bit of mask), offset f % D
      for (uint32_t f = lane; f < slots; f += 32u) {
        const uint32_t k = f >> log2D, off = f & (D - 1u);
        unsigned mm = mask;
        for (uint32_t q = 0; q < k; ++q) mm &= mm - 1u;
        const uint32_t a = (base + uint32_t(__ffs(int(mm))) - 1u) * D;
        const uint32_t len = min(D, T - a);
        if (off == 0u || off >= len) continue;
        const uint32_t t = a + off;
        if (!mf_allowed<NX>(t, ex, T)) continue;
        mf_take(mf_score<M>(cx, cy, phase(s_tab, t, tl)), t, bs, bt);
      }
    }
  }
  __syncwarp();
  for (int off = 16; off; off >>= 1) {
    const float os = __shfl_xor_sync(0xffffffffu, bs, off);
    const uint32_t ot = __shfl_xor_sync(0xffffffffu, bt, off);
    mf_take(os, ot, bs, bt);
  }
  *best_s = bs;
  *best_t = bt;
}

// Lane l < m holds c_{l+1}; every lane gets all M (zero beyond m) in
// registers as duplicated pairs.
template <int M>
__device__ __forceinline__ void broadcast_c(float2 mine, float2 (&cx)[M], float2 (&cy)[M]) {
#pragma unroll
  for (int l = 0; l < M; ++l) {
    const float x = __shfl_sync(0xffffffffu, mine.x, l), y = __shfl_sync(0xffffffffu, mine.y, l);
    cx[l] = make_float2(x, x);
    cy[l] = make_float2(y, y);
  }
}

// Passes k .. K-1 of a pixel (lane l < m holds the residual r_l of the
// earlier passes, starting from z_l): subtract point k-1's fit, score
// conj(hhat) r, take the argmax outside the earlier points' exclusion zones.
template <int K, int M, int k>
__device__ __forceinline__ void later_passes(uint32_t lane, uint32_t m, uint32_t cnt, uint32_t T, float invT,
                                             const float2* s_tab, bool tl, const float2* s_wg, float* s_grid,
                                             uint32_t D, uint32_t G, const float2* s_hh, float E2, float prune_alpha,
                                             float min_sep, float2 r, float2 (&cx)[M], float2 (&cy)[M],
                                             float (&a)[K], float (&t)[K], uint32_t (&ti)[K], bool (&act)[K]) {
  if constexpr (k < K) {
    float2 mine = make_float2(0.f, 0.f);
    if (lane < m) {
      const float2 hv = s_hh[lane];
      const float2 e = phase(s_tab, mulmod(lane + 1u, ti[k - 1], T, invT), tl);
      const float f = (a[k - 1] >= prune_alpha) ? a[k - 1] : 0.f;
      const float2 fit = cmul(hv, e);
      r = make_float2(r.x - f * fit.x, r.y - f * fit.y);
      mine = cmul(make_float2(hv.x, -hv.y), r);
    }
    broadcast_c<M>(mine, cx, cy);
    __syncwarp();
    Excl<k> ex;
#pragma unroll
    for (int i = 0; i < k; ++i) ex.t[i] = ti[i];
    ex.min_sep = min_sep;
    ex.used = k;
    float sk;
    uint32_t tk;
    warp_argmax_scores<M, k>(mine, cx, cy, T, s_tab, tl, s_wg, s_grid, D, G, ex, &sk, &tk);
    if (tk >= T) {
      tk = 0u;
      sk = 0.f;
    }
    a[k] = fmaxf(0.f, sk / E2);
    t[k] = float(tk);
    ti[k] = tk;
    act[k] = (a[k] >= prune_alpha) && cnt > 0;
    later_passes<K, M, k + 1>(lane, m, cnt, T, invT, s_tab, tl, s_wg, s_grid, D, G, s_hh, E2, prune_alpha, min_sep,
                              r, cx, cy, a, t, ti, act);
  }
}

// Matched-filter initialisation of pixel p by one warp.
template <int K, int M>
__device__ __forceinline__ void init_pixel(uint32_t p, const float2* __restrict__ z, const uint32_t* __restrict__ n,
                                           uint32_t T, uint32_t m, const float2* s_tab, bool tl,
                                           const float2* s_wg, float* s_grid, uint32_t D, uint32_t G,
                                           const float2* s_hh, float E2, float prune_alpha, float min_sep,
                                           float* __restrict__ depth, float* __restrict__ alpha,
                                           uint8_t* __restrict__ active, float* __restrict__ alpha0) {
  const uint32_t lane = threadIdx.x & 31u;
  const float invT = 1.0f / float(T);
  const uint32_t cnt = n[p];
  float2 zl = make_float2(0.f, 0.f), mine = make_float2(0.f, 0.f);
  if (lane < m) {
    zl = z[size_t(p) * m + lane];
    mine = cmul(make_float2(s_hh[lane].x, -s_hh[lane].y), zl);
  }
  float2 cx[M], cy[M];
  broadcast_c<M>(mine, cx, cy);
  float s1;
  uint32_t t1;
  warp_argmax_scores<M, 0>(mine, cx, cy, T, s_tab, tl, s_wg, s_grid, D, G, Excl<0>{{0u}, 0.f, 0}, &s1, &t1);
  if (t1 >= T) {  // no finite score (cannot happen for finite z)
    t1 = 0u;
    s1 = 0.f;
  }
  float a[K], t[K];
  bool act[K];
  uint32_t ti[K];
  a[0] = fmaxf(0.f, s1 / E2);
  t[0] = float(t1);
  ti[0] = t1;
  act[0] = (a[0] >= prune_alpha) && cnt > 0;
  later_passes<K, M, 1>(lane, m, cnt, T, invT, s_tab, tl, s_wg, s_grid, D, G, s_hh, E2, prune_alpha, min_sep, zl,
                        cx, cy, a, t, ti, act);
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (!act[k]) a[k] = 0.f;
    sum += a[k];
  }
  if (sum > 1.f) {
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = a[k] / sum;
    sum = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) sum += a[k];
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      depth[size_t(p) * K + k] = t[k];
      alpha[size_t(p) * K + k] = a[k];
      active[size_t(p) * K + k] = act[k] ? 1 : 0;
    }
    alpha0[p] = 1.f - sum;
  }
  __syncwarp();
}

// One warp per pixel. Dynamic shared memory: the phase table, the coarse
// table e^{i 2 pi g D / T} (G entries) and one row of G grid scores per warp.
// Also folds the frame's largest photon count n_max (zeroed by the prep
// kernel) into misc[MISC_NMAX] for the iterations' step sizes.
template <int K, int M>
__global__ void __launch_bounds__(kBlock, M <= 12 ? 4 : 1) k_init(const float2* __restrict__ z, const uint32_t* __restrict__ n,
                                                 uint32_t P, uint32_t T, uint32_t m,
                                                 const float2* __restrict__ table, uint32_t entries,
                                                 int two_level, uint32_t D, const float2* __restrict__ hh_g,
                                                 float* __restrict__ misc, float prune_alpha, float min_sep,
                                                 float* __restrict__ depth, float* __restrict__ alpha,
                                                 uint8_t* __restrict__ active, float* __restrict__ alpha0) {
  extern __shared__ float2 s_tab[];
  __shared__ float2 s_hh[kMaxM];
  const uint32_t G = (T + D - 1u) / D;
  float2* s_wg = s_tab + entries;
  float* s_grid_all = reinterpret_cast<float*>(s_wg + G);
  if (threadIdx.x < m) s_hh[threadIdx.x] = hh_g[threadIdx.x];
  const bool tl = two_level != 0;
  for (uint32_t i = threadIdx.x; i < entries; i += blockDim.x) s_tab[i] = table[i];
  __syncthreads();
  for (uint32_t g = threadIdx.x; g < G; g += blockDim.x) s_wg[g] = phase(s_tab, g * D, tl);
  __syncthreads();
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t wpb = blockDim.x >> 5;
  const float E2 = misc[MISC_E2];
  uint32_t nmax = 0u;  // largest photon count seen by this warp
  for (uint32_t p = blockIdx.x * wpb + warp; p < P; p += gridDim.x * wpb) {
    nmax = max(nmax, n[p]);
    init_pixel<K, M>(p, z, n, T, m, s_tab, tl, s_wg, s_grid_all + warp * G, D, G, s_hh, E2, prune_alpha, min_sep,
                     depth, alpha, active, alpha0);
  }
  if ((threadIdx.x & 31u) == 0u) atomicMax(reinterpret_cast<unsigned*>(misc) + MISC_NMAX, nmax);
}

// Batched: items (frame, first pixel, last pixel); the CTA reloads the tables
// when the frame changes. Dynamic shared memory is sized for the largest
// frame of the batch, M for its largest m.
template <int K, int M>
__global__ void __launch_bounds__(kBlock, 1) k_init_batch(const BatchFrame* __restrict__ frames,
                                                       const uint3* __restrict__ items, uint32_t num_items,
                                                       uint32_t max_entries, uint32_t max_G, float prune_alpha,
                                                       float min_sep) {
  extern __shared__ float2 s_tab[];
  __shared__ float2 s_hh[kMaxM];
  float2* s_wg = s_tab + max_entries;
  float* s_grid_all = reinterpret_cast<float*>(s_wg + max_G);
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t wpb = blockDim.x >> 5;
  uint32_t cur = 0xffffffffu;
  for (uint32_t it = blockIdx.x; it < num_items; it += gridDim.x) {
    const uint3 item = items[it];
    const BatchFrame& f = frames[item.x];
    const uint32_t G = (f.T + f.D - 1u) / f.D;
    const bool tl = f.two_level != 0;
    if (item.x != cur) {
      __syncthreads();
      if (threadIdx.x < f.m) s_hh[threadIdx.x] = f.hh[threadIdx.x];
      for (uint32_t i = threadIdx.x; i < f.tab_entries; i += blockDim.x) s_tab[i] = f.table[i];
      __syncthreads();
      for (uint32_t g = threadIdx.x; g < G; g += blockDim.x) s_wg[g] = phase(s_tab, g * f.D, tl);
      __syncthreads();
      cur = item.x;
    }
    const float E2 = f.misc[MISC_E2];
    uint32_t nmax = 0u;
    for (uint32_t p = item.y + warp; p < item.z; p += wpb) {
      nmax = max(nmax, f.n[p]);
      init_pixel<K, M>(p, f.S, f.n, f.T, f.m, s_tab, tl, s_wg, s_grid_all + warp * max_G, f.D, G, s_hh, E2,
                       prune_alpha, min_sep, f.depth, f.alpha, f.active, f.alpha0);
    }
    if ((threadIdx.x & 31u) == 0u) atomicMax(reinterpret_cast<unsigned*>(f.misc) + MISC_NMAX, nmax);
  }
}

// Solves G x = y for the symmetric positive definite n x n system (n <= N)
// held in the leading rows of G, by elimination without pivoting (G is a
// Gram matrix of signatures at least min_sep apart, well conditioned).
template <int N>
__device__ __forceinline__ void solve_spd(float (&G)[N][N], float (&y)[N], int n) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (i >= n) break;
    const float inv = 1.f / G[i][i];
#pragma unroll
    for (int r = i + 1; r < N; ++r) {
      if (r >= n) break;
      const float f = G[r][i] * inv;
#pragma unroll
      for (int c = i; c < N; ++c) G[r][c] -= f * G[i][c];
      y[r] -= f * y[i];
    }
  }
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    if (i >= n) continue;
    float v = y[i];
#pragma unroll
    for (int c = i + 1; c < N; ++c)
      if (c < n) v -= G[i][c] * y[c];
    y[i] = v / G[i][i];
  }
}

__device__ __forceinline__ float warp_sum(float v) {
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// RT3D birth move on the sketched loss (a reading: RT3D's moves are cited,
// not stated, in Sec. 3) as one step of orthogonal matching pursuit, one warp
// per pixel with a free slot: the intensities beta of the active points are
// fitted to z by least squares at their current depths (lane l holds harmonic
// l's signatures hhat_l e^{i w_l t_k}, the phase of t_k from the table at its
// integer part times the fractional part's phasor; the Gram matrix and the
// right-hand side are warp sums), the residual's matched filter over integer
// t at circular distance >= min_sep from the nearest integer of every active
// depth takes its exact FP32 argmax t* (smallest t on ties) with the init's
// branch and bound, and the new point's intensity is its coefficient in the
// joint least-squares fit, alpha* = s(t*) / (sum |hhat|^2 - c^T G^-1 c), c_j
// = the correlation of the new signature with point j's. A point with
// alpha* >= prune_alpha is born in the first free slot (the others keep their
// intensities), and the pixel is rescaled if its intensities sum above 1. The
// state is updated in place.
template <int K, int M>
__global__ void __launch_bounds__(kBlock, 2) k_birth(const float2* __restrict__ z, const uint32_t* __restrict__ n,
                                                   uint32_t P, uint32_t T, uint32_t m,
                                                   const float2* __restrict__ table, uint32_t entries, int two_level,
                                                   uint32_t D, const float2* __restrict__ hh_g,
                                                   float* __restrict__ misc, float prune_alpha, float min_sep,
                                                   float* __restrict__ depth, float* __restrict__ alpha,
                                                   uint8_t* __restrict__ active, float* __restrict__ alpha0) {
  extern __shared__ float2 s_tab[];
  __shared__ float2 s_hh[kMaxM];
  const uint32_t G = (T + D - 1u) / D;
  float2* s_wg = s_tab + entries;
  float* s_grid_all = reinterpret_cast<float*>(s_wg + G);
  if (threadIdx.x < m) s_hh[threadIdx.x] = hh_g[threadIdx.x];
  const bool tl = two_level != 0;
  for (uint32_t i = threadIdx.x; i < entries; i += blockDim.x) s_tab[i] = table[i];
  __syncthreads();
  for (uint32_t g = threadIdx.x; g < G; g += blockDim.x) s_wg[g] = phase(s_tab, g * D, tl);
  __syncthreads();
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint32_t wpb = blockDim.x >> 5;
  const float E2 = misc[MISC_E2];
  const float invT = 1.0f / float(T);
  float* s_grid = s_grid_all + warp * G;
  for (uint32_t p = blockIdx.x * wpb + warp; p < P; p += gridDim.x * wpb) {
    float t[K], a[K];
    bool act[K];
    bool any_free = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      t[k] = depth[size_t(p) * K + k];
      a[k] = alpha[size_t(p) * K + k];
      act[k] = active[size_t(p) * K + k] != 0;
      any_free = any_free || !act[k];
    }
    if (!any_free || n[p] == 0u) continue;  // uniform over the warp
    // the active points' signatures, packed to the front (na of them)
    const bool lv = lane < m;
    const float2 hv = lv ? s_hh[lane] : make_float2(0.f, 0.f);
    const float2 zl = lv ? z[size_t(p) * m + lane] : make_float2(0.f, 0.f);
    float2 q[K];
    int na = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      q[k] = make_float2(0.f, 0.f);
      if (!act[k]) continue;
      float2 qk = make_float2(0.f, 0.f);
      if (lv) {
        const float fl = floorf(t[k]);
        const uint32_t ti = min(uint32_t(fl), T - 1u);
        float sf, cf;
        sincospif(2.f * float(lane + 1u) * (t[k] - fl) * invT, &sf, &cf);
        qk = cmul(hv, cmul(phase(s_tab, mulmod(lane + 1u, ti, T, invT), tl), make_float2(cf, sf)));
      }
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (j == na) q[j] = qk;
      ++na;
    }
    // least-squares intensities at the active depths: Gram matrix and
    // right-hand side as warp sums of Re(conj(q_j) q_k), Re(conj(q_j) z)
    constexpr int KA = K > 1 ? K - 1 : 1;  // at most K - 1 points are active here
    float Gm[KA][KA], beta[KA];
#pragma unroll
    for (int j = 0; j < KA; ++j) {
      beta[j] = warp_sum(q[j].x * zl.x + q[j].y * zl.y);
#pragma unroll
      for (int k = 0; k < KA; ++k)
        Gm[j][k] = (k >= j) ? warp_sum(q[j].x * q[k].x + q[j].y * q[k].y) : 0.f;
    }
#pragma unroll
    for (int j = 0; j < KA; ++j)
#pragma unroll
      for (int k = 0; k < j; ++k) Gm[j][k] = Gm[k][j];
    float Gc[KA][KA];
#pragma unroll
    for (int j = 0; j < KA; ++j)
#pragma unroll
      for (int k = 0; k < KA; ++k) Gc[j][k] = Gm[j][k];
    solve_spd<KA>(Gc, beta, na);
    float2 r = zl;
#pragma unroll
    for (int j = 0; j < KA; ++j)
      if (j < na) r = make_float2(r.x - beta[j] * q[j].x, r.y - beta[j] * q[j].y);
    const float2 mine = lv ? cmul(make_float2(hv.x, -hv.y), r) : make_float2(0.f, 0.f);
    float2 cx[M], cy[M];
    broadcast_c<M>(mine, cx, cy);
    __syncwarp();
    Excl<K> ex;
    ex.min_sep = min_sep;
    ex.used = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      ex.t[k] = 0u;
      if (act[k]) {
        uint32_t ti = uint32_t(floorf(t[k] + 0.5f));
        ti = ti >= T ? ti - T : ti;
#pragma unroll
        for (int j = 0; j < K; ++j)  // compact the active depths to the front
          if (j == ex.used) ex.t[j] = ti;
        ++ex.used;
      }
    }
    float sb;
    uint32_t tb;
    warp_argmax_scores<M, K>(mine, cx, cy, T, s_tab, tl, s_wg, s_grid, D, G, ex, &sb, &tb);
    if (tb < T) {
      // the new point's coefficient in the joint fit: s / (E2 - c^T G^-1 c)
      const float2 qs = lv ? cmul(hv, phase(s_tab, mulmod(lane + 1u, tb, T, invT), tl)) : make_float2(0.f, 0.f);
      float c[KA], y[KA];
#pragma unroll
      for (int j = 0; j < KA; ++j) y[j] = c[j] = warp_sum(q[j].x * qs.x + q[j].y * qs.y);
#pragma unroll
      for (int j = 0; j < KA; ++j)
#pragma unroll
        for (int k = 0; k < KA; ++k) Gc[j][k] = Gm[j][k];
      solve_spd<KA>(Gc, y, na);
      float den = E2;
#pragma unroll
      for (int j = 0; j < KA; ++j)
        if (j < na) den -= c[j] * y[j];
      const float an = den > 1e-6f * E2 ? fmaxf(0.f, sb / den) : 0.f;
      if (an >= prune_alpha) {
        bool placed = false;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (!act[k] && !placed) {
            t[k] = float(tb);
            a[k] = an;
            act[k] = true;
            placed = true;
          }
        }
      }
    }
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) sum += act[k] ? a[k] : 0.f;
    if (sum > 1.f) {
#pragma unroll
      for (int k = 0; k < K; ++k) a[k] = a[k] / sum;
      sum = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) sum += act[k] ? a[k] : 0.f;
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        depth[size_t(p) * K + k] = t[k];
        alpha[size_t(p) * K + k] = act[k] ? a[k] : 0.f;
        active[size_t(p) * K + k] = act[k] ? 1 : 0;
      }
      alpha0[p] = 1.f - sum;
    }
    __syncwarp();
  }
}

using InitFn = void (*)(const float2*, const uint32_t*, uint32_t, uint32_t, uint32_t, const float2*, uint32_t, int,
                        uint32_t, const float2*, float*, float, float, float*, float*, uint8_t*, float*);
using InitBatchFn = void (*)(const BatchFrame*, const uint3*, uint32_t, uint32_t, uint32_t, float, float);

template <int K>
InitFn init_fn(int M) {
  switch (M) {
#define CASE(k) \
  case k: return &k_init<K, k>;
    CASE(2) CASE(4) CASE(6) CASE(8) CASE(10) CASE(12) CASE(16) CASE(20) CASE(24) CASE(32)
#undef CASE
    default: return nullptr;
  }
}

template <int K>
InitFn birth_fn(int M) {
  switch (M) {
#define CASE(k) \
  case k: return &k_birth<K, k>;
    CASE(2) CASE(4) CASE(6) CASE(8) CASE(10) CASE(12) CASE(16) CASE(20) CASE(24) CASE(32)
#undef CASE
    default: return nullptr;
  }
}

template <int K>
InitBatchFn init_batch_fn(int M) {
  switch (M) {
#define CASE(k) \
  case k: return &k_init_batch<K, k>;
    CASE(2) CASE(4) CASE(6) CASE(8) CASE(10) CASE(12) CASE(16) CASE(20) CASE(24) CASE(32)
#undef CASE
    default: return nullptr;
  }
}

}  // namespace

int init_round_m(uint32_t m) {
  for (int k : kInitM)
    if (uint32_t(k) >= m) return k;
  return -1;
}

uint32_t mf_grid_spacing_host(uint32_t T, uint32_t m) { return mf_grid_spacing_impl(T, m); }

srt3d_status launch_init(srt3d_ctx* ctx, const float2* z, const uint32_t* n, uint32_t P, uint32_t T, uint32_t m,
                         uint32_t K, const PhaseTable& tab, const float2* hh, float* misc,
                         const srt3d_params& prm, float* depth, float* alpha, uint8_t* active, float* alpha0,
                         cudaStream_t stream) {
  const int M = init_round_m(m);
  InitFn fn = K == 1 ? init_fn<1>(M) : K == 2 ? init_fn<2>(M) : K == 3 ? init_fn<3>(M) : init_fn<4>(M);
  if (!fn) return set_error(ctx, SRT3D_EINVAL, "unsupported m");
  const uint32_t D = mf_grid_spacing_impl(T, m);
  const uint32_t G = (T + D - 1u) / D;
  const size_t smem = size_t(tab.entries) * sizeof(float2) + size_t(G) * sizeof(float2) +
                      size_t(kBlock / 32) * G * sizeof(float);
  // static + dynamic shared memory may exceed the 48 KB default
  SRT3D_CUDA_TRY(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  int bps = 0;
  SRT3D_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kBlock, smem));
  if (bps < 1) bps = 1;
  const uint32_t wpb = kBlock / 32;
  const uint64_t need = (uint64_t(P) + wpb - 1) / wpb;
  const uint32_t grid = uint32_t(std::min<uint64_t>(need, uint64_t(ctx->num_sms) * bps));
  const ProfMark mk = prof_begin(ctx, KID_INIT, stream);
  fn<<<grid, kBlock, smem, stream>>>(z, n, P, T, m, tab.dev, tab.entries, tab.two_level ? 1 : 0, D, hh, misc,
                                     prm.prune_alpha, prm.min_sep, depth, alpha, active, alpha0);
  prof_end(ctx, KID_INIT, mk, stream);
  SRT3D_CUDA_TRY(ctx, cudaGetLastError());
  return SRT3D_OK;
}

srt3d_status launch_birth(srt3d_ctx* ctx, const float2* z, const uint32_t* n, uint32_t P, uint32_t T, uint32_t m,
                          uint32_t K, const PhaseTable& tab, const float2* hh, const float* misc,
                          const srt3d_params& prm, float* depth, float* alpha, uint8_t* active, float* alpha0,
                          cudaStream_t stream) {
  const int M = init_round_m(m);
  InitFn fn = K == 1 ? birth_fn<1>(M) : K == 2 ? birth_fn<2>(M) : K == 3 ? birth_fn<3>(M) : birth_fn<4>(M);
  if (!fn) return set_error(ctx, SRT3D_EINVAL, "unsupported m");
  const uint32_t D = mf_grid_spacing_impl(T, m);
  const uint32_t G = (T + D - 1u) / D;
  const size_t smem = size_t(tab.entries) * sizeof(float2) + size_t(G) * sizeof(float2) +
                      size_t(kBlock / 32) * G * sizeof(float);
  SRT3D_CUDA_TRY(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  int bps = 0;
  SRT3D_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kBlock, smem));
  if (bps < 1) bps = 1;
  const uint32_t wpb = kBlock / 32;
  const uint64_t need = (uint64_t(P) + wpb - 1) / wpb;
  const uint32_t grid = uint32_t(std::min<uint64_t>(need, uint64_t(ctx->num_sms) * bps));
  const ProfMark mk = prof_begin(ctx, KID_BIRTH, stream);
  fn<<<grid, kBlock, smem, stream>>>(z, n, P, T, m, tab.dev, tab.entries, tab.two_level ? 1 : 0, D, hh,
                                     const_cast<float*>(misc), prm.prune_alpha, prm.min_sep, depth, alpha, active,
                                     alpha0);
  prof_end(ctx, KID_BIRTH, mk, stream);
  SRT3D_CUDA_TRY(ctx, cudaGetLastError());
  return SRT3D_OK;
}

srt3d_status launch_init_batch(srt3d_ctx* ctx, const BatchFrame* d_frames, const uint3* d_items,
                               uint32_t num_items, uint32_t K, int M, uint32_t max_entries, uint32_t max_G,
                               const srt3d_params& prm, cudaStream_t stream) {
  InitBatchFn fn = K == 1   ? init_batch_fn<1>(M)
                   : K == 2 ? init_batch_fn<2>(M)
                   : K == 3 ? init_batch_fn<3>(M)
                            : init_batch_fn<4>(M);
  if (!fn) return set_error(ctx, SRT3D_EINVAL, "unsupported m");
  const size_t smem = size_t(max_entries) * sizeof(float2) + size_t(max_G) * sizeof(float2) +
                      size_t(kBlock / 32) * max_G * sizeof(float);
  // static + dynamic shared memory may exceed the 48 KB default
  SRT3D_CUDA_TRY(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  int bps = 0;
  SRT3D_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kBlock, smem));
  if (bps < 1) bps = 1;
  const uint32_t grid = std::min<uint32_t>(num_items, uint32_t(ctx->num_sms) * uint32_t(bps));
  const ProfMark mk = prof_begin(ctx, KID_INIT, stream);
  fn<<<grid, kBlock, smem, stream>>>(d_frames, d_items, num_items, max_entries, max_G, prm.prune_alpha,
                                     prm.min_sep);
  prof_end(ctx, KID_INIT, mk, stream);
  SRT3D_CUDA_TRY(ctx, cudaGetLastError());
  return SRT3D_OK;
}

}  // namespace srt3d
