// Device helpers shared by the kernels of libsrt3d.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace srt3d {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Packed FP32 pairs (one instruction for both components, each rounded as
// the scalar operation would be).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// A packed FP32 pair held in one 64-bit register (low half = first
// component), so packed operations need no operand marshalling.
using pf2 = unsigned long long;

__device__ __forceinline__ pf2 pk(float lo, float hi) {
  pf2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}

__device__ __forceinline__ float2 upk(pf2 v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}

__device__ __forceinline__ float pk_lo(pf2 v) { return __uint_as_float(static_cast<unsigned>(v)); }

__device__ __forceinline__ pf2 pfma(pf2 a, pf2 b, pf2 c) {
  pf2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ pf2 padd(pf2 a, pf2 b) {
  pf2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

__device__ __forceinline__ pf2 psub(pf2 a, pf2 b) {
  pf2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

__device__ __forceinline__ pf2 pmul(pf2 a, pf2 b) {
  pf2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// (j * x) mod T, exact for j * x < 2^24: the product is exact in float, the
// float quotient is within 1 of floor(j x / T), and one correction fixes it.
__device__ __forceinline__ uint32_t mulmod(uint32_t j, uint32_t x, uint32_t T, float invT) {
  const uint32_t a = j * x;
  const uint32_t q = __float2uint_rz(__uint2float_rn(a) * invT);
  int32_t r = int32_t(a) - int32_t(q * T);
  r += (r < 0) ? int32_t(T) : 0;
  r -= (r >= int32_t(T)) ? int32_t(T) : 0;
  return uint32_t(r);
}

// e^{i 2 pi k / T} from the phase table in shared memory (direct, or
// two-level lo[256] x hi[ceil(T/256)]).
__device__ __forceinline__ float2 phase(const float2* tab, uint32_t k, bool two_level) {
  if (!two_level) return tab[k];
  return cmul(tab[k & 255u], tab[256u + (k >> 8)]);
}

}  // namespace srt3d
