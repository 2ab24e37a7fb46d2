// Pieces shared by the two parquet assemblies (the general kernel in pq_vertex.cu and the
// tiled BF16 kernel in pq_assemble_tiled.cu).
#pragma once

#include <cmath>
#include <cstdint>

#include <cuda_fp16.h>

#include "pq_common.cuh"

namespace pq {

// Fully irreducible vertex: the parquet-approximation constants (U, -U, 2U, 0), and per
// channel an optional local table on |m| <= nl[r], n, n' in [-nl[r], nl[r] - 1] (Sec. III.A:
// Lambda from an impurity calculation, supplemented by the constants outside its box),
// laid out [m + nl][n + nl][n' + nl] in the arithmetic type of the assembly.
struct Lam {
  double2 l[4];
  const void *tab[4];
  int nl[4];
};

// Lambda_r at (m, n, n'); without tables (TAB false) the constant, at no cost.
template <bool TAB, typename C>
__device__ inline C lam_at(const Lam &lam, int r, C l_r, int m, int n, int np_) {
  if constexpr (TAB) {
    const int nl = lam.nl[r];
    if (lam.tab[r] && m >= -nl && m <= nl && n >= -nl && n < nl && np_ >= -nl && np_ < nl)
      return ((const C *)lam.tab[r])[((m + nl) * 2 * nl + (n + nl)) * 2 * nl + (np_ + nl)];
  }
  return l_r;
}

// Running complex sum in FP32 with its rounding error kept (Knuth's TwoSum on each part):
// s + c holds the sum of the terms added to about twice FP32 precision, which for FP32 terms
// is as accurate as an FP64 accumulator, without FP64 work per term (the FP64 pipe is narrow
// on this part).  The split assemblies add each step's partial dF sum into one.
struct CSum2 {
  float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
  __device__ static inline void two_sum(float &s, float &c, float x) {
    const float t = s + x, z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
  }
  __device__ inline void add(float2 v) {
    two_sum(sx, cx, v.x);
    two_sum(sy, cy, v.y);
  }
  __device__ inline double2 get() const { return make_double2((double)sx + (double)cx, (double)sy + (double)cy); }
};

// BF16 rounding (to nearest, ties to even) of finite FP32 values in integer arithmetic:
// the upper half of u + 0x7FFF + (bit 16 of u).  Identical to the hardware conversion,
// but it runs on the integer ALU instead of the conversion unit, which is narrow on this
// part and otherwise bounds the assembly.
__device__ inline uint32_t bf16_round(float x) {
  const uint32_t u = __float_as_uint(x);
  return u + 0x7FFFu + ((u >> 16) & 1u);
}

// FP16 pieces of two scaled values y0, y1 (|y| <= 2^15), packed as FP16x2 words with y0 in the
// low half: h = fp16(y) rounded to nearest, l = fp16(y - h).  y - h is exact in FP32 (h is y
// rounded to 11 leading bits), so y = h + l to 2^-22 |y| (plus the FP16 subnormal spacing,
// 2^-24, for the smallest values: below 2^-39 of the scale 2^15 the values are mapped to).
// The pack conversion runs at the ALU rate on this part.
__device__ inline uint32_t f16x2_pack(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ inline void f16_split2(float y0, float y1, uint32_t &h, uint32_t &l) {
  h = f16x2_pack(y0, y1);
  const float2 hv = __half22float2(*reinterpret_cast<const __half2 *>(&h));
  l = f16x2_pack(__fsub_rn(y0, hv.x), __fsub_rn(y1, hv.y));
}
// FP32 value of FP16 bits (normal, subnormal or zero).
__host__ __device__ inline float f16_value(uint32_t h) {
#ifdef __CUDA_ARCH__
  return __half2float(__ushort_as_half((unsigned short)h));
#else
  const uint32_t e = (h >> 10) & 0x1Fu, m = h & 0x3FFu;
  const float v = e ? std::ldexp((float)(1024u + m), (int)e - 25) : std::ldexp((float)m, -24);
  return (h & 0x8000u) ? -v : v;
#endif
}
}  // namespace pq
