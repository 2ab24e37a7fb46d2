// Pieces shared by the two parquet assemblies (the general kernel in pq_vertex.cu and the
// tiled BF16 kernel in pq_assemble_tiled.cu).
#pragma once

#include <cstdint>

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

// BF16 rounding (to nearest, ties to even) of finite FP32 values in integer arithmetic:
// the upper half of u + 0x7FFF + (bit 16 of u).  Identical to the hardware conversion,
// but it runs on the integer ALU instead of the conversion unit, which is narrow on this
// part and otherwise bounds the assembly.
__device__ inline uint32_t bf16_round(float x) {
  const uint32_t u = __float_as_uint(x);
  return u + 0x7FFFu + ((u >> 16) & 1u);
}

// FP16 pieces of a scaled value y (|y| <= 2^15), in FP32 and integer arithmetic only (the
// conversion unit is narrow on this part).  Veltkamp's splitting (Dekker 1971): with
// c = (2^13 + 1) y, the difference c - (c - y) is y rounded to its 11 leading bits, and the
// remainder y - hi is exact in FP32.  y = h + l with h and l such 11-bit values; both fit
// FP16 (11-bit significand), so their bit patterns follow by rebiasing the exponent.
// Pieces below 2^-14 (the FP16 normal range) are flushed to zero: the representation error
// is at most 2^-22 |y| + 2^-14, i.e. below 2^-29 of the scale 2^15 the values are mapped to.
// The intrinsics keep the compiler from contracting the split into an FMA.
__device__ inline float f16_lead(float y) {
  const float c = __fmul_rn(y, 8193.0f);
  return __fsub_rn(c, __fsub_rn(c, y));
}
// FP16 bits of v, which has at most 11 significant bits and |v| < 2^16; 0 below 2^-14.
__device__ inline uint32_t f16_bits(float v) {
  const uint32_t u = __float_as_uint(v), a = u & 0x7FFFFFFFu;
  const uint32_t mag = a < 0x38800000u ? 0u : (a >> 13) - 0x1C000u;
  return ((u >> 16) & 0x8000u) | mag;
}
// y = h + l: the FP16 bits of both pieces.
__device__ inline void f16_split(float y, uint32_t &h, uint32_t &l) {
  const float hv = f16_lead(y);
  h = f16_bits(hv);
  l = f16_bits(f16_lead(__fsub_rn(y, hv)));
}
// FP32 value of FP16 bits written by f16_bits (normal or zero).
__host__ __device__ inline float f16_value(uint32_t h) {
  const uint32_t a = h & 0x7FFFu;
  const uint32_t u = ((h & 0x8000u) << 16) | (a ? (a << 13) + 0x38000000u : 0u);
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  __builtin_memcpy(&f, &u, 4);
  return f;
#endif
}
}  // namespace pq
