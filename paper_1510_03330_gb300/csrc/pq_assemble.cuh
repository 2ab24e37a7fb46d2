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
}  // namespace pq
