// Shared device types of the GB300 parquet solver: the grid of one solve,
// complex arithmetic on float2/double2, and the index conventions of the
// paper's compound arguments k = (k-vector, i nu_n), q = (q-vector, i w_m)
// (App. A, "Notations").
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <math_constants.h>

namespace pq {

// One solve's grids.  Fermionic box n in [n_lo, n_hi], bosonic box
// m in [m_lo, m_hi]; the self-energy lives on [e_lo, e_hi]; the kernel-term
// sums of Sigma~2 run over fermionic [bf_lo, bf_hi] and bosonic
// [bb_lo, bb_hi]; the G table covers [g_lo, g_lo + n_g - 1].
struct Grid {
  int lattice;  // 0 Bethe, 1 square
  int L, nk, n_nu, n_om, n, nQ, n_ext;
  int n_lo, n_hi, m_lo, m_hi, e_lo, e_hi;
  int bf_lo, bf_hi, bb_lo, bb_hi;
  int g_lo, n_g;
  double beta, T, U, mu, hop, mix;
};

__host__ __device__ inline int kadd(const Grid &g, int a, int b) {
  int L = g.L;
  int x = a / L + b / L, y = a % L + b % L;
  if (x >= L) x -= L;
  if (y >= L) y -= L;
  return x * L + y;
}
__host__ __device__ inline int kneg(const Grid &g, int a) {
  int L = g.L;
  int x = a / L, y = a % L;
  x = x ? L - x : 0;
  y = y ? L - y : 0;
  return x * L + y;
}
__host__ __device__ inline int ksub(const Grid &g, int a, int b) { return kadd(g, a, kneg(g, b)); }

__host__ __device__ inline double nu_of(const Grid &g, int n) { return (2.0 * n + 1.0) * CUDART_PI / g.beta; }

// ---------------------------------------------------------------- complex
__host__ __device__ inline double2 cmk(double a, double b) { return make_double2(a, b); }
__host__ __device__ inline double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cfma(double2 a, double2 b, double2 c) {  // a*b + c
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__host__ __device__ inline double2 cinv(double2 a) {
  double d = 1.0 / (a.x * a.x + a.y * a.y);
  return make_double2(a.x * d, -a.y * d);
}
__host__ __device__ inline double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

__host__ __device__ inline float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__host__ __device__ inline float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline float2 cfma(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}

// Storage <-> compute conversions.
template <typename S, typename C> __device__ inline C to_c(S v);
template <> __device__ inline double2 to_c<double2, double2>(double2 v) { return v; }
template <> __device__ inline float2 to_c<float2, float2>(float2 v) { return v; }
template <> __device__ inline float2 to_c<double2, float2>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}
template <> __device__ inline double2 to_c<float2, double2>(float2 v) { return make_double2(v.x, v.y); }

// Inverse bare propagator: square lattice i nu + mu - eps_k; Bethe lattice the
// inverse of the semicircular Hilbert transform (2/D^2)(i nu - i sgn(nu) sqrt(nu^2 + D^2)).
__device__ inline double2 g0_inverse(const Grid &g, int ik, int n) {
  double nu = nu_of(g, n);
  if (g.lattice == 1) {
    int ix = ik / g.L, iy = ik % g.L;
    double eps = -2.0 * g.hop * (cospi(2.0 * ix / g.L) + cospi(2.0 * iy / g.L));
    return make_double2(g.mu - eps, nu);
  }
  double D = g.hop;
  double s = nu > 0 ? 1.0 : -1.0;
  double im = (2.0 / (D * D)) * (nu - s * sqrt(nu * nu + D * D));  // G0 = i*im
  return make_double2(0.0, -1.0 / im);
}

}  // namespace pq
