// One-particle steps of a parquet iteration: the Dyson equation
// (App. A, Eq. PA_Dyson), the bubbles G G of the Bethe-Salpeter equations
// (Eq. PA_F_Phi), the second-order self-energy Sigma~1 in imaginary time
// (Sec. II.B), the assembly and mixing of Sigma, and the susceptibility.
// All arithmetic here is FP64.
#include <algorithm>
#include <cstdio>

#include <cuda_bf16.h>

#include "pq_assemble.cuh"
#include "pq_common.cuh"
#include "pq_internal.h"

namespace pq {

namespace {

// c1 of Sigma ~ c1/(i nu) beyond the stored range: -nu Im Sigma at the two
// outer stored frequencies, averaged over them and over momenta.
__global__ void tail_c1_kernel(Grid g, const double2 *__restrict__ sigma, double *scal) {
  __shared__ double red[256];
  double s = 0.0;
  const double nlo = nu_of(g, g.e_lo), nhi = nu_of(g, g.e_hi);
  for (int ik = threadIdx.x; ik < g.nk; ik += blockDim.x) {
    s += -(nlo * sigma[(long long)ik * g.n_ext].y + nhi * sigma[(long long)ik * g.n_ext + g.n_ext - 1].y) * 0.5;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) scal[0] = red[0] / g.nk;
}

__device__ inline double2 sigma_at(const Grid &g, const double2 *sigma, double c1, int ik, int n) {
  if (n >= g.e_lo && n <= g.e_hi) return sigma[(long long)ik * g.n_ext + (n - g.e_lo)];
  return make_double2(0.0, -c1 / nu_of(g, n));  // c1 / (i nu)
}

// Dyson equation G = [G0^-1 - Sigma]^-1 on the table range.
// G on the table range; gtab32 (split paths) receives the FP32 rounding that their
// FP32 assembly uses, so it converts nothing per element.
__global__ void green_kernel(Grid g, const double2 *__restrict__ sigma, const double *__restrict__ scal,
                             double2 *__restrict__ gtab, float2 *__restrict__ gtab32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.nk * g.n_g) return;
  int ik = i / g.n_g, n = g.g_lo + i % g.n_g;
  double2 s = sigma_at(g, sigma, scal[0], ik, n);
  const double2 v = cinv(g0_inverse(g, ik, n) - s);
  gtab[i] = v;
  if (gtab32) gtab32[i] = make_float2((float)v.x, (float)v.y);
}

__device__ inline double2 gt(const Grid &g, const double2 *gtab, int ik, int n) {
  return gtab[(long long)ik * g.n_g + (n - g.g_lo)];
}

// X_ph(Q,k) = (T/N) G(k) G(k+q), X_pp(Q,k) = (T/N) G(k) G(q-k).  With xmax (FP16 planes), the
// largest |Re|, |Im| of the FP32 copies of X_ph and X_pp are accumulated into xmax[0], xmax[1]
// (float bits: for non-negative floats the integer order is the numeric order).
__global__ void bubbles_kernel(Grid g, const double2 *__restrict__ gtab, double2 *__restrict__ xph,
                               double2 *__restrict__ xpp, float2 *__restrict__ xph32, float2 *__restrict__ xpp32,
                               unsigned *__restrict__ xmax) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (xmax) {
    float mph = 0.f, mpp = 0.f;
    if (i < (long long)g.nQ * g.n) {
      const int Q = (int)(i / g.n), k = (int)(i % g.n);
      const int iq = Q / g.n_om, m = g.m_lo + Q % g.n_om;
      const int ik = k / g.n_nu, n = g.n_lo + k % g.n_nu;
      const double c = g.T / g.nk;
      const double2 gk = gt(g, gtab, ik, n);
      const double2 a = c * cmul(gk, gt(g, gtab, kadd(g, ik, iq), n + m));
      const double2 b = c * cmul(gk, gt(g, gtab, ksub(g, iq, ik), m - n - 1));
      const float2 a32 = make_float2((float)a.x, (float)a.y), b32 = make_float2((float)b.x, (float)b.y);
      xph[i] = a;
      xpp[i] = b;
      xph32[i] = a32;
      xpp32[i] = b32;
      mph = fmaxf(fabsf(a32.x), fabsf(a32.y));
      mpp = fmaxf(fabsf(b32.x), fabsf(b32.y));
    }
    for (int o = 16; o > 0; o >>= 1) {
      mph = fmaxf(mph, __shfl_xor_sync(0xffffffffu, mph, o));
      mpp = fmaxf(mpp, __shfl_xor_sync(0xffffffffu, mpp, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMax(&xmax[0], __float_as_uint(mph));
      atomicMax(&xmax[1], __float_as_uint(mpp));
    }
    return;
  }
  if (i >= (long long)g.nQ * g.n) return;
  int Q = (int)(i / g.n), k = (int)(i % g.n);
  int iq = Q / g.n_om, m = g.m_lo + Q % g.n_om;
  int ik = k / g.n_nu, n = g.n_lo + k % g.n_nu;
  double c = g.T / g.nk;
  double2 gk = gt(g, gtab, ik, n);
  const double2 a = c * cmul(gk, gt(g, gtab, kadd(g, ik, iq), n + m));
  const double2 b = c * cmul(gk, gt(g, gtab, ksub(g, iq, ik), m - n - 1));
  xph[i] = a;
  xpp[i] = b;
  if (xph32) {
    xph32[i] = make_float2((float)a.x, (float)a.y);
    xpp32[i] = make_float2((float)b.x, (float)b.y);
  }
}

// Power-of-two scales of the FP16 operand planes of one iteration (one thread).  Per channel r,
// bounds of |Re| and |Im| follow from the state's bounds p_x (max over Phi_x of |Re|, |Im|),
// the bubbles' bounds and those of Lambda: a parquet-equation lookup is a stored Phi_x or a
// fill K1 + K2row + K2col = (row mean) + (column mean) - K1, at most 3 p_x, so
//   |Gamma_r| <= lam_r + 3 sum_i |c_i^r| p_{x_i}   (Eqs. PA_Gamma_dm, PA_Gamma_st),
//   |F_r| <= |Gamma_r| + p_r,   |s_r Gamma_r X_r| <= |s_r| 2 |Gamma_r| xmax_r.
// The scale 2^e of each operand maps its bound into [2^14, 2^15), inside the FP16 range.
// The bounds of the next state and bubbles are then reset: the products and the bubbles of
// this iteration accumulate them.
__device__ inline float pow2_scale(float bound) {
  if (!(bound > 0.f) || !isfinite(bound)) return 1.f;
  int e;
  frexpf(bound, &e);  // bound = f 2^e, f in [0.5, 1)
  e = max(-100, min(100, 15 - e));
  return ldexpf(1.f, e);
}

struct Bound4 {
  float v[4];
};

__global__ void split_scales_kernel(float *fsc, Bound4 lam_max) {
  unsigned *u = (unsigned *)fsc;
  const float p[4] = {__uint_as_float(u[FSC_PHIMAX]), __uint_as_float(u[FSC_PHIMAX + 1]),
                      __uint_as_float(u[FSC_PHIMAX + 2]), __uint_as_float(u[FSC_PHIMAX + 3])};
  const float xm[2] = {__uint_as_float(u[FSC_XMAX]), __uint_as_float(u[FSC_XMAX + 1])};
  const float *lam = lam_max.v;
  // sum_i |c_i^r| p_{x_i} of the four crossed terms of each channel
  const float cp[4] = {0.5f * p[0] + 1.5f * p[1] + 0.5f * p[2] + 1.5f * p[3],
                       0.5f * (p[0] + p[1] + p[2] + p[3]),
                       p[0] + 3.0f * p[1],
                       p[0] + p[1]};
  const float s_abs[4] = {1.f, 1.f, 0.5f, 0.5f};
  for (int r = 0; r < 4; ++r) {
    const float gam = lam[r] + 3.0f * cp[r];
    const float sa = pow2_scale(s_abs[r] * 2.0f * gam * xm[r < 2 ? 0 : 1]);
    const float sb = pow2_scale(gam + p[r]);
    fsc[FSC_SA + r] = sa;
    fsc[FSC_SB + r] = sb;
    fsc[FSC_UNS + r] = 1.f / (sa * sb);
    u[FSC_PHIMAX + r] = 0u;
  }
  u[FSC_XMAX] = u[FSC_XMAX + 1] = 0u;
}

// Density per site (both spins) of G = [i nu + mu - eps_k - Sigma]^-1 on the square lattice, and
// its derivative in mu: n = (2/N) sum_k [1/2 - beta c2/4 + T sum_nu Re(G - 1/(i nu) - c2/(i nu)^2)]
// with c2 = eps_k - mu, the tails summed in closed form and the rest over n in [-M, M-1];
// dn/dmu = (2/N) sum_k [beta/4 + T sum_nu Re(-G^2 + 1/(i nu)^2)] (dG/dmu = -G^2).  Partial sums
// per block are added into out[0], out[1] (FP64 throughout).
__global__ void density_kernel(Grid g, int M, const double2 *__restrict__ sigma, const double *__restrict__ c1p,
                               double *__restrict__ out) {
  __shared__ double r0[256], r1[256];
  const long long total = (long long)g.nk * 2 * M;
  double a = 0.0, b = 0.0;
  const double c1 = c1p[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int ik = (int)(i / (2 * M)), n = (int)(i % (2 * M)) - M;
    const double nu = nu_of(g, n);
    const double2 s = sigma_at(g, sigma, c1, ik, n);
    const double2 gi = g0_inverse(g, ik, n) - s;  // i nu + mu - eps - Sigma
    const double2 G = cinv(gi);
    const double c2 = -(g0_inverse(g, ik, n).x);  // eps - mu
    // Re(1/(i nu)) = 0, Re(c2/(i nu)^2) = -c2/nu^2; Re(1/(i nu)^2) = -1/nu^2
    a += G.x + c2 / (nu * nu);
    b += -(G.x * G.x - G.y * G.y) - 1.0 / (nu * nu);
  }
  r0[threadIdx.x] = a;
  r1[threadIdx.x] = b;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      r0[threadIdx.x] += r0[threadIdx.x + w];
      r1[threadIdx.x] += r1[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(&out[0], r0[0]);
    atomicAdd(&out[1], r1[0]);
  }
}

// Tail moments of G = 1/(i nu) + c2/(i nu)^2 + c3/(i nu)^3 + O(nu^-4).
__device__ inline void tail_moments(const Grid &g, double c1, int ik, double &c2, double &c3) {
  if (g.lattice == 1) {
    int ix = ik / g.L, iy = ik % g.L;
    double a = -2.0 * g.hop * (cospi(2.0 * ix / g.L) + cospi(2.0 * iy / g.L)) - g.mu;
    c2 = a;
    c3 = a * a + c1;
  } else {
    c2 = 0.0;
    c3 = 0.25 * g.hop * g.hop + c1;
  }
}

// Matsubara remainders R(k, n) = G(k, n) - tails, n in [-M, M-1].
__global__ void s1_remainder_kernel(Grid g, int M, const double2 *__restrict__ sigma, const double *__restrict__ c1p,
                                    double2 *__restrict__ R) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.nk * 2 * M) return;
  int ik = i / (2 * M), n = -M + i % (2 * M);
  double c1 = c1p[0], c2, c3;
  tail_moments(g, c1, ik, c2, c3);
  double2 G = cinv(g0_inverse(g, ik, n) - sigma_at(g, sigma, c1, ik, n));
  double nu = nu_of(g, n);
  // 1/(i nu) = -i/nu; 1/(i nu)^2 = -1/nu^2; 1/(i nu)^3 = i/nu^3
  double2 tail = make_double2(-c2 / (nu * nu), -1.0 / nu + c3 / (nu * nu * nu));
  R[i] = G - tail;
}

// G(k, tau) += analytic transforms of the subtracted tails (0 < tau < beta):
// 1/(i nu) -> -1/2, 1/(i nu)^2 -> tau/2 - beta/4, 1/(i nu)^3 -> tau (beta - tau)/4.
__global__ void s1_tails_kernel(Grid g, int ntau, const double *__restrict__ tau, const double *__restrict__ c1p,
                                double2 *__restrict__ gkt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.nk * ntau) return;
  int ik = i / ntau, j = i % ntau;
  double c2, c3;
  tail_moments(g, c1p[0], ik, c2, c3);
  double t = tau[j], b = g.beta;
  gkt[i].x += -0.5 + c2 * (0.5 * t - 0.25 * b) + c3 * t * (b - t) * 0.25;
}

// Sigma(r, tau) = -U^2 G(r,tau)^2 G(-r,-tau) = U^2 G(r,tau)^2 G(-r, beta - tau);
// the nodes are symmetric about beta/2, so beta - tau_j is node ntau-1-j.
__global__ void s1_product_kernel(Grid g, int ntau, const double2 *__restrict__ grt, double2 *__restrict__ srt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.nk * ntau) return;
  int ir = i / ntau, j = i % ntau;
  double2 a = grt[i];
  double2 b = grt[(long long)kneg(g, ir) * ntau + (ntau - 1 - j)];
  srt[i] = (g.U * g.U) * cmul(cmul(a, a), b);
}

// Sigma_new = Sigma~1 + Sigma~2 + dF part; max |Sigma_new - Sigma|; Sigma <- mix.
__global__ void sigma_update_kernel(Grid g, const double2 *__restrict__ s1, const double2 *__restrict__ s2,
                                    const double2 *__restrict__ dfpart, double2 *__restrict__ sigma,
                                    double2 *__restrict__ sigma_new, double *scal) {
  __shared__ double red[256];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double d = 0.0;
  bool bad = false;
  if (i < g.nk * g.n_ext) {
    int ik = i / g.n_ext, n = g.e_lo + i % g.n_ext;
    double2 s = s1[i] + s2[i];
    if (n >= g.n_lo && n <= g.n_hi) {
      int k = ik * g.n_nu + (n - g.n_lo);
      for (int j = 0; j < g.nk; ++j) s = s + dfpart[(long long)k * g.nk + j];
    }
    double2 old = sigma[i];
    sigma_new[i] = s;
    d = sqrt(cabs2(s - old));
    bad = !(isfinite(s.x) && isfinite(s.y));
    sigma[i] = g.mix * s + (1.0 - g.mix) * old;
  }
  red[threadIdx.x] = bad ? 1e300 : d;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicMax((unsigned long long *)&scal[1], (unsigned long long)__double_as_longlong(red[0]));
    if (red[0] >= 1e300) scal[2] = 1.0;
  }
}

// Element e of the F operand buffer of the FP64 path.
__device__ inline double2 f_elem64(const void *fv, long long e) { return ((const double2 *)fv)[e]; }

// Element e of the F operand buffer of a split path in FP32: the complex64 value, or the sum
// of the three BF16 pieces (h + l is exact; adding r rounds once, at 2^-24 relative).
template <int FMT>
__device__ inline float2 f_elem32(const void *fv, long long ps, long long e, float inv_sb = 1.f) {
  if constexpr (FMT == V_C64) {
    return ((const float2 *)fv)[e];
  } else if constexpr (FMT == V_F16P) {
    // FP16 planes (Re h, Im h, Re l, Im l) of the scaled value: (h + l) / scale, exact in FP32
    const uint16_t *p = (const uint16_t *)fv;
    return make_float2((f16_value(p[e]) + f16_value(p[2 * ps + e])) * inv_sb,
                       (f16_value(p[ps + e]) + f16_value(p[3 * ps + e])) * inv_sb);
  } else {
    const uint16_t *p = (const uint16_t *)fv;
    auto bf = [&](long long i) { return __uint_as_float((uint32_t)p[i] << 16); };
    return make_float2((bf(e) + bf(2 * ps + e)) + bf(4 * ps + e), (bf(ps + e) + bf(3 * ps + e)) + bf(5 * ps + e));
  }
}

// Running FP32 sum with its rounding error kept (Knuth's TwoSum): s + c is the exact sum of
// the terms added, to about twice FP32 precision.
struct Sum2 {
  float s = 0.f, c = 0.f;
  __device__ inline void add(float x) {
    const float t = s + x, z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
  }
  __device__ inline void add(const Sum2 &o) {
    add(o.s);
    c += o.c;
  }
};

// chi_r(Q) = -sum_k X(k) - sum_{k,k'} X(k) F_r(Q)[k][k'] X(k') for the slices in the operand
// buffer (nq q-momenta from qb), in two deterministic stages: partial sums over blocks of
// CHI_ROWS rows (one warp per row at a time, lanes along k'), then their sum per (r, Q).
// FP64 path: FP64 throughout.  Split paths: the row sums sum_k' F X in FP32 products with
// compensated FP32 accumulation (no per-element work on the FP64 pipe, which is narrow on
// this part), each row's result then combined in FP64.
constexpr int CHI_ROWS = 64;

template <int FMT>
__global__ void chi_partial_kernel(Grid g, const void *__restrict__ fv, int ld, int qb, int nq, int q_chunk,
                                   const double2 *__restrict__ xph, const double2 *__restrict__ xpp,
                                   const float2 *__restrict__ xph32, const float2 *__restrict__ xpp32,
                                   double2 *__restrict__ part, const float *__restrict__ fsc) {
  __shared__ double2 red[8];
  const int chunk = blockIdx.x, Ql = blockIdx.y, r = blockIdx.z, Q = qb * g.n_om + Ql;
  const long long slabs = (long long)nq * g.n_om;                      // slices per channel in this pass
  const long long ps = 4LL * q_chunk * g.n_om * g.n * (long long)ld;   // plane stride of the buffer
  const double2 *X = (r < 2 ? xph : xpp) + (long long)Q * g.n;
  const long long base = ((long long)r * slabs + Ql) * g.n * (long long)ld;
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int k_end = min(g.n, (chunk + 1) * CHI_ROWS);
  double2 acc = make_double2(0.0, 0.0);
  for (int k = chunk * CHI_ROWS + warp; k < k_end; k += 8) {
    double2 rs;
    if constexpr (FMT == V_C128) {
      rs = make_double2(0.0, 0.0);
      for (int kp = lane; kp < g.n; kp += 32) rs = cfma(f_elem64(fv, base + (long long)k * ld + kp), X[kp], rs);
      for (int o = 16; o > 0; o >>= 1)
        rs = make_double2(rs.x + __shfl_xor_sync(0xffffffffu, rs.x, o), rs.y + __shfl_xor_sync(0xffffffffu, rs.y, o));
    } else {
      const float2 *X32 = (r < 2 ? xph32 : xpp32) + (long long)Q * g.n;
      const float inv_sb = FMT == V_F16P ? 1.f / fsc[FSC_SB + r] : 1.f;
      Sum2 re, im;
      for (int kp = lane; kp < g.n; kp += 32) {
        const float2 f = f_elem32<FMT>(fv, ps, base + (long long)k * ld + kp, inv_sb), x = X32[kp];
        re.add(fmaf(f.x, x.x, -f.y * x.y));
        im.add(fmaf(f.x, x.y, f.y * x.x));
      }
      for (int o = 16; o > 0; o >>= 1) {
        Sum2 ore, oim;
        ore.s = __shfl_xor_sync(0xffffffffu, re.s, o), ore.c = __shfl_xor_sync(0xffffffffu, re.c, o);
        oim.s = __shfl_xor_sync(0xffffffffu, im.s, o), oim.c = __shfl_xor_sync(0xffffffffu, im.c, o);
        re.add(ore);
        im.add(oim);
      }
      rs = make_double2((double)re.s + (double)re.c, (double)im.s + (double)im.c);
    }
    if (lane == 0) acc = acc + cfma(X[k], rs, X[k]);
  }
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = red[0];
    for (int w = 1; w < 8; ++w) t = t + red[w];
    part[((long long)r * slabs + Ql) * gridDim.x + chunk] = t;
  }
}

__global__ void chi_sum_kernel(Grid g, int qb, int nq, int nchunk, const double2 *__restrict__ part,
                               double2 *__restrict__ chi) {
  const long long slabs = (long long)nq * g.n_om;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= 4 * slabs) return;
  const int r = (int)(i / slabs), Ql = (int)(i % slabs);
  double2 t = make_double2(0.0, 0.0);
  for (int c = 0; c < nchunk; ++c) t = t + part[i * nchunk + c];
  chi[(long long)r * g.nQ + qb * g.n_om + Ql] = make_double2(-t.x, -t.y);
}

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// Truncated Schwinger-Dyson scheme (the ablation of the regulated Sigma, Sec. II.B): Eq.
// PA_Sigma on the box with the vertex cut off there.  Its F - Lambda^0 part is the box sum the
// assembly accumulates; the Lambda^0 = (U, -U, 2U, 0) part factorises through the bubbles:
//   -(U/4)(T/N)^2 2U sum_{k',q in box} [G(k+q) G(k'+q) G(k') + G(q-k') G(q-k) G(k')]
//     = -(U^2/2)(T/N) sum_Q [G(k+q) S_ph(Q) + G(q-k) S_pp(Q)],   S_x(Q) = sum_{k' in box} X_x(Q,k'),
// for k in the box; zero outside it.  One block per Q for the row sums, then one thread per output.
__global__ void box_bubble_sums(Grid g, const double2 *__restrict__ xph, const double2 *__restrict__ xpp,
                                double2 *__restrict__ sph, double2 *__restrict__ spp) {
  __shared__ double2 ra[256], rb[256];
  const int Q = blockIdx.x;
  double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
  for (int k = threadIdx.x; k < g.n; k += blockDim.x) {
    a = a + xph[(long long)Q * g.n + k];
    b = b + xpp[(long long)Q * g.n + k];
  }
  ra[threadIdx.x] = a;
  rb[threadIdx.x] = b;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      ra[threadIdx.x] = ra[threadIdx.x] + ra[threadIdx.x + w];
      rb[threadIdx.x] = rb[threadIdx.x] + rb[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sph[Q] = ra[0];
    spp[Q] = rb[0];
  }
}

__global__ void sigma_box_lambda0(Grid g, const double2 *__restrict__ gtab, const double2 *__restrict__ sph,
                                  const double2 *__restrict__ spp, double2 *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.nk * g.n_ext) return;
  const int ik = i / g.n_ext, n = g.e_lo + i % g.n_ext;
  double2 s = make_double2(0.0, 0.0);
  if (n >= g.n_lo && n <= g.n_hi) {
    for (int Q = 0; Q < g.nQ; ++Q) {
      const int iq = Q / g.n_om, m = g.m_lo + Q % g.n_om;
      const double2 gkq = gtab[(long long)kadd(g, ik, iq) * g.n_g + (n + m - g.g_lo)];
      const double2 gqk = gtab[(long long)ksub(g, iq, ik) * g.n_g + (m - n - 1 - g.g_lo)];
      s = cfma(gkq, sph[Q], cfma(gqk, spp[Q], s));
    }
    s = (-0.5 * g.U * g.U * g.T / g.nk) * s;
  }
  out[i] = s;
}



}  // namespace

cudaError_t launch_tail_and_green(cudaStream_t st, const Grid &g, Buffers &b) {
  tail_c1_kernel<<<1, 256, 0, st>>>(g, b.sigma, b.scal);
  green_kernel<<<nblk((long long)g.nk * g.n_g, 256), 256, 0, st>>>(g, b.sigma, b.scal, b.gtab, b.gtab32);
  return cudaGetLastError();
}

cudaError_t launch_bubbles(cudaStream_t st, const Grid &g, Buffers &b) {
  unsigned *xmax = b.vfmt == V_F16P ? (unsigned *)(b.fsc + FSC_XMAX) : nullptr;
  bubbles_kernel<<<nblk((long long)g.nQ * g.n, 256), 256, 0, st>>>(g, b.gtab, b.xph, b.xpp, b.xph32, b.xpp32, xmax);
  return cudaGetLastError();
}

cudaError_t launch_density(cudaStream_t st, const Grid &g, int M, const double2 *sigma, const double *c1,
                           double *out2) {
  cudaError_t e = cudaMemsetAsync(out2, 0, 2 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  const long long total = (long long)g.nk * 2 * M;
  density_kernel<<<(unsigned)std::min<long long>((total + 255) / 256, 1024), 256, 0, st>>>(g, M, sigma, c1, out2);
  return cudaGetLastError();
}

cudaError_t launch_split_scales(cudaStream_t st, Buffers &b, const double *lam_max) {
  Bound4 lm;
  for (int r = 0; r < 4; ++r) lm.v[r] = (float)lam_max[r];
  split_scales_kernel<<<1, 1, 0, st>>>(b.fsc, lm);
  return cudaGetLastError();
}

Sigma1Args sigma1_args(Buffers &b, const double2 *sigma, double *c1, double2 *out) {
  Sigma1Args a;
  a.sigma = sigma;
  a.c1 = c1;
  a.out = out;
  a.R = b.s1_R;
  a.gkt = b.s1_gkt;
  a.grt = b.s1_grt;
  a.srn = b.s1_srn;
  a.E = b.s1_E;
  a.Ef = b.s1_Ef;
  a.ph = b.s1_ph;
  a.phc = b.s1_phc;
  a.tau = b.s1_tau;
  a.work = b.gemm_work;
  a.work_elems = b.gemm_work_elems;
  return a;
}

// E[a][j] = exp(-i nu_a tau_j), nu_a = (2 (a - M) + 1) pi / beta for a in [0, 2M): the Matsubara-
// to-imaginary-time transform of Sigma~1 (tau_j the quadrature nodes), computed where it is used
// instead of on the host (4 M x N_tau complex exponentials).
__global__ void e_table_kernel(double2 *E, const double *tau, int two_m, int ntau, double beta) {
  const long long total = (long long)two_m * ntau;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(i / ntau), j = (int)(i - (long long)a * ntau);
    const double nu = (2.0 * (a - two_m / 2) + 1.0) * CUDART_PI / beta;
    double sn, cs;
    sincos(-nu * tau[j], &sn, &cs);
    E[i] = make_double2(cs, sn);
  }
}

cudaError_t launch_e_table(cudaStream_t st, double2 *E, const double *tau, int two_m, int ntau, double beta) {
  e_table_kernel<<<1216, 256, 0, st>>>(E, tau, two_m, ntau, beta);
  return cudaGetLastError();
}

cudaError_t launch_tail_c1(cudaStream_t st, const Grid &g, const double2 *sigma, double *c1) {
  tail_c1_kernel<<<1, 256, 0, st>>>(g, sigma, c1);
  return cudaGetLastError();
}

// Sigma~1 from the given self-energy (its tail coefficient c1 already in a.c1):
// R = G - tails; G(k,tau) = T R E + tails(tau); G(r,tau) = ph G(k,tau);
// Sigma(r,tau) = U^2 G(r,tau)^2 G(-r,beta-tau); Sigma(r,nu) = Sigma(r,tau) Ef; Sigma~1 = phc Sigma(r,nu).
cudaError_t launch_sigma1(cudaStream_t st, const Grid &g, const Sizes &z, const Sigma1Args &a) {
  const int M = z.M, nt = z.ntau;
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  s1_remainder_kernel<<<nblk((long long)g.nk * 2 * M, 256), 256, 0, st>>>(g, M, a.sigma, a.c1, a.R);
  cudaError_t e = zgemm_fp64_splitk(st, g.nk, nt, 2 * M, make_double2(g.T, 0.0), a.R, 2 * M, a.E, nt, zero, a.gkt,
                                    nt, a.work, a.work_elems);
  if (e != cudaSuccess) return e;
  s1_tails_kernel<<<nblk((long long)g.nk * nt, 256), 256, 0, st>>>(g, nt, a.tau, a.c1, a.gkt);
  e = zgemm_fp64_splitk(st, g.nk, nt, g.nk, one, a.ph, g.nk, a.gkt, nt, zero, a.grt, nt, a.work, a.work_elems);
  if (e != cudaSuccess) return e;
  s1_product_kernel<<<nblk((long long)g.nk * nt, 256), 256, 0, st>>>(g, nt, a.grt, a.gkt);
  e = zgemm_fp64_splitk(st, g.nk, g.n_ext, nt, one, a.gkt, nt, a.Ef, g.n_ext, zero, a.srn, g.n_ext, a.work,
                        a.work_elems);
  if (e != cudaSuccess) return e;
  e = zgemm_fp64_splitk(st, g.nk, g.n_ext, g.nk, one, a.phc, g.nk, a.srn, g.n_ext, zero, a.out, g.n_ext, a.work,
                        a.work_elems);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_sigma_truncated(cudaStream_t st, const Grid &g, Buffers &b) {
  // S_ph, S_pp in the chi partial-sum scratch (4 N_Q n / CHI_ROWS >= 2 N_Q entries)
  if (b.chi_part_elems < 2LL * g.nQ) return cudaErrorInvalidValue;
  double2 *sph = b.chi_part, *spp = b.chi_part + g.nQ;
  cudaError_t e = cudaMemsetAsync(b.sigma1, 0, sizeof(double2) * (size_t)g.nk * g.n_ext, st);
  if (e != cudaSuccess) return e;
  box_bubble_sums<<<g.nQ, 256, 0, st>>>(g, b.xph, b.xpp, sph, spp);
  sigma_box_lambda0<<<nblk((long long)g.nk * g.n_ext, 256), 256, 0, st>>>(g, b.gtab, sph, spp, b.sigma2);
  return cudaGetLastError();
}

cudaError_t launch_sigma_update(cudaStream_t st, const Grid &g, Buffers &b) {
  cudaMemsetAsync(b.scal + 1, 0, 2 * sizeof(double), st);
  sigma_update_kernel<<<nblk((long long)g.nk * g.n_ext, 256), 256, 0, st>>>(g, b.sigma1, b.sigma2, b.dfpart,
                                                                            b.sigma, b.sigma_new, b.scal);
  return cudaGetLastError();
}

cudaError_t launch_chi(cudaStream_t st, const Grid &g, Buffers &b, int qb, int nq) {
  const int nchunk = (g.n + CHI_ROWS - 1) / CHI_ROWS;
  const long long slabs = (long long)nq * g.n_om;
  if (4 * slabs * nchunk > b.chi_part_elems) return cudaErrorInvalidValue;
  dim3 grid(nchunk, (unsigned)slabs, 4);
  if (b.vfmt == V_C128)
    chi_partial_kernel<V_C128><<<grid, 256, 0, st>>>(g, b.fv, b.ld, qb, nq, b.q_chunk, b.xph, b.xpp, nullptr, nullptr,
                                                     b.chi_part, b.fsc);
  else if (b.vfmt == V_C64)
    chi_partial_kernel<V_C64><<<grid, 256, 0, st>>>(g, b.fv, b.ld, qb, nq, b.q_chunk, b.xph, b.xpp, b.xph32, b.xpp32,
                                                    b.chi_part, b.fsc);
  else if (b.vfmt == V_F16P)
    chi_partial_kernel<V_F16P><<<grid, 256, 0, st>>>(g, b.fv, b.ld, qb, nq, b.q_chunk, b.xph, b.xpp, b.xph32,
                                                     b.xpp32, b.chi_part, b.fsc);
  else
    chi_partial_kernel<V_BF16P><<<grid, 256, 0, st>>>(g, b.fv, b.ld, qb, nq, b.q_chunk, b.xph, b.xpp, b.xph32,
                                                      b.xpp32, b.chi_part, b.fsc);
  chi_sum_kernel<<<nblk(4 * slabs, 256), 256, 0, st>>>(g, qb, nq, nchunk, b.chi_part, b.chi);
  return cudaGetLastError();
}

}  // namespace pq
