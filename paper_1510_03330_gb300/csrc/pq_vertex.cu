// Vertex steps of a parquet iteration:
//  * kernel functions K1, K2 of the reducible vertex (Sec. II.A: first level at
//    the four corners of the frequency box, second level at the two frequency
//    edges of the other leg, momentum averaged);
//  * the parquet equations Gamma_r = Lambda_r + sum_i c_i Phi[crossed args]
//    with the kernel fill (Eq. PA_F; App. A, Eqs. PA_Gamma_dm, PA_Gamma_st),
//    F_r = Gamma_r + Phi_r (Eq. PA_F_G), the BSE left operand
//    s_r Gamma_r diag(X_r) (Eq. PA_F_Phi), and the box sum of Eq. PA_Sigma over
//    F - Lambda^0 used by the regulated self-energy (Sec. II.B).
//
// The crossed arguments are gathers across transfer slices.  For a fixed row
// leg k every crossed map is an affine permutation of the (Q, k') plane of row
// k, so one CTA per (k, k'-momentum) walks the q-momenta and, per step, loads
// six frequency blocks [m~][n_c] (NOmega x Nnu each, coalesced along n_c):
//   R_x = Phi_x[(k'-k, .)][k][(k+q, .)]   x = d, m   (maps A and C)
//   P_x = Phi_x[(q, .)][k][(k', .)]        x = d, m   (own d/m, map D)
//   S_x = Psi_x[(q', .)][k][(k', .)]       x = s, t   (map B, own s/t)
// with q' = k + k' + q, and writes the d/m outputs at transfer q and the s/t
// outputs at transfer q'.  Every element of Phi is read exactly once.
#include <cuda_bf16.h>

#include "pq_common.cuh"
#include "pq_assemble.cuh"
#include "pq_internal.h"

namespace pq {

namespace {

// Running sum of edge values: FP64 for the FP64 path; for the complex64 path a compensated
// FP32 sum (Knuth's TwoSum: s + c holds the running sum to about twice FP32 precision), so
// that no element is converted or added on the FP64 pipe, which is narrow on this part.
template <typename S>
struct EdgeSum {
  double2 v = make_double2(0.0, 0.0);
  __device__ inline void add(S x) { v = v + to_c<S, double2>(x); }
  __device__ inline double2 get() const { return v; }
};
template <>
struct EdgeSum<float2> {
  float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
  __device__ static inline void two_sum(float &s, float &c, float x) {
    const float t = s + x, z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
  }
  __device__ inline void add(float2 x) {
    two_sum(sx, cx, x.x);
    two_sum(sy, cy, x.y);
  }
  __device__ inline double2 get() const { return make_double2((double)sx + (double)cx, (double)sy + (double)cy); }
};

// K1[r][Q], K2row[r][k][Q], K2col[r][k'][Q]; one block per (Q, r).
// ROWSUM: the row-edge sums of K2row come from krow ([r][k][Q], accumulated by the BSE
// epilogue that wrote this Phi) instead of strided reads of Phi.
// Ablations of Sec. II.A: lower_edge takes the lower frequency edge of the other leg alone
// (K1: the corner at the lower edges of both legs); first_level keeps K1 only (K2 = 0).
template <typename S, bool ROWSUM>
__global__ void kernels_kernel(Grid g, const S *__restrict__ phi, double2 *__restrict__ k1,
                               double2 *__restrict__ k2row, double2 *__restrict__ k2col,
                               const double2 *__restrict__ krow, bool lower_edge, bool first_level) {
  __shared__ double2 red[256];
  __shared__ double2 sk1;
  const int Q = blockIdx.x, r = blockIdx.y;
  const long long n = g.n;
  const S *V = phi + ((long long)r * g.nQ + Q) * n * n;
  const int nn = g.n_nu, nk = g.nk;
  const int ne = lower_edge ? 1 : 2;  // frequency edges averaged
  const double inv = 1.0 / ((double)ne * nk);
  double2 *K2r = k2row + (long long)r * g.n * g.nQ + Q, *K2c = k2col + (long long)r * g.n * g.nQ + Q;
  // edge means of the other leg (momentum averaged), kept until K1 is known; the first level
  // is their mean over the edge columns, i.e. over the four corners and all momentum pairs
  double2 acc = make_double2(0.0, 0.0);
  for (int k = threadIdx.x; k < g.n; k += blockDim.x) {
    double2 rs, cs;
    EdgeSum<S> es_r, es_c;
    if constexpr (ROWSUM) {
      rs = krow[((long long)r * g.n + k) * g.nQ + Q];
#pragma unroll 8
      for (int b = 0; b < nk; ++b) {
        es_c.add(V[(long long)(b * nn) * n + k]);
        es_c.add(V[(long long)(b * nn + nn - 1) * n + k]);
      }
    } else {
      // unrolled so that the loads of several momentum blocks are in flight together
#pragma unroll 8
      for (int b = 0; b < nk; ++b) {
        es_r.add(V[k * n + b * nn]);
        es_c.add(V[(long long)(b * nn) * n + k]);
        if (!lower_edge) {
          es_r.add(V[k * n + b * nn + nn - 1]);
          es_c.add(V[(long long)(b * nn + nn - 1) * n + k]);
        }
      }
      rs = es_r.get();
    }
    cs = es_c.get();
    K2r[(long long)k * g.nQ] = inv * rs;
    K2c[(long long)k * g.nQ] = inv * cs;
    const int f = k % nn;
    if (f == 0 || (!lower_edge && f == nn - 1)) acc = acc + cs;  // corners: edge rows x edge columns
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sk1 = (1.0 / ((double)ne * ne * nk * nk)) * red[0];
    k1[(long long)r * g.nQ + Q] = sk1;
  }
  __syncthreads();
  const double2 K1 = sk1;
  for (int k = threadIdx.x; k < g.n; k += blockDim.x) {
    const double2 z = make_double2(0.0, 0.0);
    K2r[(long long)k * g.nQ] = first_level ? z : K2r[(long long)k * g.nQ] - K1;
    K2c[(long long)k * g.nQ] = first_level ? z : K2c[(long long)k * g.nQ] - K1;
  }
}

template <typename C> __device__ inline C cz();
template <> __device__ inline double2 cz<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ inline float2 cz<float2>() { return make_float2(0.f, 0.f); }
template <typename C> __device__ inline C cfrom(double2 v);
template <> __device__ inline double2 cfrom<double2>(double2 v) { return v; }
template <> __device__ inline float2 cfrom<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <typename C> __device__ inline double2 cdbl(C v);
template <> __device__ inline double2 cdbl<double2>(double2 v) { return v; }
template <> __device__ inline double2 cdbl<float2>(float2 v) { return make_double2(v.x, v.y); }

// The dF box sum of a thread across the gather steps: in FP64 the accumulator itself; in the
// FP32 (split) paths each step's partial sum is moved into a compensated sum (CSum2), so the
// sum over all transfers keeps FP64-grade accuracy.
template <typename C>
struct DfSum {
  __device__ inline void step(C &) {}
  __device__ inline double2 get(const C &acc) const { return cdbl<C>(acc); }
};
template <>
struct DfSum<float2> {
  CSum2 s;
  __device__ inline void step(float2 &acc) {
    s.add(acc);
    acc = make_float2(0.f, 0.f);
  }
  __device__ inline double2 get(const float2 &) const { return s.get(); }
};

// (k', k'+1) values -> packed BF16 pair (k' in the low half) and the FP32 remainders
__device__ inline uint32_t split_pair(float x0, float x1, float &r0, float &r1) {
  const uint32_t a = bf16_round(x0), b = bf16_round(x1);
  r0 = x0 - __uint_as_float(a & 0xFFFF0000u);
  r1 = x1 - __uint_as_float(b & 0xFFFF0000u);
  return __byte_perm(a, b, 0x7632);
}
__device__ inline uint32_t pack_pair(float x0, float x1) {
  return __byte_perm(bf16_round(x0), bf16_round(x1), 0x7632);
}

// Output of the BSE operands.  Lanes 2j and 2j+1 of a warp always hold consecutive
// columns k', k'+1 of one row (Nnu is even and the element index has the lane's parity),
// so each pair shares its stores: one shuffle gives the even lane both elements' real
// parts and the odd lane both imaginary parts, and each writes its half as 4-byte BF16
// pairs (split planes), or, for complex64, the even lane writes the pair's Gamma X and
// the odd lane its F as 16-byte stores.
//
// BF16 planes: x = h + l (+ r for F), each piece the BF16 rounding of what the previous
// pieces leave (the differences are exact in FP32).  Plane order: Gamma X (Re h, Re l,
// Im h, Im l), F (Re h, Im h, Re l, Im l, Re r, Im r).  FP16 planes: the channel's scaled
// value x * 2^e = h + l (f16_split2), planes Gamma X (Re h, Re l, Im h, Im l), F (Re h, Im h,
// Re l, Im l).
template <typename S, int PL>
struct Out {
  void *gam, *fv;
  long long ps;  // plane stride in elements (PL)
  // element o of this lane (o is even on even lanes, odd on odd lanes); sa, sb: the scales of
  // Gamma X and F (FP16 planes)
  __device__ inline void put(long long o, float2 ga, float2 f, float sa = 1.f, float sb = 1.f) const {
    const unsigned mask = __activemask();
    const bool odd = threadIdx.x & 1;
    // even lanes send Im, odd lanes send Re: each receives the partner's half it stores
    const float ga_in = __shfl_xor_sync(mask, odd ? ga.x : ga.y, 1);
    const float f_in = __shfl_xor_sync(mask, odd ? f.x : f.y, 1);
    const long long o2 = o >> 1;  // the pair's index in BF16x2 units
    if constexpr (PL == V_F16P) {
      uint32_t *pg = (uint32_t *)gam, *pf = (uint32_t *)fv;
      const long long ps2 = ps >> 1;
      const float g0 = odd ? ga_in : ga.x, g1 = odd ? ga.y : ga_in;
      const float f0 = odd ? f_in : f.x, f1 = odd ? f.y : f_in;
      const int part = odd ? 1 : 0;
      uint32_t h, l;
      f16_split2(sa * g0, sa * g1, h, l);
      pg[(2 * part) * ps2 + o2] = h;
      pg[(2 * part + 1) * ps2 + o2] = l;
      f16_split2(sb * f0, sb * f1, h, l);
      pf[part * ps2 + o2] = h;
      pf[(2 + part) * ps2 + o2] = l;
    } else if constexpr (PL == V_BF16P) {
      uint32_t *pg = (uint32_t *)gam, *pf = (uint32_t *)fv;
      const long long ps2 = ps >> 1;
      // (element k', element k'+1) of this lane's part
      const float g0 = odd ? ga_in : ga.x, g1 = odd ? ga.y : ga_in;
      const float f0 = odd ? f_in : f.x, f1 = odd ? f.y : f_in;
      const int part = odd ? 1 : 0;
      float r0, r1, s0, s1;
      pg[(2 * part) * ps2 + o2] = split_pair(g0, g1, r0, r1);
      pg[(2 * part + 1) * ps2 + o2] = pack_pair(r0, r1);
      pf[part * ps2 + o2] = split_pair(f0, f1, r0, r1);
      pf[(2 + part) * ps2 + o2] = split_pair(r0, r1, s0, s1);
      pf[(4 + part) * ps2 + o2] = pack_pair(s0, s1);
    } else {
      // complex64: the even lane needs the odd lane's Gamma X, the odd lane the even lane's F
      const float ga_y = __shfl_xor_sync(mask, ga.y, 1), f_x = __shfl_xor_sync(mask, f.x, 1);
      if (!odd)
        *reinterpret_cast<float4 *>((S *)gam + 2 * o2) = make_float4(ga.x, ga.y, ga_in, ga_y);
      else
        *reinterpret_cast<float4 *>((S *)fv + 2 * o2) = make_float4(f_x, f_in, f.x, f.y);
    }
  }
  __device__ inline void put(long long o, double2 ga, double2 f, float = 1.f, float = 1.f) const {
    ((S *)gam)[o] = ga;
    ((S *)fv)[o] = f;
  }
};

// S: storage type of vertices, C: arithmetic type (double2 for FP64, float2 for the split path);
// PL: operands written as BF16 (V_BF16P) or FP16 (V_F16P) planes, else as complex values.
// Pass p covers the output transfers with q-momentum in [p.qb, p.qb + p.nq); the operand
// buffers hold their 4 * nq * NOmega slices with rows of ld elements.  A fused pass (all
// momenta) writes the d/m outputs at q and the s/t outputs at q' = k + k' + q of one gather
// step; otherwise each target momentum takes two gather steps, one per channel pair.
template <typename S, typename C, int PL, bool TAB>
__global__ void __launch_bounds__(256, 4) assemble_kernel(Grid g, const S *__restrict__ phi, Out<S, PL> out, int ld,
                                                       const double2 *__restrict__ k1,
                                                       const double2 *__restrict__ k2row,
                                                       const C *__restrict__ xph, const C *__restrict__ xpp,
                                                       const C *__restrict__ gtab, double2 *__restrict__ dfpart,
                                                       Lam lam, Pass pass, const float *__restrict__ fsc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NB = g.n_om * g.n_nu;
  // R blocks are read along columns (map A) and anti-diagonals (map C): rows padded by two
  // elements keep both strides off the shared-memory bank period
  const int RS = g.n_nu + 2;
  S *Rd = (S *)smem_raw;
  S *Rm = Rd + g.n_om * RS;
  S *Pd = Rm + g.n_om * RS;
  S *Pm = Pd + NB;
  S *Ss = Pm + NB;
  S *St = Ss + NB;
  C *FKd = (C *)(St + NB);  // K1 + K2row(k) at transfer (k'-k, m~), x = d
  C *FKm = FKd + g.n_om;
  __shared__ double2 red[256];
  __shared__ float ssc[8];  // FP16 planes: scales of Gamma X and F per channel
  if (PL == V_F16P && threadIdx.x < 8) ssc[threadIdx.x] = fsc[threadIdx.x < 4 ? FSC_SA + threadIdx.x : FSC_SB + threadIdx.x - 4];

  const int ikp = blockIdx.x, k = blockIdx.y;
  const int ik = k / g.n_nu, n = g.n_lo + k % g.n_nu;
  const long long nn = g.n;
  const long long chan = (long long)g.nQ * nn * nn;                        // channel stride of Phi
  const long long ochan = (long long)pass.nq * g.n_om * nn * ld;            // channel stride of the outputs
  const int tmom = ksub(g, ikp, ik);
  const C *xph_ = xph, *xpp_ = xpp;
  // exact e / Nnu for e < 2^16 by multiply-high with ceil(2^32 / Nnu) (Nnu >= 2)
  const unsigned nnu_magic = 0xFFFFFFFFu / (unsigned)g.n_nu + 1u;

  for (int t = threadIdx.x; t < 2 * g.n_om; t += blockDim.x) {
    int x = t / g.n_om, mt = t % g.n_om;
    int Qt = tmom * g.n_om + mt;
    double2 v = k1[(long long)x * g.nQ + Qt] + k2row[((long long)x * g.n + k) * g.nQ + Qt];
    (x == 0 ? FKd : FKm)[mt] = cfrom<C>(v);
  }

  const C l0 = cfrom<C>(lam.l[0]), l1 = cfrom<C>(lam.l[1]), l2 = cfrom<C>(lam.l[2]), l3 = cfrom<C>(lam.l[3]);
  const double2 U2 = make_double2(2.0 * g.U, 0.0);
  const C twoU = cfrom<C>(U2);
  C acc = cz<C>();     // FP64 path: the dF box sum itself
  DfSum<C> acc_all;    // split paths: a compensated sum of the per-step partial sums

  const int nstep = pass.fused ? 1 : 2;
  for (int iqc = pass.qb; iqc < pass.qb + pass.nq; ++iqc)
  for (int step = 0; step < nstep; ++step) {
    const bool do_dm = pass.fused || step == 0, do_st = pass.fused || step == 1;
    // step 1 gathers for the s/t outputs at q' = iqc, i.e. from q = q' - k - k'
    const int iq = step == 0 ? iqc : ksub(g, ksub(g, iqc, ik), ikp);
    const int iqp = kadd(g, kadd(g, ik, ikp), iq);
    const int cmom = kadd(g, ik, iq);
    const int pqk = ksub(g, iqp, ik);  // momentum of q' - k
    __syncthreads();
    for (int e = threadIdx.x; e < NB; e += blockDim.x) {
      const int mt = e / g.n_nu, c = e % g.n_nu;
      const long long rrow = ((long long)(tmom * g.n_om + mt) * nn + k) * nn + cmom * g.n_nu + c;
      const long long prow = ((long long)(iq * g.n_om + mt) * nn + k) * nn + ikp * g.n_nu + c;
      const long long srow = ((long long)(iqp * g.n_om + mt) * nn + k) * nn + ikp * g.n_nu + c;
      Rd[mt * RS + c] = phi[rrow];
      Rm[mt * RS + c] = phi[chan + rrow];
      Pd[e] = phi[prow];
      Pm[e] = phi[chan + prow];
      Ss[e] = phi[2 * chan + srow];
      St[e] = phi[3 * chan + srow];
    }
    __syncthreads();
    acc_all.step(acc);
    for (int e = threadIdx.x; e < NB; e += blockDim.x) {
      const int mi = (int)__umulhi((unsigned)e, nnu_magic), npi = e - mi * g.n_nu;
      const int m = g.m_lo + mi, np_ = g.n_lo + npi;
      const int mt = np_ - n;  // transfer k' - k of maps A and C
      const bool inT = (mt >= g.m_lo && mt <= g.m_hi);
      const int ti = mt - g.m_lo;
      if (do_dm) {
      // ---------------- d/m at Q = (q, m)
      C Ad = cz<C>(), Am = cz<C>();
      const int nc = n + m;  // column k + q of map A
      if (inT) {
        if (nc >= g.n_lo && nc <= g.n_hi) {
          Ad = to_c<S, C>(Rd[ti * RS + nc - g.n_lo]);
          Am = to_c<S, C>(Rm[ti * RS + nc - g.n_lo]);
        } else {
          Ad = FKd[ti];
          Am = FKm[ti];
        }
      }
      C Bs = cz<C>(), Bt = cz<C>();
      const int mb = n + np_ + m + 1;  // transfer k + k' + q of map B
      if (mb >= g.m_lo && mb <= g.m_hi) {
        Bs = to_c<S, C>(Ss[(mb - g.m_lo) * g.n_nu + npi]);
        Bt = to_c<S, C>(St[(mb - g.m_lo) * g.n_nu + npi]);
      }
      const C od = to_c<S, C>(Pd[e]), om = to_c<S, C>(Pm[e]);
      const C Gd = lam_at<TAB, C>(lam, 0, l0, m, n, np_) + (-0.5f) * Ad + (-1.5f) * Am + 0.5f * Bs + 1.5f * Bt;
      const C Gm = lam_at<TAB, C>(lam, 1, l1, m, n, np_) + (-0.5f) * Ad + 0.5f * Am + (-0.5f) * Bs + 0.5f * Bt;
      const C Fd = Gd + od, Fm = Gm + om;
      const int Q = iq * g.n_om + mi;
      const long long o_dm = ((long long)(Q - pass.qb * g.n_om) * nn + k) * ld + ikp * g.n_nu + npi;
      const C xq = (xph_[(long long)Q * nn + ikp * g.n_nu + npi]);
      out.put(o_dm, cmul(Gd, xq), Fd, ssc[0], ssc[4]);
      out.put(ochan + o_dm, cmul(Gm, xq), Fm, ssc[1], ssc[5]);
      // Eq. PA_Sigma, ph part: G(k+q) X_ph(Q,k') [F_d - F_m - (Lambda0_d - Lambda0_m)]
      const C gkq = (gtab[(long long)cmom * g.n_g + (n + m - g.g_lo)]);
      acc = cfma(cmul(gkq, xq), Fd - Fm - twoU, acc);
      }
      if (do_st) {
      // ---------------- s/t at Q' = (q', m)
      C Cd = cz<C>(), Cm = cz<C>();
      const int nc2 = m - np_ - 1;  // column q' - k' of map C
      if (inT) {
        if (nc2 >= g.n_lo && nc2 <= g.n_hi) {
          Cd = to_c<S, C>(Rd[ti * RS + nc2 - g.n_lo]);
          Cm = to_c<S, C>(Rm[ti * RS + nc2 - g.n_lo]);
        } else {
          Cd = FKd[ti];
          Cm = FKm[ti];
        }
      }
      C Dd = cz<C>(), Dm = cz<C>();
      const int md = m - n - np_ - 1;  // transfer q' - k - k' = q of map D
      if (md >= g.m_lo && md <= g.m_hi) {
        Dd = to_c<S, C>(Pd[(md - g.m_lo) * g.n_nu + npi]);
        Dm = to_c<S, C>(Pm[(md - g.m_lo) * g.n_nu + npi]);
      }
      const C os = to_c<S, C>(Ss[e]), ot = to_c<S, C>(St[e]);
      const C Gs = lam_at<TAB, C>(lam, 2, l2, m, n, np_) + 0.5f * Cd + (-1.5f) * Cm + 0.5f * Dd + (-1.5f) * Dm;
      const C Gt = lam_at<TAB, C>(lam, 3, l3, m, n, np_) + (-0.5f) * Cd + (-0.5f) * Cm + 0.5f * Dd + 0.5f * Dm;
      const C Fs = Gs + os, Ft = Gt + ot;
      const int Qp = iqp * g.n_om + mi;
      const long long o_st = ((long long)(Qp - pass.qb * g.n_om) * nn + k) * ld + ikp * g.n_nu + npi;
      const C xqp = (xpp_[(long long)Qp * nn + ikp * g.n_nu + npi]);
      out.put(2 * ochan + o_st, (-0.5f) * cmul(Gs, xqp), Fs, ssc[2], ssc[6]);
      out.put(3 * ochan + o_st, 0.5f * cmul(Gt, xqp), Ft, ssc[3], ssc[7]);
      // pp part: G(q'-k) X_pp(Q',k') [F_s + F_t - (Lambda0_s + Lambda0_t)]
      const C gqk = (gtab[(long long)pqk * g.n_g + (m - n - 1 - g.g_lo)]);
      acc = cfma(cmul(gqk, xqp), Fs + Ft - twoU, acc);
      }
    }
  }
  acc_all.step(acc);
  red[threadIdx.x] = acc_all.get(acc);
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // -(U/4)(T/N)^2 sum GGG: one T/N sits in X
    double pref = -(g.U * 0.25) * g.T / g.nk;
    double2 v = pref * red[0];
    if (pass.accumulate) v = v + dfpart[(long long)k * g.nk + ikp];
    dfpart[(long long)k * g.nk + ikp] = v;
  }
}

}  // namespace

size_t assemble_smem_bytes(const Grid &g, bool c64) {
  size_t es = c64 ? sizeof(float2) : sizeof(double2);
  return (2 * (size_t)g.n_om * (g.n_nu + 2) + 4 * (size_t)g.n_om * g.n_nu + 2 * (size_t)g.n_om) * es;
}

cudaError_t launch_kernels_extract(cudaStream_t st, const Grid &g, Buffers &b, bool c64, bool rowsums) {
  dim3 grid(g.nQ, 4);
  if (c64 && rowsums && !b.lower_edge)  // the products' row sums span both edges
    kernels_kernel<float2, true><<<grid, 256, 0, st>>>(g, (const float2 *)b.phi, b.k1, b.k2row, b.k2col, b.krow,
                                                       false, b.first_level);
  else if (c64)
    kernels_kernel<float2, false><<<grid, 256, 0, st>>>(g, (const float2 *)b.phi, b.k1, b.k2row, b.k2col, nullptr,
                                                        b.lower_edge, b.first_level);
  else
    kernels_kernel<double2, false><<<grid, 256, 0, st>>>(g, (const double2 *)b.phi, b.k1, b.k2row, b.k2col, nullptr,
                                                         b.lower_edge, b.first_level);
  return cudaGetLastError();
}

template <typename S, typename C, int PL, bool TAB>
static cudaError_t assemble_launch(cudaStream_t st, const Grid &g, Buffers &b, Lam lam, const Pass &p, long long ps) {
  auto kfn = assemble_kernel<S, C, PL, TAB>;
  const size_t sm = assemble_smem_bytes(g, sizeof(S) == sizeof(float2));
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  Out<S, PL> out{b.gam, b.fv, ps};
  // the FP32 assembly reads FP32 copies of the one-particle tables (no conversion per element)
  const C *xph, *xpp, *gtab;
  if constexpr (sizeof(C) == sizeof(float2)) {
    xph = (const C *)b.xph32;
    xpp = (const C *)b.xpp32;
    gtab = (const C *)b.gtab32;
  } else {
    xph = (const C *)b.xph;
    xpp = (const C *)b.xpp;
    gtab = (const C *)b.gtab;
  }
  kfn<<<dim3(g.nk, g.n), 256, sm, st>>>(g, (const S *)b.phi, out, b.ld, b.k1, b.k2row, xph, xpp, gtab, b.dfpart, lam,
                                        p, b.fsc);
  return cudaGetLastError();
}

cudaError_t launch_assemble(cudaStream_t st, const Grid &g, Buffers &b, const double *lam4, const Pass &p) {
  Lam lam;
  bool tab = false;
  for (int r = 0; r < 4; ++r) {
    lam.l[r] = make_double2(lam4[2 * r], lam4[2 * r + 1]);
    lam.tab[r] = b.lam_tab[r];
    lam.nl[r] = b.lam_nl[r];
    tab = tab || b.lam_tab[r];
  }
  // plane stride: fixed by the buffer size (q_chunk momenta), which the tensor maps assume,
  // also for a last pass with fewer momenta
  const long long ps = 4LL * b.q_chunk * g.n_om * g.n * (long long)b.ld;
  switch (b.vfmt) {
    case V_C128:
      return tab ? assemble_launch<double2, double2, 0, true>(st, g, b, lam, p, ps)
                 : assemble_launch<double2, double2, 0, false>(st, g, b, lam, p, ps);
    case V_C64:
      return tab ? assemble_launch<float2, float2, 0, true>(st, g, b, lam, p, ps)
                 : assemble_launch<float2, float2, 0, false>(st, g, b, lam, p, ps);
    case V_F16P:
      if (b.assembly == 0 && assemble_tiled_ok(g)) return launch_assemble_tiled(st, g, b, lam, p, ps, tab);
      return tab ? assemble_launch<float2, float2, V_F16P, true>(st, g, b, lam, p, ps)
                 : assemble_launch<float2, float2, V_F16P, false>(st, g, b, lam, p, ps);
    default:
      if (b.assembly == 0 && assemble_tiled_ok(g)) return launch_assemble_tiled(st, g, b, lam, p, ps, tab);
      return tab ? assemble_launch<float2, float2, V_BF16P, true>(st, g, b, lam, p, ps)
                 : assemble_launch<float2, float2, V_BF16P, false>(st, g, b, lam, p, ps);
  }
}

}  // namespace pq
