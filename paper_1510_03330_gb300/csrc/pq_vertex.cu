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
#include "pq_internal.h"

namespace pq {

namespace {

template <typename S>
__device__ inline double2 ld2(const S *p) {
  return to_c<S, double2>(*p);
}

// K1[r][Q], K2row[r][k][Q], K2col[r][k'][Q]; one block per (Q, r), FP64 sums.
template <typename S>
__global__ void kernels_kernel(Grid g, const S *__restrict__ phi, double2 *__restrict__ k1,
                               double2 *__restrict__ k2row, double2 *__restrict__ k2col) {
  __shared__ double2 red[256];
  __shared__ double2 sk1;
  const int Q = blockIdx.x, r = blockIdx.y;
  const long long n = g.n;
  const S *V = phi + ((long long)r * g.nQ + Q) * n * n;
  const int nn = g.n_nu, nk = g.nk;
  // first level: four corners, all momentum pairs
  double2 acc = make_double2(0.0, 0.0);
  const int ncorner = 4 * nk * nk;
  for (int c = threadIdx.x; c < ncorner; c += blockDim.x) {
    int e = c & 3, pair = c >> 2;
    int a = pair / nk, b = pair % nk;
    int ra = a * nn + ((e & 1) ? nn - 1 : 0), cb = b * nn + ((e & 2) ? nn - 1 : 0);
    acc = acc + ld2(V + ra * n + cb);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sk1 = (1.0 / ncorner) * red[0];
    k1[(long long)r * g.nQ + Q] = sk1;
  }
  __syncthreads();
  const double2 K1 = sk1;
  const double inv = 1.0 / (2.0 * nk);
  for (int k = threadIdx.x; k < g.n; k += blockDim.x) {
    double2 rs = make_double2(0.0, 0.0), cs = make_double2(0.0, 0.0);
    for (int b = 0; b < nk; ++b) {
      rs = rs + ld2(V + k * n + b * nn) + ld2(V + k * n + b * nn + nn - 1);
      cs = cs + ld2(V + (long long)(b * nn) * n + k) + ld2(V + (long long)(b * nn + nn - 1) * n + k);
    }
    k2row[((long long)r * g.n + k) * g.nQ + Q] = inv * rs - K1;
    k2col[((long long)r * g.n + k) * g.nQ + Q] = inv * cs - K1;
  }
}

struct Lam {
  double2 l[4];  // Lambda_r (parquet approximation: U, -U, 2U, 0)
};

template <typename C> __device__ inline C cz();
template <> __device__ inline double2 cz<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ inline float2 cz<float2>() { return make_float2(0.f, 0.f); }
template <typename C> __device__ inline C cfrom(double2 v);
template <> __device__ inline double2 cfrom<double2>(double2 v) { return v; }
template <> __device__ inline float2 cfrom<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <typename C> __device__ inline double2 cdbl(C v);
template <> __device__ inline double2 cdbl<double2>(double2 v) { return v; }
template <> __device__ inline double2 cdbl<float2>(float2 v) { return make_double2(v.x, v.y); }

// BF16 operand planes of the split BSE: x = h + l (+ r for F), each piece the
// BF16 rounding of what the previous pieces leave (the differences are exact in FP32).
__device__ inline void store_planes2(__nv_bfloat16 *p, long long ps, long long o, float2 v) {
  const __nv_bfloat16 rh = __float2bfloat16_rn(v.x), ih = __float2bfloat16_rn(v.y);
  p[o] = rh;
  p[ps + o] = __float2bfloat16_rn(v.x - __bfloat162float(rh));
  p[2 * ps + o] = ih;
  p[3 * ps + o] = __float2bfloat16_rn(v.y - __bfloat162float(ih));
}
__device__ inline void store_planes3(__nv_bfloat16 *p, long long ps, long long o, float2 v) {
  const __nv_bfloat16 rh = __float2bfloat16_rn(v.x), ih = __float2bfloat16_rn(v.y);
  const float rr = v.x - __bfloat162float(rh), ir = v.y - __bfloat162float(ih);
  const __nv_bfloat16 rl = __float2bfloat16_rn(rr), il = __float2bfloat16_rn(ir);
  p[o] = rh;
  p[ps + o] = ih;
  p[2 * ps + o] = rl;
  p[3 * ps + o] = il;
  p[4 * ps + o] = __float2bfloat16_rn(rr - __bfloat162float(rl));
  p[5 * ps + o] = __float2bfloat16_rn(ir - __bfloat162float(il));
}

template <typename S, bool PL>
struct Out {
  void *gam, *fv;
  long long ps;  // plane stride (PL)
  __device__ inline void put(long long o, float2 ga, float2 f) const {
    if constexpr (PL) {
      store_planes2((__nv_bfloat16 *)gam, ps, o, ga);
      store_planes3((__nv_bfloat16 *)fv, ps, o, f);
    } else {
      ((S *)gam)[o] = ga;
      ((S *)fv)[o] = f;
    }
  }
  __device__ inline void put(long long o, double2 ga, double2 f) const {
    ((S *)gam)[o] = ga;
    ((S *)fv)[o] = f;
  }
};

// S: storage type of vertices, C: arithmetic type (double2 for FP64, float2 for the split path);
// PL: operands written as BF16 planes.
// Pass p covers the output transfers with q-momentum in [p.qb, p.qb + p.nq); the operand
// buffers hold their 4 * nq * NOmega slices with rows of ld elements.  A fused pass (all
// momenta) writes the d/m outputs at q and the s/t outputs at q' = k + k' + q of one gather
// step; otherwise each target momentum takes two gather steps, one per channel pair.
template <typename S, typename C, bool PL>
__global__ void __launch_bounds__(256) assemble_kernel(Grid g, const S *__restrict__ phi, Out<S, PL> out, int ld,
                                                       const double2 *__restrict__ k1,
                                                       const double2 *__restrict__ k2row,
                                                       const double2 *__restrict__ xph,
                                                       const double2 *__restrict__ xpp,
                                                       const double2 *__restrict__ gtab, double2 *__restrict__ dfpart,
                                                       Lam lam, Pass pass) {
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

  const int ikp = blockIdx.x, k = blockIdx.y;
  const int ik = k / g.n_nu, n = g.n_lo + k % g.n_nu;
  const long long nn = g.n;
  const long long chan = (long long)g.nQ * nn * nn;                        // channel stride of Phi
  const long long ochan = (long long)pass.nq * g.n_om * nn * ld;            // channel stride of the outputs
  const int tmom = ksub(g, ikp, ik);
  const double2 *xph_ = xph, *xpp_ = xpp;

  for (int t = threadIdx.x; t < 2 * g.n_om; t += blockDim.x) {
    int x = t / g.n_om, mt = t % g.n_om;
    int Qt = tmom * g.n_om + mt;
    double2 v = k1[(long long)x * g.nQ + Qt] + k2row[((long long)x * g.n + k) * g.nQ + Qt];
    (x == 0 ? FKd : FKm)[mt] = cfrom<C>(v);
  }

  const C l0 = cfrom<C>(lam.l[0]), l1 = cfrom<C>(lam.l[1]), l2 = cfrom<C>(lam.l[2]), l3 = cfrom<C>(lam.l[3]);
  const double2 U2 = make_double2(2.0 * g.U, 0.0);
  const C twoU = cfrom<C>(U2);
  C acc = cz<C>();

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
    for (int e = threadIdx.x; e < NB; e += blockDim.x) {
      const int mi = e / g.n_nu, npi = e % g.n_nu;
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
      const C Gd = l0 + (-0.5f) * Ad + (-1.5f) * Am + 0.5f * Bs + 1.5f * Bt;
      const C Gm = l1 + (-0.5f) * Ad + 0.5f * Am + (-0.5f) * Bs + 0.5f * Bt;
      const C Fd = Gd + od, Fm = Gm + om;
      const int Q = iq * g.n_om + mi;
      const long long o_dm = ((long long)(Q - pass.qb * g.n_om) * nn + k) * ld + ikp * g.n_nu + npi;
      const C xq = cfrom<C>(xph_[(long long)Q * nn + ikp * g.n_nu + npi]);
      out.put(o_dm, cmul(Gd, xq), Fd);
      out.put(ochan + o_dm, cmul(Gm, xq), Fm);
      // Eq. PA_Sigma, ph part: G(k+q) X_ph(Q,k') [F_d - F_m - (Lambda0_d - Lambda0_m)]
      const C gkq = cfrom<C>(gtab[(long long)cmom * g.n_g + (n + m - g.g_lo)]);
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
      const C Gs = l2 + 0.5f * Cd + (-1.5f) * Cm + 0.5f * Dd + (-1.5f) * Dm;
      const C Gt = l3 + (-0.5f) * Cd + (-0.5f) * Cm + 0.5f * Dd + 0.5f * Dm;
      const C Fs = Gs + os, Ft = Gt + ot;
      const int Qp = iqp * g.n_om + mi;
      const long long o_st = ((long long)(Qp - pass.qb * g.n_om) * nn + k) * ld + ikp * g.n_nu + npi;
      const C xqp = cfrom<C>(xpp_[(long long)Qp * nn + ikp * g.n_nu + npi]);
      out.put(2 * ochan + o_st, (-0.5f) * cmul(Gs, xqp), Fs);
      out.put(3 * ochan + o_st, 0.5f * cmul(Gt, xqp), Ft);
      // pp part: G(q'-k) X_pp(Q',k') [F_s + F_t - (Lambda0_s + Lambda0_t)]
      const C gqk = cfrom<C>(gtab[(long long)pqk * g.n_g + (m - n - 1 - g.g_lo)]);
      acc = cfma(cmul(gqk, xqp), Fs + Ft - twoU, acc);
      }
    }
  }
  red[threadIdx.x] = cdbl<C>(acc);
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

cudaError_t launch_kernels_extract(cudaStream_t st, const Grid &g, Buffers &b, bool c64) {
  dim3 grid(g.nQ, 4);
  if (c64)
    kernels_kernel<float2><<<grid, 256, 0, st>>>(g, (const float2 *)b.phi, b.k1, b.k2row, b.k2col);
  else
    kernels_kernel<double2><<<grid, 256, 0, st>>>(g, (const double2 *)b.phi, b.k1, b.k2row, b.k2col);
  return cudaGetLastError();
}

template <typename S, typename C, bool PL>
static cudaError_t assemble_launch(cudaStream_t st, const Grid &g, Buffers &b, Lam lam, const Pass &p, long long ps) {
  auto kfn = assemble_kernel<S, C, PL>;
  const size_t sm = assemble_smem_bytes(g, sizeof(S) == sizeof(float2));
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  Out<S, PL> out{b.gam, b.fv, ps};
  kfn<<<dim3(g.nk, g.n), 256, sm, st>>>(g, (const S *)b.phi, out, b.ld, b.k1, b.k2row, b.xph, b.xpp, b.gtab,
                                        b.dfpart, lam, p);
  return cudaGetLastError();
}

cudaError_t launch_assemble(cudaStream_t st, const Grid &g, Buffers &b, const double *lam4, const Pass &p) {
  Lam lam;
  for (int r = 0; r < 4; ++r) lam.l[r] = make_double2(lam4[2 * r], lam4[2 * r + 1]);
  // plane stride: fixed by the buffer size (q_chunk momenta), which the tensor maps assume,
  // also for a last pass with fewer momenta
  const long long ps = 4LL * b.q_chunk * g.n_om * g.n * (long long)b.ld;
  switch (b.vfmt) {
    case V_C128: return assemble_launch<double2, double2, false>(st, g, b, lam, p, ps);
    case V_C64: return assemble_launch<float2, float2, false>(st, g, b, lam, p, ps);
    default: return assemble_launch<float2, float2, true>(st, g, b, lam, p, ps);
  }
}

}  // namespace pq
