// Kernel-function part of the regulated self-energy (Sec. II.B):
//   Sigma~2(k) = -(U/4)(T/N)^2 sum_{k' in BF, q in BB}
//                [G(k+q) G(k'+q) G(k') (F~_d - F~_m - 2U) + G(q-k') G(q-k) G(k') (F~_s + F~_t - 2U)],
// the Schwinger-Dyson equation (Eq. PA_Sigma) with the auxiliary vertex F~
// (Eq. auxiliary_function, level-2 kernels) minus Lambda^0, summed on the box
// BF x BB enlarged sigma2_factor times.  F~ - Lambda^0 is a sum of kernel
// terms, each a function of one transfer P and at most one further leg, so
// after substituting P for the transfer every term factorises into
//   G(one leg of k) x (momentum-summed bubble of P over a frequency window),
// which is what the code evaluates: the literal double sum, reordered.
//
// Tables, for P in the vertex bosonic box (momentum sums over j-vector):
//   Bph[P][j] = sum G(j) G(j+P)            Bpp[P][j] = sum G(P-j) G(j)
//   Cph[x][P][j] = sum G(j) G(j+P) K2col_x(j;P)   x = d-m, m   (j in the box)
//   Cpp[P][j]    = sum G(P-j) G(j) K2col_{s+t}(j;P)             (j in the box)
// Six terms per (k, P) with the coefficients of F~_d - F~_m and F~_s + F~_t:
//   own ph (d-m at q), -2 Phi~_m^{k,k+q}(k'-k), Psi~_{s+t}^{k,k'}(k+k'+q),
//   own pp (s+t at q), -2 Phi~_m^{k,q-k'}(k'-k), Phi~_{d-m}^{k,k'}(q-k-k').
#include "pq_common.cuh"
#include "pq_internal.h"

namespace pq {

namespace {

__device__ inline double2 gt(const Grid &g, const double2 *gtab, int ik, int n) {
  return gtab[(long long)ik * g.n_g + (n - g.g_lo)];
}

__global__ void s2_bubble_tables(Grid g, int j_lo, int nj, const double2 *__restrict__ gtab,
                                 double2 *__restrict__ bph, double2 *__restrict__ bpp) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.nQ * nj) return;
  int P = i / nj, j = j_lo + i % nj;
  int iP = P / g.n_om, mP = g.m_lo + P % g.n_om;
  double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
  for (int ij = 0; ij < g.nk; ++ij) {
    double2 gj = gt(g, gtab, ij, j);
    a = cfma(gj, gt(g, gtab, kadd(g, ij, iP), j + mP), a);
    b = cfma(gj, gt(g, gtab, ksub(g, iP, ij), mP - j - 1), b);
  }
  bph[i] = a;
  bpp[i] = b;
}

__global__ void s2_weighted_tables(Grid g, const double2 *__restrict__ gtab, const double2 *__restrict__ k2col,
                                   double2 *__restrict__ cph, double2 *__restrict__ cpp) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.nQ * g.n_nu) return;
  int P = i / g.n_nu, jj = i % g.n_nu, j = g.n_lo + jj;
  int iP = P / g.n_om, mP = g.m_lo + P % g.n_om;
  const long long cs = (long long)g.n * g.nQ;  // one channel of K2col
  double2 adm = make_double2(0.0, 0.0), am = make_double2(0.0, 0.0), ast = make_double2(0.0, 0.0);
  for (int ij = 0; ij < g.nk; ++ij) {
    long long kc = (long long)(ij * g.n_nu + jj) * g.nQ + P;
    double2 cd = k2col[kc], cm = k2col[cs + kc], css = k2col[2 * cs + kc], ct = k2col[3 * cs + kc];
    double2 gj = gt(g, gtab, ij, j);
    double2 wph = cmul(gj, gt(g, gtab, kadd(g, ij, iP), j + mP));
    double2 wpp = cmul(gj, gt(g, gtab, ksub(g, iP, ij), mP - j - 1));
    adm = cfma(wph, cd - cm, adm);
    am = cfma(wph, cm, am);
    ast = cfma(wpp, css + ct, ast);
  }
  cph[i] = adm;
  cph[(long long)g.nQ * g.n_nu + i] = am;
  cpp[i] = ast;
}

struct Box {
  int bf_lo, bf_hi, bb_lo, bb_hi;  // summation box of k' (fermionic) and q (bosonic)
  int o_lo, o_hi;                  // output fermionic range
  double sign;
  int accumulate;
};

// The tables are turned into inclusive prefix sums along j (FP64), so that every
// frequency-window sum below is the difference of two entries.
__global__ void s2_prefix_rows(double2 *__restrict__ t, long long rows, int len) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= rows) return;
  double2 *row = t + i * len;
  double2 s = make_double2(0.0, 0.0);
  for (int j = 0; j < len; ++j) {
    s = s + row[j];
    row[j] = s;
  }
}

__device__ inline double2 wsum(const double2 *cum, int j_lo, int nj, int a, int b) {
  // sum of the table row over j in [a, b] (clipped to its range) from its prefix sums
  if (a < j_lo) a = j_lo;
  if (b > j_lo + nj - 1) b = j_lo + nj - 1;
  if (a > b) return make_double2(0.0, 0.0);
  double2 s = cum[b - j_lo];
  if (a > j_lo) s = s - cum[a - 1 - j_lo];
  return s;
}

// One warp per output k = (k-vector, n); lanes split the transfers P.
__global__ void s2_output(Grid g, Box bx, int j_lo, int nj, const double2 *__restrict__ gtab,
                          const double2 *__restrict__ k1, const double2 *__restrict__ k2row,
                          const double2 *__restrict__ bph, const double2 *__restrict__ bpp,
                          const double2 *__restrict__ cph, const double2 *__restrict__ cpp,
                          double2 *__restrict__ out) {
  const int nout = bx.o_hi - bx.o_lo + 1;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  if (w >= g.nk * nout) return;
  const int ik = w / nout, n = bx.o_lo + w % nout;
  const bool kin = (n >= g.n_lo && n <= g.n_hi);
  const int krow = ik * g.n_nu + (n - g.n_lo);
  const long long cq = g.nQ;
  const long long kq = (long long)g.n * g.nQ;
  const int nb = g.n_nu;
  double2 acc = make_double2(0.0, 0.0);
  for (int P = lane; P < g.nQ; P += 32) {
    const int iP = P / g.n_om, mP = g.m_lo + P % g.n_om;
    double2 K1d = k1[P], K1m = k1[cq + P], K1s = k1[2 * cq + P], K1t = k1[3 * cq + P];
    double2 Rd = make_double2(0, 0), Rm = Rd, Rs = Rd, Rt = Rd;
    if (kin) {
      long long o = (long long)krow * g.nQ + P;
      Rd = k2row[o];
      Rm = k2row[kq + o];
      Rs = k2row[2 * kq + o];
      Rt = k2row[3 * kq + o];
    }
    const double2 kdm = (K1d - K1m) + (Rd - Rm);
    const double2 km = K1m + Rm;
    const double2 kst = (K1s + K1t) + (Rs + Rt);
    const double2 *Bph = bph + (long long)P * nj;
    const double2 *Bpp = bpp + (long long)P * nj;
    const double2 *Cdm = cph + (long long)P * nb;
    const double2 *Cm = cph + (long long)g.nQ * nb + (long long)P * nb;
    const double2 *Cst = cpp + (long long)P * nb;
    const int f_lo = g.n_lo, f_hi = g.n_hi;
    const double2 gkP = gt(g, gtab, kadd(g, ik, iP), n + mP);  // G(k+P)
    const double2 gPk = gt(g, gtab, ksub(g, iP, ik), mP - n - 1);  // G(P-k)
    double2 t;
    // own ph: G(k+q) sum_{k' in BF} G(k'+q) G(k') Phi~_{d-m}^{k,k'}(q)
    t = cmul(kdm, wsum(Bph, j_lo, nj, bx.bf_lo, bx.bf_hi)) + wsum(Cdm, f_lo, nb, bx.bf_lo, bx.bf_hi);
    acc = cfma(gkP, t, acc);
    // own pp: G(q-k) sum_{k' in BF} G(q-k') G(k') Psi~_{s+t}^{k,k'}(q)
    t = cmul(kst, wsum(Bpp, j_lo, nj, bx.bf_lo, bx.bf_hi)) + wsum(Cst, f_lo, nb, bx.bf_lo, bx.bf_hi);
    acc = cfma(gPk, t, acc);
    // Psi~_{s+t}^{k,k'}(k+k'+q): P = k+k'+q, q in BB <=> k' in [mP-n-1-bb_hi, mP-n-1-bb_lo]
    {
      int a = max(bx.bf_lo, mP - n - 1 - bx.bb_hi), b = min(bx.bf_hi, mP - n - 1 - bx.bb_lo);
      if (a <= b) {
        t = cmul(kst, wsum(Bpp, j_lo, nj, a, b)) + wsum(Cst, f_lo, nb, max(a, f_lo), min(b, f_hi));
        acc = cfma(gPk, t, acc);
      }
    }
    // Phi~_{d-m}^{k,k'}(q-k-k'): P = q-k-k', q in BB <=> k' in [bb_lo-mP-n-1, bb_hi-mP-n-1]
    {
      int a = max(bx.bf_lo, bx.bb_lo - mP - n - 1), b = min(bx.bf_hi, bx.bb_hi - mP - n - 1);
      if (a <= b) {
        t = cmul(kdm, wsum(Bph, j_lo, nj, a, b)) + wsum(Cdm, f_lo, nb, max(a, f_lo), min(b, f_hi));
        acc = cfma(gkP, t, acc);
      }
    }
    // -2 Phi~_m^{k,k+q}(k'-k) and -2 Phi~_m^{k,q-k'}(k'-k): P = k'-k, k' = k+P in BF
    if (n + mP >= bx.bf_lo && n + mP <= bx.bf_hi) {
      // map A: j = k+q with q in BB, column leg j
      double2 ta = cmul(km, wsum(Bph, j_lo, nj, n + bx.bb_lo, n + bx.bb_hi)) +
                   wsum(Cm, f_lo, nb, max(n + bx.bb_lo, f_lo), min(n + bx.bb_hi, f_hi));
      // map C: j = q-k with q in BB, column leg j-P; tables shifted by mP
      int a = bx.bb_lo - n - 1 - mP, b = bx.bb_hi - n - 1 - mP;
      double2 tc = cmul(km, wsum(Bph, j_lo, nj, a, b)) + wsum(Cm, f_lo, nb, max(a, f_lo), min(b, f_hi));
      acc = cfma(gkP, (-2.0) * (ta + tc), acc);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) {
    double pref = -(g.U * 0.25) * (g.T / g.nk) * (g.T / g.nk) * bx.sign;
    double2 v = pref * acc;
    double2 *dst = out + (long long)ik * g.n_ext + (n - g.e_lo);
    *dst = bx.accumulate ? (*dst + v) : v;
  }
}

}  // namespace

cudaError_t launch_sigma2(cudaStream_t st, const Grid &g, const Sizes &z, Buffers &b) {
  int nt = 256;
  s2_bubble_tables<<<(g.nQ * z.nj + nt - 1) / nt, nt, 0, st>>>(g, z.j_lo, z.nj, b.gtab, b.s2_bph, b.s2_bpp);
  s2_weighted_tables<<<(g.nQ * g.n_nu + nt - 1) / nt, nt, 0, st>>>(g, b.gtab, b.k2col, b.s2_cph, b.s2_cpp);
  // prefix sums of every row: B tables (rows of nj), C tables (rows of Nnu; cph holds two)
  s2_prefix_rows<<<(2 * g.nQ + nt - 1) / nt, nt, 0, st>>>(b.s2_bph, g.nQ, z.nj);
  s2_prefix_rows<<<(2 * g.nQ + nt - 1) / nt, nt, 0, st>>>(b.s2_bpp, g.nQ, z.nj);
  s2_prefix_rows<<<(2 * g.nQ + nt - 1) / nt, nt, 0, st>>>(b.s2_cph, 2LL * g.nQ, g.n_nu);
  s2_prefix_rows<<<(g.nQ + nt - 1) / nt, nt, 0, st>>>(b.s2_cpp, g.nQ, g.n_nu);
  // enlarged box over the whole extended range
  Box big{g.bf_lo, g.bf_hi, g.bb_lo, g.bb_hi, g.e_lo, g.e_hi, 1.0, 0};
  int warps = g.nk * (g.e_hi - g.e_lo + 1);
  s2_output<<<(warps * 32 + nt - 1) / nt, nt, 0, st>>>(g, big, z.j_lo, z.nj, b.gtab, b.k1, b.k2row, b.s2_bph,
                                                       b.s2_bpp, b.s2_cph, b.s2_cpp, b.sigma2);
  // minus the same sum on the vertex box, whose F - F~ remainder the vertex pass adds as F - Lambda^0
  Box box{g.n_lo, g.n_hi, g.m_lo, g.m_hi, g.n_lo, g.n_hi, -1.0, 1};
  warps = g.nk * g.n_nu;
  s2_output<<<(warps * 32 + nt - 1) / nt, nt, 0, st>>>(g, box, z.j_lo, z.nj, b.gtab, b.k1, b.k2row, b.s2_bph,
                                                       b.s2_bpp, b.s2_cph, b.s2_cpp, b.sigma2);
  return cudaGetLastError();
}

}  // namespace pq
