// Tiled parquet assembly for the split paths that write operand planes (BF16x3, FP16x3): the
// parquet equations with the kernel fill (Eq. PA_F; App. A, Eqs. PA_Gamma_dm, PA_Gamma_st;
// Sec. II.A), F = Gamma + Phi, the BSE left operand s_r Gamma_r diag(X_r) (Eq. PA_F_Phi) split
// into BF16 or FP16 planes, and the box sum of Eq. PA_Sigma over F - Lambda^0 (Sec. II.B).  The arithmetic per element is that of the
// general assembly in pq_vertex.cu; what differs is how the work is cut, so that every
// operand row is written in runs of G * Nnu contiguous columns instead of Nnu.
//
// One CTA per (row leg k, group of G k'-momenta p_a = p_0 + a that are consecutive in one
// lattice row, G | L).  Per q-momentum step it gathers, completing on one mbarrier:
//   R_x[a] = Phi_x[(p_a - k, .)][k][(k + q, .)]      x = d, m   (maps A and C; a TMA box each)
//   P_x    = Phi_x[(q, .)][k][(p_0 .. p_G-1, .)]      x = d, m   (own d/m, map D; a bulk copy per row)
//   S_x[a] = Phi_x[(k + p_a + q, .)][k][(p_a, .)]     x = s, t   (map B, own s/t; a bulk copy per row)
// and each thread computes four consecutive k' of one output row (one frequency m).
//
// The d/m outputs of a step fill rows (q, m) over all G blocks.  The s/t outputs of block a
// belong to q' = k + p_a + q, a different row for every block.  With q walking along a
// lattice row (y fastest), block a of a given q' row comes a steps before its block 0, so
// each thread keeps its last a s/t results in a private shared-memory delay line and writes
// them in the step that produces block 0 of that row: all G blocks of the row are then
// stored by one warp instruction.  Rows whose blocks straddle the end of a lattice row of q
// are written block by block.
//
// Without room for the delay line (or in the passes of a multi-pass iteration) every target
// momentum takes two steps: the d/m step above, and an s/t step that gathers, for all
// blocks, the slices feeding q' = the target itself.
//
// Every wait on the gather barrier is bounded in time; a wait that gives up sets the error
// flag, waits once more (bounded) for the copies in flight and ends the CTA.
#include <cuda.h>

#include <algorithm>

#include "pq_assemble.cuh"
#include "pq_common.cuh"
#include "pq_internal.h"
#include "pq_tc.cuh"
#include "pq_tma.cuh"

namespace pq {

namespace {

constexpr int TT = 256;                             // threads per CTA at most
constexpr uint64_t GATHER_WAIT_NS = 2000000000ull;  // 2 s per wait

struct TGeo {
  int G;      // k'-momentum blocks per CTA
  int hb;     // Nnu / 4: thread columns per block
  int upr;    // G * hb: thread columns per output row
  int rows;   // output rows (frequencies m) per sweep
  int nthr;   // blockDim: upr * rows rounded up to whole warps (the copies are issued by a full warp)
  int RS, RA; // row stride (= the TMA box width) and block stride (float2) of the R tiles
  int sh;     // R tile of block a: its Nnu columns start a * sh words into each row
  int PW, BW; // row stride and block stride (float2) of the S tile
  int PPW;    // row stride (float2) of the P tile, whose blocks are adjacent (block stride Nnu)
  int oR, oP, oS, oFK, oRing, oBar, smem;  // shared-memory layout (bytes)
  int tx;     // bytes gathered per step
  int ring_n; // threads per block index a (hb * rows)
  unsigned long long m_per, m_gn, m_nom;  // x / d = (x * m_d) >> 32 for x < 2^16 (d = 3 tiles' copies, G NOmega, NOmega)
  unsigned long long m_L;                 // the same for d = L (momentum indices x < L^2 < 2^16)
};

__device__ __forceinline__ int mdiv(int x, unsigned long long m) { return (int)(((unsigned long long)x * m) >> 32); }

// Lattice momentum arithmetic (a + b, -a, a - b on the L x L grid, index x L + y) with the
// divisions by L done by mdiv: a division by a runtime divisor goes through int <-> float
// conversions, which run on the narrow FP64 pipe of this part, and the step tables are
// rebuilt every step while the other warps wait.
__device__ __forceinline__ int tadd(const Grid &g, const TGeo &t, int a, int b) {
  const int L = g.L, xa = mdiv(a, t.m_L), xb = mdiv(b, t.m_L);
  int x = xa + xb, y = (a - xa * L) + (b - xb * L);
  if (x >= L) x -= L;
  if (y >= L) y -= L;
  return x * L + y;
}
__device__ __forceinline__ int tneg(const Grid &g, const TGeo &t, int a) {
  const int L = g.L, x = mdiv(a, t.m_L), y = a - x * L;
  return (x ? L - x : 0) * L + (y ? L - y : 0);
}
__device__ __forceinline__ int tsub(const Grid &g, const TGeo &t, int a, int b) { return tadd(g, t, a, tneg(g, t, b)); }

// Momentum bookkeeping of one step, T_N ints per block b: the transfer groups (and the R
// column block) its gathers read, and the output rows of the step.  Kept in shared memory so
// that the lattice additions (integer divisions by L) are done once per block and step.
enum { T_QR, T_CR, T_QP, T_QS, T_PQK, T_CM, T_Q0, T_N };
// dm: the gathers of q = qt (the d/m step, or a fused step); else those feeding q' = qt.
__device__ inline void step_table(const Grid &g, const TGeo &t, bool dm, int qt, int ik, int p0, int b, int *e) {
  const int pb = p0 + b;
  const int qb_ = dm ? qt : tsub(g, t, tsub(g, t, qt, ik), pb);  // q of this block's slices
  const int x = dm ? tadd(g, t, tadd(g, t, ik, pb), qt) : qt;    // q' = k + p_b + q: S group, s/t output row
  e[T_QR] = tsub(g, t, pb, ik);
  e[T_CR] = tadd(g, t, ik, qb_);
  e[T_QP] = qb_;
  e[T_QS] = x;
  e[T_PQK] = tsub(g, t, x, ik);
  e[T_CM] = tadd(g, t, ik, qt);
  e[T_Q0] = tadd(g, t, tadd(g, t, ik, p0), qt);
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// One gather step, issued by all threads of the CTA (thread 0 posts the byte count), with
// the sources of the step table tb.  Per block b, for the d/m step of q = qt:
//   R from transfer group p_b - k at column block k + qt, P from group qt, S from k + p_b + qt;
// for the s/t step of q' = qt, with q_b = qt - k - p_b:
//   R from group p_b - k at column block k + q_b, P from group q_b, S from group qt.
// P and S take column block p_b.
__device__ inline void issue_gather(const Grid &g, const TGeo &t, const CUtensorMap *rmap, const int *tb,
                                    const float2 *phi, int k, int p0, float2 *Rt, float2 *Pt, float2 *St, uint64_t *bar,
                                    bool merge) {
  const int G = t.G, nom = g.n_om, nnu = g.n_nu;
  const long long nn = g.n, chan = (long long)g.nQ * nn * nn;
  const uint32_t b = tc::smem_u32(bar);
  if (threadIdx.x == 0) asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(t.tx) : "memory");
  // one copy per (tile, channel, block, transfer row): the blocks of an S row sit at a
  // padded stride in shared memory (bank spread), so they are copied separately; the G
  // blocks of a P row are adjacent in the tile and, on d/m steps (merge), come from one
  // transfer, so they take one copy (the copies, not their bytes, bound the issue).  A warp
  // issues its lanes' copies one after another, so every warp takes an equal share of
  // them (consecutive indices, lanes round robin): the gather is issued when the warp with
  // the most copies is done.
  const int per = 2 * G * nom, nR = 2 * G, nP = merge ? 2 * nom : per, nall = nR + nP + per;
  const uint32_t bytes = (uint32_t)nnu * 8u;
  const int nw = blockDim.x >> 5, wpc = (nall + nw - 1) / nw, w0 = (threadIdx.x >> 5) * wpc;
  for (int j = threadIdx.x & 31; j < wpc && w0 + j < nall; j += 32) {
    const int i = w0 + j;
    if (i < nR) {
      // R of channel x and block a: one tensor box of RS columns x NOmega transfers, started
      // a * sh columns early so that the block's Nnu columns sit a * sh words into each row
      const int x = i >= G, a = i - x * G;
      const int *e = tb + a * T_N;
      tma::load3(tc::smem_u32(Rt + (x * G + a) * t.RA), rmap, e[T_CR] * nnu - a * t.sh, k,
                 x * g.nQ + e[T_QR] * nom, bar);
      continue;
    }
    const int tile = i < nR + nP ? 1 : 2;
    const int ii = i - (tile == 1 ? nR : nR + nP);
    const float2 *src;
    float2 *dst;
    uint32_t nb = bytes;
    if (tile == 1 && merge) {
      // the G blocks of a P row are adjacent in Phi and in the tile: one copy
      const int x = mdiv(ii, t.m_nom), mt = ii - x * nom;
      src = phi + x * chan + ((long long)(tb[T_QP] * nom + mt) * nn + k) * nn + (long long)p0 * nnu;
      dst = Pt + (x * nom + mt) * t.PPW;
      nb = (uint32_t)G * bytes;
    } else {
      const int x = mdiv(ii, t.m_gn), rem = ii - x * G * nom;
      const int a = mdiv(rem, t.m_nom), mt = rem - a * nom;
      const int *e = tb + a * T_N;
      const int qg = tile == 1 ? e[T_QP] : e[T_QS];
      src = phi + (x + (tile == 1 ? 0 : 2)) * chan + ((long long)(qg * nom + mt) * nn + k) * nn + (long long)(p0 + a) * nnu;
      dst = tile == 1 ? Pt + (x * nom + mt) * t.PPW + a * nnu : St + (x * nom + mt) * t.PW + a * t.BW;
    }
    bulk_load(tc::smem_u32(dst), src, nb, b);
  }
}

// Four consecutive k' of one channel -> the BF16 planes.  Gamma X: x = h + l, planes
// (Re h, Re l, Im h, Im l); F: x = h + l + r, planes (Re h, Im h, Re l, Im l, Re r, Im r).
// Each piece is the BF16 rounding of what the previous pieces leave (exact in FP32).
struct Split4 {
  uint2 h, l, r;
};
__device__ inline uint2 pack4(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3) {
  return make_uint2(__byte_perm(a0, a1, 0x7632), __byte_perm(a2, a3, 0x7632));
}
__device__ inline float hi_part(uint32_t rounded) { return __uint_as_float(rounded & 0xFFFF0000u); }
template <bool THIRD>
__device__ inline Split4 split4(float x0, float x1, float x2, float x3) {
  const uint32_t h0 = bf16_round(x0), h1 = bf16_round(x1), h2 = bf16_round(x2), h3 = bf16_round(x3);
  const float r0 = x0 - hi_part(h0), r1 = x1 - hi_part(h1), r2 = x2 - hi_part(h2), r3 = x3 - hi_part(h3);
  const uint32_t l0 = bf16_round(r0), l1 = bf16_round(r1), l2 = bf16_round(r2), l3 = bf16_round(r3);
  Split4 s;
  s.h = pack4(h0, h1, h2, h3);
  s.l = pack4(l0, l1, l2, l3);
  if constexpr (THIRD) {
    s.r = pack4(bf16_round(r0 - hi_part(l0)), bf16_round(r1 - hi_part(l1)), bf16_round(r2 - hi_part(l2)),
                bf16_round(r3 - hi_part(l3)));
  }
  return s;
}
__device__ inline void put4(uint16_t *gam, uint16_t *fv, long long ps, long long o, const float2 *gx,
                            const float2 *f) {
  const Split4 gr = split4<false>(gx[0].x, gx[1].x, gx[2].x, gx[3].x);
  const Split4 gi = split4<false>(gx[0].y, gx[1].y, gx[2].y, gx[3].y);
  *(uint2 *)(gam + o) = gr.h;
  *(uint2 *)(gam + ps + o) = gr.l;
  *(uint2 *)(gam + 2 * ps + o) = gi.h;
  *(uint2 *)(gam + 3 * ps + o) = gi.l;
  const Split4 fr = split4<true>(f[0].x, f[1].x, f[2].x, f[3].x);
  const Split4 fi = split4<true>(f[0].y, f[1].y, f[2].y, f[3].y);
  *(uint2 *)(fv + o) = fr.h;
  *(uint2 *)(fv + ps + o) = fi.h;
  *(uint2 *)(fv + 2 * ps + o) = fr.l;
  *(uint2 *)(fv + 3 * ps + o) = fi.l;
  *(uint2 *)(fv + 4 * ps + o) = fr.r;
  *(uint2 *)(fv + 5 * ps + o) = fi.r;
}

// FP16 planes: the same four k' of Gamma X (scaled by sa) and F (scaled by sb) as h + l, planes
// Gamma X (Re h, Re l, Im h, Im l) and F (Re h, Im h, Re l, Im l).
__device__ inline void split4h(float sc, float x0, float x1, float x2, float x3, uint2 &h, uint2 &l) {
  f16_split2(sc * x0, sc * x1, h.x, l.x);
  f16_split2(sc * x2, sc * x3, h.y, l.y);
}
__device__ inline void put4h(uint16_t *gam, uint16_t *fv, long long ps, long long o, const float2 *gx,
                             const float2 *f, float sa, float sb) {
  uint2 h, l;
  split4h(sa, gx[0].x, gx[1].x, gx[2].x, gx[3].x, h, l);
  *(uint2 *)(gam + o) = h;
  *(uint2 *)(gam + ps + o) = l;
  split4h(sa, gx[0].y, gx[1].y, gx[2].y, gx[3].y, h, l);
  *(uint2 *)(gam + 2 * ps + o) = h;
  *(uint2 *)(gam + 3 * ps + o) = l;
  split4h(sb, f[0].x, f[1].x, f[2].x, f[3].x, h, l);
  *(uint2 *)(fv + o) = h;
  *(uint2 *)(fv + 2 * ps + o) = l;
  split4h(sb, f[0].y, f[1].y, f[2].y, f[3].y, h, l);
  *(uint2 *)(fv + ps + o) = h;
  *(uint2 *)(fv + 3 * ps + o) = l;
}

// Operand output of channel r in the plane format PF (V_BF16P or V_F16P).
template <int PF>
__device__ inline void put_ops(uint16_t *gam, uint16_t *fv, long long ps, long long o, const float2 *gx,
                               const float2 *f, const float *ssc, int r) {
  if constexpr (PF == V_F16P)
    put4h(gam, fv, ps, o, gx, f, ssc[r], ssc[4 + r]);
  else
    put4(gam, fv, ps, o, gx, f);
}

__device__ inline float2 f2(double2 v) { return make_float2((float)v.x, (float)v.y); }

// Everything one thread needs to evaluate its four elements of a step.
struct Ctx {
  const float2 *Rt, *Pt, *St, *FK;
  int G, RS, RA, PW, BW, PPW, nom, nnu, a, npi0, n, mi, ash;
};

// map A (column nc = k + q) or C (column nc2 = q' - k') of the R tile of block a, or the fill
// K1 + K2 outside the frequency box, or zero outside the transfer box
__device__ inline void r_at(const Grid &g, const Ctx &c, int ti, bool inT, int col, float2 &vd, float2 &vm) {
  vd = vm = make_float2(0.f, 0.f);
  if (!inT) return;
  if (col >= g.n_lo && col <= g.n_hi) {
    vd = c.Rt[(0 * c.G + c.a) * c.RA + ti * c.RS + c.ash + col - g.n_lo];
    vm = c.Rt[(1 * c.G + c.a) * c.RA + ti * c.RS + c.ash + col - g.n_lo];
  } else {
    vd = c.FK[(0 * c.G + c.a) * c.nom + ti];
    vm = c.FK[(1 * c.G + c.a) * c.nom + ti];
  }
}

// d/m at Q = (q, m): Gamma_d, Gamma_m (Eq. PA_Gamma_dm), F = Gamma + Phi, s Gamma X, and the
// ph part of the dF box sum.  Outputs of the four elements in gx[0..1][i], f[0..1][i].
template <bool TAB>
__device__ inline void elems_dm(const Grid &g, const Ctx &c, const Lam &lam, float2 l0, float2 l1, float2 twoU,
                                const float2 *xq, float2 gkq, float2 (*gx)[4], float2 (*f)[4], float2 &acc) {
  const int m = g.m_lo + c.mi, n = c.n;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int npi = c.npi0 + i, np_ = g.n_lo + npi;
    const int mt = np_ - n;  // transfer k' - k of maps A and C
    const bool inT = (mt >= g.m_lo && mt <= g.m_hi);
    float2 Ad, Am;
    r_at(g, c, mt - g.m_lo, inT, n + m, Ad, Am);
    float2 Bs = make_float2(0.f, 0.f), Bt = Bs;
    const int mb = n + np_ + m + 1;  // transfer k + k' + q of map B
    if (mb >= g.m_lo && mb <= g.m_hi) {
      Bs = c.St[(0 * c.nom + mb - g.m_lo) * c.PW + c.a * c.BW + npi];
      Bt = c.St[(1 * c.nom + mb - g.m_lo) * c.PW + c.a * c.BW + npi];
    }
    const float2 od = c.Pt[(0 * c.nom + c.mi) * c.PPW + c.a * c.nnu + npi];
    const float2 om = c.Pt[(1 * c.nom + c.mi) * c.PPW + c.a * c.nnu + npi];
    const float2 Gd = lam_at<TAB, float2>(lam, 0, l0, m, n, np_) + (-0.5f) * Ad + (-1.5f) * Am + 0.5f * Bs + 1.5f * Bt;
    const float2 Gm = lam_at<TAB, float2>(lam, 1, l1, m, n, np_) + (-0.5f) * Ad + 0.5f * Am + (-0.5f) * Bs + 0.5f * Bt;
    const float2 Fd = Gd + od, Fm = Gm + om;
    f[0][i] = Fd;
    f[1][i] = Fm;
    gx[0][i] = cmul(Gd, xq[i]);
    gx[1][i] = cmul(Gm, xq[i]);
    // Eq. PA_Sigma, ph part: G(k+q) X_ph(Q,k') [F_d - F_m - (Lambda0_d - Lambda0_m)]
    acc = cfma(cmul(gkq, xq[i]), Fd - Fm - twoU, acc);
  }
}

// s/t at Q' = (q', m) (Eq. PA_Gamma_st), with the BSE signs -1/2, +1/2 folded into Gamma X,
// and the pp part of the dF box sum.
template <bool TAB>
__device__ inline void elems_st(const Grid &g, const Ctx &c, const Lam &lam, float2 l2, float2 l3, float2 twoU,
                                const float2 *xqp, float2 gqk, float2 (*gx)[4], float2 (*f)[4], float2 &acc) {
  const int m = g.m_lo + c.mi, n = c.n;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int npi = c.npi0 + i, np_ = g.n_lo + npi;
    const int mt = np_ - n;
    const bool inT = (mt >= g.m_lo && mt <= g.m_hi);
    float2 Cd, Cm;
    r_at(g, c, mt - g.m_lo, inT, m - np_ - 1, Cd, Cm);  // column q' - k' of map C
    float2 Dd = make_float2(0.f, 0.f), Dm = Dd;
    const int md = m - n - np_ - 1;  // transfer q' - k - k' = q of map D
    if (md >= g.m_lo && md <= g.m_hi) {
      Dd = c.Pt[(0 * c.nom + md - g.m_lo) * c.PPW + c.a * c.nnu + npi];
      Dm = c.Pt[(1 * c.nom + md - g.m_lo) * c.PPW + c.a * c.nnu + npi];
    }
    const float2 os = c.St[(0 * c.nom + c.mi) * c.PW + c.a * c.BW + npi];
    const float2 ot = c.St[(1 * c.nom + c.mi) * c.PW + c.a * c.BW + npi];
    const float2 Gs = lam_at<TAB, float2>(lam, 2, l2, m, n, np_) + 0.5f * Cd + (-1.5f) * Cm + 0.5f * Dd + (-1.5f) * Dm;
    const float2 Gt = lam_at<TAB, float2>(lam, 3, l3, m, n, np_) + (-0.5f) * Cd + (-0.5f) * Cm + 0.5f * Dd + 0.5f * Dm;
    const float2 Fs = Gs + os, Ft = Gt + ot;
    f[0][i] = Fs;
    f[1][i] = Ft;
    gx[0][i] = (-0.5f) * cmul(Gs, xqp[i]);
    gx[1][i] = 0.5f * cmul(Gt, xqp[i]);
    // pp part: G(q'-k) X_pp(Q',k') [F_s + F_t - (Lambda0_s + Lambda0_t)]
    acc = cfma(cmul(gqk, xqp[i]), Fs + Ft - twoU, acc);
  }
}

__device__ inline void load4(const float2 *p, float2 *v) {
  const float4 u = ((const float4 *)p)[0], w = ((const float4 *)p)[1];
  v[0] = make_float2(u.x, u.y);
  v[1] = make_float2(u.z, u.w);
  v[2] = make_float2(w.x, w.y);
  v[3] = make_float2(w.z, w.w);
}

// FUSED: one gather per q, s/t rows completed through the delay line (needs rows == NOmega).
// Otherwise: two gathers per target momentum of the pass.
template <bool FUSED, bool TAB, int PF>
__global__ void __launch_bounds__(TT, 2)
    assemble_tiled_kernel(Grid g, TGeo t, const float2 *__restrict__ phi, uint16_t *__restrict__ gam,
                          uint16_t *__restrict__ fv, long long ps, int ld, const double2 *__restrict__ k1,
                          const double2 *__restrict__ k2row, const float2 *__restrict__ xph,
                          const float2 *__restrict__ xpp, const float2 *__restrict__ gtab,
                          double2 *__restrict__ dfpart, Lam lam, Pass pass, const float *__restrict__ fsc,
                          int *err, const __grid_constant__ CUtensorMap rmap) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double2 red[TT];
  __shared__ float ssc[8];  // FP16 planes: scales of Gamma X and F per channel
  __shared__ int abort_flag;
  __shared__ int stab[2][4 * T_N];  // step tables of this step and the next
  float2 *Rt = (float2 *)(smem + t.oR), *Pt = (float2 *)(smem + t.oP), *St = (float2 *)(smem + t.oS);
  float2 *FK = (float2 *)(smem + t.oFK);
  float4 *ring = (float4 *)(smem + t.oRing);
  uint64_t *bar = (uint64_t *)(smem + t.oBar);

  const int G = t.G, nom = g.n_om, nnu = g.n_nu;
  const int p0 = blockIdx.x * G, k = blockIdx.y;
  const int ik = k / nnu, n = g.n_lo + k % nnu;
  const long long nn = g.n;
  const long long ochan = (long long)pass.nq * nom * nn * ld;  // channel stride of the outputs
  const int tid = threadIdx.x;
  const int cu = tid % t.upr, row0 = tid / t.upr;
  const bool worker = tid < t.upr * t.rows;  // the padding threads only take part in the barriers
  const int a = cu / t.hb;
  const int col0 = p0 * nnu + 4 * cu;  // first output column of this thread: p_a Nnu + npi0

  for (int i = tid; i < 2 * G * nom; i += blockDim.x) {
    const int x = mdiv(i, t.m_gn), rem = i - x * G * nom;
    const int b = mdiv(rem, t.m_nom), mt = rem - b * nom;
    const int Qt = tsub(g, t, p0 + b, ik) * nom + mt;
    FK[i] = f2(k1[(long long)x * g.nQ + Qt] + k2row[((long long)x * g.n + k) * g.nQ + Qt]);
  }
  const int nsteps = FUSED ? g.nk : 2 * pass.nq;
  // step -> (kind, q): FUSED walks q = 0..nk-1 (both kinds); otherwise target qt, d/m then s/t
  auto step_q = [&](int st) { return FUSED ? st : pass.qb + st / 2; };
  auto step_dm = [&](int st) { return FUSED || (st & 1) == 0; };
  if (tid < G) step_table(g, t, step_dm(0), step_q(0), ik, p0, tid, stab[0] + tid * T_N);
  if (PF == V_F16P && tid < 8) ssc[tid] = fsc[tid < 4 ? FSC_SA + tid : FSC_SB + tid - 4];
  if (tid == 0) {
    abort_flag = 0;
    tc::mbar_init(bar, 1);
    tc::mbar_fence_init();
  }
  __syncthreads();

  const float2 l0 = f2(lam.l[0]), l1 = f2(lam.l[1]), l2 = f2(lam.l[2]), l3 = f2(lam.l[3]);
  const float2 twoU = make_float2((float)(2.0 * g.U), 0.f);
  CSum2 acc;  // this thread's dF box sum: a compensated sum of the per-step partial sums
  Ctx c{Rt, Pt, St, FK, G, t.RS, t.RA, t.PW, t.BW, t.PPW, nom, nnu, a, 4 * (cu % t.hb), n, row0, a * t.sh};
  // this thread's delay line: a slots of 8 float4 (Gamma X_s, Gamma X_t, F_s, F_t of 4 elements)
  float4 *dl = ring + (size_t)8 * t.ring_n * (a * (a - 1) / 2) + row0 * t.hb + cu % t.hb;
  uint32_t phase = 0;

  int qy = 0;    // FUSED: y coordinate of q (q = step)
  int slot = 0;  // FUSED, a > 0: qy % a, this step's delay-line slot
  for (int step = 0; step < nsteps;
       ++step, qy = (qy + 1 == g.L) ? 0 : qy + 1, slot = (qy == 0 || slot + 1 == a) ? 0 : slot + 1) {
    const bool do_dm = step_dm(step), do_st = FUSED || !do_dm;
    const int qt = step_q(step);
    const int *tb = stab[step & 1];
    issue_gather(g, t, &rmap, tb, phi, k, p0, Rt, Pt, St, bar, do_dm);
    if (!tc::mbar_wait_ns(bar, phase, GATHER_WAIT_NS)) abort_flag = 1;
    __syncthreads();
    if (abort_flag) {
      if (tid == 0) {
        atomicExch(err, 1);
        tc::mbar_wait_ns(bar, phase, GATHER_WAIT_NS);  // the copies still in flight
      }
      __syncthreads();
      return;
    }
    phase ^= 1u;
    if (tid < G && step + 1 < nsteps)
      step_table(g, t, step_dm(step + 1), step_q(step + 1), ik, p0, tid, stab[(step + 1) & 1] + tid * T_N);

    float2 sacc = make_float2(0.f, 0.f);  // this step's part of the dF box sum
    for (int mi = row0; worker && mi < nom; mi += t.rows) {
      c.mi = mi;
      const int m = g.m_lo + mi;
      float2 gx[2][4], f[2][4];
      if (do_dm) {
        const int Q = qt * nom + mi;
        float2 xq[4];
        load4(xph + (long long)Q * nn + col0, xq);
        const float2 gkq = gtab[(long long)tb[T_CM] * g.n_g + (n + m - g.g_lo)];
        elems_dm<TAB>(g, c, lam, l0, l1, twoU, xq, gkq, gx, f, sacc);
        const long long o = ((long long)(Q - pass.qb * nom) * nn + k) * ld + col0;
        put_ops<PF>(gam, fv, ps, o, gx[0], f[0], ssc, 0);
        put_ops<PF>(gam, fv, ps, ochan + o, gx[1], f[1], ssc, 1);
      }
      if (do_st) {
        const int qp = tb[a * T_N + T_QS];  // q' of this thread's block
        const int Qp = qp * nom + mi;
        float2 xqp[4];
        load4(xpp + (long long)Qp * nn + col0, xqp);
        const float2 gqk = gtab[(long long)tb[a * T_N + T_PQK] * g.n_g + (m - n - 1 - g.g_lo)];
        elems_st<TAB>(g, c, lam, l2, l3, twoU, xqp, gqk, gx, f, sacc);
        if constexpr (FUSED) {
          // Block 0 of row q0 = k + p_0 + q is produced now; block a >= 1 of that row was
          // produced a steps ago (same lattice row of q) and waits in the delay line.  All
          // blocks of the row are stored by one put4 (one warp instruction per plane).
          float4 *sl = dl + (size_t)8 * t.ring_n * (a > 0 ? slot : 0);
          if (a == 0 || qy >= a) {
            float2 wg[2][4], wf[2][4];
            if (a == 0) {
#pragma unroll
              for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int i = 0; i < 4; ++i) wg[h][i] = gx[h][i], wf[h][i] = f[h][i];
            } else {
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const float4 u0 = sl[(4 * h + 0) * t.ring_n], u1 = sl[(4 * h + 1) * t.ring_n];
                const float4 v0 = sl[(4 * h + 2) * t.ring_n], v1 = sl[(4 * h + 3) * t.ring_n];
                wg[h][0] = make_float2(u0.x, u0.y), wg[h][1] = make_float2(u0.z, u0.w);
                wg[h][2] = make_float2(u1.x, u1.y), wg[h][3] = make_float2(u1.z, u1.w);
                wf[h][0] = make_float2(v0.x, v0.y), wf[h][1] = make_float2(v0.z, v0.w);
                wf[h][2] = make_float2(v1.x, v1.y), wf[h][3] = make_float2(v1.z, v1.w);
              }
            }
            const int q0 = tb[T_Q0];
            const long long o = ((long long)(q0 * nom + mi) * nn + k) * ld + col0;
            put_ops<PF>(gam, fv, ps, 2 * ochan + o, wg[0], wf[0], ssc, 2);
            put_ops<PF>(gam, fv, ps, 3 * ochan + o, wg[1], wf[1], ssc, 3);
          }
          if (a > 0) {
            if (qy + a >= g.L) {
              // block 0 of this row came earlier in the lattice row of q: store this block alone
              const long long o = ((long long)Qp * nn + k) * ld + col0;
              put_ops<PF>(gam, fv, ps, 2 * ochan + o, gx[0], f[0], ssc, 2);
              put_ops<PF>(gam, fv, ps, 3 * ochan + o, gx[1], f[1], ssc, 3);
            } else {
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                sl[(4 * h + 0) * t.ring_n] = make_float4(gx[h][0].x, gx[h][0].y, gx[h][1].x, gx[h][1].y);
                sl[(4 * h + 1) * t.ring_n] = make_float4(gx[h][2].x, gx[h][2].y, gx[h][3].x, gx[h][3].y);
                sl[(4 * h + 2) * t.ring_n] = make_float4(f[h][0].x, f[h][0].y, f[h][1].x, f[h][1].y);
                sl[(4 * h + 3) * t.ring_n] = make_float4(f[h][2].x, f[h][2].y, f[h][3].x, f[h][3].y);
              }
            }
          }
        } else {
          const long long o = ((long long)(Qp - pass.qb * nom) * nn + k) * ld + col0;
          put_ops<PF>(gam, fv, ps, 2 * ochan + o, gx[0], f[0], ssc, 2);
          put_ops<PF>(gam, fv, ps, 3 * ochan + o, gx[1], f[1], ssc, 3);
        }
      }
    }
    acc.add(sacc);
    __syncthreads();  // the tiles are free for the next gather
  }

  // dF box sum per (k, p_a): the threads of block a
  red[tid] = acc.get();
  __syncthreads();
  if (tid < G) {
    double2 s = make_double2(0.0, 0.0);
    for (int r = 0; r < t.rows; ++r)
      for (int cc = 0; cc < t.hb; ++cc) s = s + red[r * t.upr + tid * t.hb + cc];
    // -(U/4)(T/N)^2 sum GGG: one T/N sits in X
    const double pref = -(g.U * 0.25) * g.T / g.nk;
    double2 v = pref * s;
    const long long di = (long long)k * g.nk + p0 + tid;
    if (pass.accumulate) v = v + dfpart[di];
    dfpart[di] = v;
  }
}

int align128(int x) { return (x + 127) & ~127; }

// Dynamic shared memory of a CTA such that two fit on an SM (228 KB, less 1 KB reserved
// and the static arrays per CTA, 4480 bytes with the FP16 scales).
constexpr int SMEM_TWO_PER_SM = (228 * 1024) / 2 - 1024 - 4480;

// Tile geometry for G blocks; false if it does not serve the shape.
bool tiled_geo_g(const Grid &g, bool fused, int G, TGeo &t) {
  // the multiply-high divisions (mdiv) are exact for dividends below 2^16
  if (6 * G * g.n_om >= 65536 || g.L * g.L >= 65536) return false;
  t.G = G;
  t.hb = g.n_nu / 4;
  t.upr = G * t.hb;
  if (t.upr > TT) return false;
  // rows of a sweep balanced over the sweeps that NOmega needs
  const int sweeps = (g.n_om + TT / t.upr - 1) / (TT / t.upr);
  t.rows = (g.n_om + sweeps - 1) / sweeps;
  t.nthr = (t.upr * t.rows + 31) / 32 * 32;
  if (fused && t.rows < g.n_om) return false;
  if (g.n_om > 256 || g.n_nu + 6 > 256) return false;  // TMA box dimensions
  // R rows: TMA boxes of Nnu + 2 max(G - 1, 1) words (16-byte multiples, = 2 mod 4 words so
  // that consecutive transfer rows fall on different banks), block a shifted by 2a words
  // (bank spread between the blocks); blocks at 128-byte boundaries (TMA destinations)
  t.sh = G > 1 ? 2 : 0;
  t.RS = g.n_nu + 2 * std::max(G - 1, 1);
  t.RA = (g.n_om * t.RS + 15) / 16 * 16;
  t.BW = g.n_nu + 2;
  t.PW = G * t.BW;
  t.PPW = G * g.n_nu + 2;
  t.ring_n = t.hb * t.rows;
  int o = 0;
  t.oR = o;
  o = align128(o + 2 * G * t.RA * 8);
  t.oP = o;
  o = align128(o + 2 * g.n_om * t.PPW * 8);
  t.oS = o;
  o = align128(o + 2 * g.n_om * t.PW * 8);
  t.oFK = o;
  o = align128(o + 2 * G * g.n_om * 8);
  t.oRing = o;
  if (fused) o = align128(o + 16 * 8 * t.ring_n * (G * (G - 1) / 2));
  t.oBar = o;
  t.smem = o + 8;
  t.tx = 2 * G * g.n_om * t.RS * 8 + 4 * G * g.n_om * g.n_nu * 8;  // R boxes (whole boxes), P, S
  auto magic = [](unsigned d) { return (unsigned long long)(0xFFFFFFFFull / d) + 1ull; };
  t.m_per = magic(2 * G * g.n_om);
  t.m_gn = magic(G * g.n_om);
  t.m_nom = magic(g.n_om);
  t.m_L = magic(g.L);
  return t.smem <= 200 * 1024;
}

// Geometry of the launch; false if the shape is not served by the tiled kernel (Nnu % 4 != 0).
// G is the widest block count dividing L (4, 2, 1) whose CTA leaves room for a second one on
// the SM, else the widest that fits at all.  fused: the delay line is wanted.
bool tiled_geo(const Grid &g, bool fused, TGeo &t) {
  if (g.n_nu % 4 != 0) return false;
  bool any = false;
  TGeo first;
  for (int G = 4; G >= 1; G /= 2) {
    if (g.L % G != 0) continue;
    TGeo c;
    if (!tiled_geo_g(g, fused, G, c)) continue;
    if (c.smem <= SMEM_TWO_PER_SM) {
      t = c;
      return true;
    }
    if (!any) first = c, any = true;
  }
  if (any) t = first;
  return any;
}

template <bool FUSED, bool TAB, int PF>
cudaError_t tiled_launch(cudaStream_t st, const Grid &g, const TGeo &t, Buffers &b, const Lam &lam, const Pass &p,
                         long long ps) {
  auto kfn = assemble_tiled_kernel<FUSED, TAB, PF>;
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, t.smem);
  if (e != cudaSuccess) return e;
  CUtensorMap rmap;
  if (make_phi_rows_map(b.phi, g.n, 4LL * g.nQ, t.RS, g.n_om, &rmap) != CUDA_SUCCESS) return cudaErrorInvalidValue;
  kfn<<<dim3(g.nk / t.G, g.n), t.nthr, t.smem, st>>>(
      g, t, (const float2 *)b.phi, (uint16_t *)b.gam, (uint16_t *)b.fv, ps, b.ld, b.k1, b.k2row, b.xph32, b.xpp32,
      b.gtab32, b.dfpart, lam, p, b.fsc, (int *)(b.scal + 4), rmap);
  return cudaGetLastError();
}

template <int PF>
cudaError_t tiled_dispatch(cudaStream_t st, const Grid &g, const TGeo &t, bool fused, bool tab, Buffers &b,
                           const Lam &lam, const Pass &p, long long ps) {
  if (fused)
    return tab ? tiled_launch<true, true, PF>(st, g, t, b, lam, p, ps) : tiled_launch<true, false, PF>(st, g, t, b, lam, p, ps);
  return tab ? tiled_launch<false, true, PF>(st, g, t, b, lam, p, ps) : tiled_launch<false, false, PF>(st, g, t, b, lam, p, ps);
}

}  // namespace

bool assemble_tiled_ok(const Grid &g) {
  TGeo t;
  return tiled_geo(g, false, t);
}

cudaError_t launch_assemble_tiled(cudaStream_t st, const Grid &g, Buffers &b, const Lam &lam, const Pass &p,
                                  long long ps, bool tab) {
  TGeo t;
  const bool fused = p.fused && tiled_geo(g, true, t);
  if (!fused && !tiled_geo(g, false, t)) return cudaErrorInvalidValue;
  if (b.vfmt == V_F16P) return tiled_dispatch<V_F16P>(st, g, t, fused, tab, b, lam, p, ps);
  return tiled_dispatch<V_BF16P>(st, g, t, fused, tab, b, lam, p, ps);
}

}  // namespace pq
