// C ABI of the GB300 parquet solver (include/parquet.h): context life cycle,
// device memory, and the iteration driver that sequences the steps of one
// self-consistent parquet iteration (Sec. II) on one stream.
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <initializer_list>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pq_assemble.cuh"
#include "pq_ctx.h"
#include "pq_tc.cuh"

using pq::Buffers;
using pq::Grid;
using pq::Sizes;

namespace {

std::string g_init_err;
constexpr double kDivergeFactor = 10.0;  // divergence detection: growth over the first max |dSigma|

const char *kStepNames[PQ_NSTEPS] = {"dyson",    "bubbles",      "kernels", "sigma1", "sigma2",
                                     "assemble", "sigma_update", "bse",     "total"};

}  // namespace

pq_status pq::fail(pq_ctx *c, pq_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) {
    c->err = buf;
    if (s == PQ_ECUDA || s == PQ_ENAN) c->poisoned = true;
  } else {
    g_init_err = buf;
  }
  return s;
}

namespace {
using pq::fail;

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(c, PQ_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

void *dalloc(pq_ctx *c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void *p = nullptr;
  if (c->opt.dev_alloc) {
    p = c->opt.dev_alloc(bytes, c->opt.alloc_ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    c->allocs.push_back({p, bytes});
    c->bytes += bytes;
  }
  return p;
}

void release_all(pq_ctx *c) {
  for (auto &a : c->allocs) {
    if (c->opt.dev_free)
      c->opt.dev_free(a.first, a.second, c->opt.alloc_ctx);
    else
      cudaFree(a.first);
  }
  c->allocs.clear();
  c->bytes = 0;
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_p.
void gauss_legendre(int p, std::vector<double> &x, std::vector<double> &w) {
  x.assign(p, 0.0);
  w.assign(p, 0.0);
  for (int i = 0; i < p; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (p + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= p; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      if (p == 1) {
        p1 = z;
        p0 = 1.0;
      }
      dp = p * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    x[p - 1 - i] = z;
    w[p - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

size_t vbytes(const pq_ctx *c) {
  return (size_t)4 * c->g.nQ * (size_t)c->g.n * c->g.n * (c->c64 ? sizeof(float2) : sizeof(double2));
}

// Bytes per complex element of the BSE operands (gam, fv) in each storage format.
size_t gam_es(int vfmt) { return vfmt == pq::V_C128 ? 16 : 8; }
size_t fv_es(int vfmt) { return vfmt == pq::V_C128 ? 16 : vfmt == pq::V_BF16P ? 12 : 8; }

int num_passes(const pq_ctx *c) { return (c->g.nk + c->b.q_chunk - 1) / c->b.q_chunk; }

size_t b_fv_bytes(const pq_ctx *c) {
  return (size_t)c->b.q_chunk * 4 * c->g.n_om * (size_t)c->g.n * c->b.ld * fv_es(c->b.vfmt);
}

__global__ void phi_from_c128(float2 *dst, const double2 *src, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}

// Density per site (both spins) of the state's G at chemical potential mu, and d n / d mu
// (square lattice): the device sums the Matsubara remainders, the closed-form tails are added
// here.  Synchronous.
pq_status density_at(pq_ctx *c, double mu, double *n, double *dn) {
  Grid g = c->g;
  g.mu = mu;
  double *out = c->b.scal + 6;
  CK(pq::launch_tail_c1(c->st, g, c->b.sigma, c->b.scal + 3));
  CK(pq::launch_density(c->st, g, c->z.M, c->b.sigma, c->b.scal + 3, out));
  double h[2];
  CK(cudaMemcpyAsync(h, out, sizeof h, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  double sum_c2 = 0.0;  // sum_k (eps_k - mu)
  for (int ik = 0; ik < g.nk; ++ik) {
    const int ix = ik / g.L, iy = ik % g.L;
    sum_c2 += -2.0 * g.hop * (std::cos(2.0 * M_PI * ix / g.L) + std::cos(2.0 * M_PI * iy / g.L)) - mu;
  }
  *n = (2.0 / g.nk) * (0.5 * g.nk - g.beta * sum_c2 / 4.0) + 2.0 * g.T / g.nk * h[0];
  *dn = 0.5 * g.beta + 2.0 * g.T / g.nk * h[1];
  return PQ_OK;
}

// Chemical potential that gives the state's G the target density: Newton steps on n(mu), kept
// inside a bracket that bisection shrinks whenever a step leaves it (n increases with mu).
pq_status find_mu(pq_ctx *c, double target, double *mu_out) {
  double lo = -20.0 * std::max(1.0, std::fabs(c->g.hop)) - 10.0 * std::fabs(c->g.U), hi = -lo;
  double mu = c->g.mu, n = 0.0, dn = 0.0;
  for (int it = 0; it < 100; ++it) {
    pq_status s = density_at(c, mu, &n, &dn);
    if (s != PQ_OK) return s;
    const double f = n - target;
    if (std::fabs(f) < 1e-14 * std::max(1.0, target)) break;
    if (f > 0) hi = mu;
    else lo = mu;
    double next = dn > 0 ? mu - f / dn : 0.5 * (lo + hi);
    if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
    if (hi - lo < 1e-15 * std::max(1.0, std::fabs(mu))) break;
    mu = next;
  }
  if (!std::isfinite(n) || std::fabs(n - target) > 1e-9)
    return fail(c, PQ_ENOTCONV, "mu search: density %.15g instead of %.15g", n, target);
  *mu_out = mu;
  return PQ_OK;
}

// Device work of one iteration, queued on the context's stream without waiting.  With
// bse == false the products of a single-pass iteration are left out (a batch runs them in
// its grouped launch); timing records the step events.
}  // namespace

namespace pq {
// Named host range (NVTX) around the enqueue of one step group, so that a profiler's timeline
// (or ncu --nvtx-include "pq.assemble/") ties the kernels to the steps of the iteration.  The
// calls cost nothing when no profiler is attached.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace pq

pq_status pq::enqueue_iteration(pq_ctx *c, bool bse, bool timing) {
  NvtxRange whole("pq.iteration");
  cudaStream_t st = c->st;
  Grid &g = c->g;
  Buffers &b = c->b;
  const bool tm = timing;
  auto mark = [&](int i) {
    if (tm) cudaEventRecord(c->ev[i], st);
  };
  if (c->opt.target_density > 0.0) {
    // fixed density: mu for the state's Sigma, then the iteration at that mu
    double mu = g.mu;
    pq_status s = find_mu(c, c->opt.target_density, &mu);
    if (s != PQ_OK) return s;
    g.mu = mu;
  }
  mark(0);
  {
    NvtxRange r("pq.one_body");
    CK(pq::launch_tail_and_green(st, g, b));
    mark(1);
    CK(pq::launch_bubbles(st, g, b));
    if (b.vfmt == pq::V_F16P) CK(pq::launch_split_scales(st, b, c->lam_max));
    mark(2);
  }
  {
    NvtxRange r("pq.kernels");
    CK(pq::launch_kernels_extract(st, g, b, c->c64, pq::split_planes(b.vfmt) && c->krow_ok));
  }
  mark(3);
  {
    NvtxRange r("pq.sigma");
    if (b.truncated) {
      mark(4);
      CK(pq::launch_sigma_truncated(st, g, b));
    } else {
      CK(pq::launch_sigma1(st, g, c->z, pq::sigma1_args(b, b.sigma, b.scal, b.sigma1)));
      mark(4);
      CK(pq::launch_sigma2(st, g, c->z, b));
    }
  }
  mark(5);
  const long long nn = g.n;
  const int np = num_passes(c);
  const bool fused = (np == 1);
  c->chi_ready = false;
  for (int ip = 0; ip < np; ++ip) {
    pq::Pass p;
    p.qb = ip * b.q_chunk;
    p.nq = std::min(b.q_chunk, g.nk - p.qb);
    p.fused = fused;
    p.accumulate = ip > 0;
    const int zc = p.nq * g.n_om;
    const long long q0 = (long long)p.qb * g.n_om;
    if (tm && !fused) cudaEventRecord(c->pev[3 * ip], st);
    {
      NvtxRange r("pq.assemble");
      CK(pq::launch_assemble(st, g, b, c->lam, p));
      if (!fused) CK(pq::launch_chi(st, g, b, p.qb, p.nq));
    }
    if (fused) {
      mark(6);
      CK(pq::launch_sigma_update(st, g, b));
      mark(7);
    } else if (tm) {
      cudaEventRecord(c->pev[3 * ip + 1], st);
    }
    void *phi_out = fused ? b.phi : b.phi_new;
    if (pq::split_planes(b.vfmt) && ip == 0)  // the products of this iteration sum the new Phi's row edges
      CK(cudaMemsetAsync(b.krow, 0, sizeof(double2) * 4 * (size_t)g.n * g.nQ, st));
    NvtxRange rb("pq.bse");
    if (!bse) {
      // left to the caller
    } else if (pq::split_planes(b.vfmt)) {
      const pq::BseProblem *pr = c->probs + (fused ? 0 : (c->swapped ? np : 0) + ip);
      const int bnc = c->bse_cols;
      CK(pq::launch_bse_tma(st, bnc, b.vfmt == pq::V_F16P, pr, 1, pq::bse_tiles(bnc, g.n, 4 * zc),
                            (int *)(b.scal + 4), 0));
    } else {
      // in-place products: a separate Jacobi target first receives the old slices
      const size_t es = b.vfmt == pq::V_C128 ? sizeof(double2) : sizeof(float2);
      const int nr = fused ? 1 : 4;  // one launch over all channels, or one per channel slice range
      for (int r = 0; r < nr; ++r) {
        const size_t po = ((size_t)r * g.nQ + q0) * nn * nn * es, oo = (size_t)r * zc * nn * nn * es;
        char *dst = (char *)phi_out + po;
        if (!fused) CK(cudaMemcpyAsync(dst, (const char *)b.phi + po, (size_t)zc * nn * nn * es,
                                       cudaMemcpyDeviceToDevice, st));
        const int batch = fused ? 4 * zc : zc;
        if (b.vfmt == pq::V_C128) {
          CK(pq::zgemm_fp64(st, g.n, g.n, g.n, make_double2(g.mix, 0.0), (const double2 *)((char *)b.gam + oo), g.n,
                            nn * nn, (const double2 *)((char *)b.fv + oo), g.n, nn * nn,
                            make_double2(1.0 - g.mix, 0.0), (double2 *)dst, g.n, nn * nn, batch));
        } else {
          CK(pq::launch_bse_split(st, g.n, batch, (const float2 *)((char *)b.gam + oo),
                                  (const float2 *)((char *)b.fv + oo), (float2 *)dst, (float)g.mix,
                                  (int *)(b.scal + 4)));
        }
      }
    }
    if (tm && !fused) cudaEventRecord(c->pev[3 * ip + 2], st);
    c->last_qb = p.qb;
  }
  if (!fused) {
    mark(6);
    CK(pq::launch_sigma_update(st, g, b));
    mark(7);
    std::swap(b.phi, b.phi_new);
    c->swapped = !c->swapped;
    c->chi_ready = true;
  }
  mark(8);
  if (pq::split_planes(b.vfmt)) c->krow_ok = true;
  return PQ_OK;
}

// Host side of the end of an iteration: h = the first five scalars of the context
// (max |dSigma|, non-finite flag, tensor-core timeout flag) read after the work completed.
pq_status pq::finish_iteration(pq_ctx *c, const double *h, double *dmax, bool timing) {
  const int np = num_passes(c);
  const bool fused = (np == 1);
  int timeout_flag;
  std::memcpy(&timeout_flag, &h[4], sizeof timeout_flag);
  if (timeout_flag) {
    c->poisoned = true;
    return fail(c, PQ_ETIMEOUT, "a bounded device wait (tensor-core pipeline) gave up; the state is invalid");
  }
  auto elapsed = [](cudaEvent_t a, cudaEvent_t z) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, z) != cudaSuccess) {
      cudaGetLastError();  // leave no error for the next launch check to find
      ms = 0.f;
    }
    return ms;
  };
  if (timing) {
    for (int i = 0; i < PQ_NSTEPS - 1; ++i) c->times[i] = elapsed(c->ev[i], c->ev[i + 1]);
    c->times[PQ_NSTEPS - 1] = elapsed(c->ev[0], c->ev[PQ_NSTEPS - 1]);
    if (!fused) {
      // the passes interleave assembly and products: sum each over the passes
      float t_asm = 0.f, t_bse = 0.f;
      for (int ip = 0; ip < np; ++ip) {
        t_asm += elapsed(c->pev[3 * ip], c->pev[3 * ip + 1]);
        t_bse += elapsed(c->pev[3 * ip + 1], c->pev[3 * ip + 2]);
      }
      c->times[5] = t_asm;  // assemble (with chi)
      c->times[7] = t_bse;  // bse
    }
  }
  if (h[2] != 0.0 || !std::isfinite(h[1])) return fail(c, PQ_ENAN, "non-finite self-energy after iteration");
  *dmax = h[1];
  c->iterations++;
  return PQ_OK;
}

namespace {

pq_status run_iteration(pq_ctx *c, double *dmax) {
  const bool tm = c->opt.time_steps != 0;
  pq_status s = pq::enqueue_iteration(c, true, tm);
  if (s != PQ_OK) return s;
  double h[5];
  CK(cudaMemcpyAsync(h, c->b.scal, sizeof h, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return pq::finish_iteration(c, h, dmax, tm);
}

}  // namespace

namespace {
// One thread waits on an mbarrier that expects one arrival which never comes.
__global__ void wait_selftest_kernel(uint64_t limit_ns, int *flag) {
  __shared__ __align__(8) uint64_t bar;
  pq::tc::mbar_init(&bar, 1);
  pq::tc::mbar_fence_init();
  if (!pq::tc::mbar_wait_ns(&bar, 0, limit_ns)) atomicExch(flag, 1);
}
}  // namespace

namespace pq {
// Message for pq_last_error(NULL) from a call that has no context.
void set_context_free_error(const char *msg) { g_init_err = msg; }
}  // namespace pq

extern "C" {

void pq_default_options(pq_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->precision = PQ_FP64;
  o->mix_alpha = 0.5;
  o->sigma2_box_factor = 3;
  o->hop = 1.0;
  o->tau_panels = 64;
  o->tau_order = 16;
  o->tau_matsubara = 2048;
}

pq_status pq_init(pq_ctx **out, int lattice, double beta, double U, double mu, int L, int n_nu, int n_Omega,
                  const pq_options *opt) {
  if (!out) return fail(nullptr, PQ_EINVAL, "out is NULL");
  *out = nullptr;
  pq_options o;
  pq_default_options(&o);
  if (opt) o = *opt;
  if (lattice != PQ_BETHE && lattice != PQ_SQUARE) return fail(nullptr, PQ_EINVAL, "unknown lattice %d", lattice);
  if (!(beta > 0.0) || !std::isfinite(beta)) return fail(nullptr, PQ_EINVAL, "beta must be positive");
  if (L < 1 || (lattice == PQ_BETHE && L != 1)) return fail(nullptr, PQ_EINVAL, "L must be >= 1 (1 for Bethe)");
  if (n_nu < 2 || n_nu % 2) return fail(nullptr, PQ_EINVAL, "n_nu must be even and >= 2");
  if (n_Omega < 1) return fail(nullptr, PQ_EINVAL, "n_Omega must be >= 1");
  if (o.sigma2_box_factor < 1) return fail(nullptr, PQ_EINVAL, "sigma2_box_factor must be >= 1");
  if (o.tau_panels < 1 || o.tau_order < 2 || o.tau_matsubara < 1)
    return fail(nullptr, PQ_EINVAL, "bad imaginary-time quadrature sizes");
  if (o.precision < PQ_FP64 || o.precision > PQ_SPLIT_FP16X3) return fail(nullptr, PQ_EINVAL, "unknown precision");
  if (o.precision == PQ_SPLIT_BF16X6)
    return fail(nullptr, PQ_EINVAL, "BF16x6 split products are not available in this build");
  if (!(o.mix_alpha > 0.0 && o.mix_alpha <= 1.0)) return fail(nullptr, PQ_EINVAL, "mix_alpha must be in (0, 1]");
  if ((o.dev_alloc == nullptr) != (o.dev_free == nullptr))
    return fail(nullptr, PQ_EINVAL, "dev_alloc and dev_free must be given together");
  if (o.bse_tile_cols != 0 && o.bse_tile_cols != 64 && o.bse_tile_cols != 128)
    return fail(nullptr, PQ_EINVAL, "bse_tile_cols must be 0, 64 or 128");
  if (o.diverge_window < 0) return fail(nullptr, PQ_EINVAL, "diverge_window must be >= 0");
  if (o.target_density < 0.0 || o.target_density >= 2.0 || (o.target_density > 0.0 && lattice != PQ_SQUARE))
    return fail(nullptr, PQ_EINVAL, "target_density must be 0 (fixed mu) or in (0, 2) on the square lattice");

  pq_ctx *c = new pq_ctx();
  c->opt = o;
  c->st = (cudaStream_t)o.cuda_stream;
  c->c64 = (o.precision != PQ_FP64);
  Grid &g = c->g;
  g.lattice = lattice;
  g.L = L;
  g.nk = L * L;
  g.n_nu = n_nu;
  g.n_om = n_Omega;
  g.n = g.nk * n_nu;
  g.nQ = g.nk * n_Omega;
  g.n_ext = n_Omega + n_nu - 1;
  g.n_lo = -n_nu / 2;
  g.n_hi = n_nu / 2 - 1;
  g.m_lo = -(n_Omega / 2);
  g.m_hi = g.m_lo + n_Omega - 1;
  g.e_lo = g.m_lo + g.n_lo;
  g.e_hi = g.m_hi + g.n_hi;
  const int f = o.sigma2_box_factor;
  g.bf_lo = -(f * n_nu) / 2;
  g.bf_hi = (f * n_nu) / 2 - 1;
  g.bb_lo = -((f * n_Omega) / 2);
  g.bb_hi = g.bb_lo + f * n_Omega - 1;
  g.beta = beta;
  g.T = 1.0 / beta;
  g.U = U;
  g.mu = mu;
  g.hop = o.hop;
  g.mix = o.mix_alpha;
  // frequency range of the Sigma~2 bubble tables and of the G table
  Sizes &z = c->z;
  int j_lo = std::min(std::min(g.bf_lo, g.e_lo + g.bb_lo), g.bb_lo - g.e_hi - 1 - g.m_hi);
  int j_hi = std::max(std::max(g.bf_hi, g.e_hi + g.bb_hi), g.bb_hi - g.e_lo - 1 - g.m_lo);
  z.j_lo = j_lo;
  z.nj = j_hi - j_lo + 1;
  int lo = std::min({j_lo, j_lo + g.m_lo, g.m_lo - j_hi - 1, g.e_lo + g.m_lo, g.m_lo - g.e_hi - 1, g.e_lo + g.bb_lo});
  int hi = std::max({j_hi, j_hi + g.m_hi, g.m_hi - j_lo - 1, g.e_hi + g.m_hi, g.m_hi - g.e_lo - 1, g.e_hi + g.bb_hi});
  g.g_lo = lo;
  g.n_g = hi - lo + 1;
  z.M = o.tau_matsubara;
  z.ntau = o.tau_panels * o.tau_order;
  c->lam[0] = U;
  c->lam[2] = -U;
  c->lam[4] = 2.0 * U;
  c->lam[6] = 0.0;
  for (int r = 0; r < 4; ++r) c->lam_max[r] = std::fabs(c->lam[2 * r]);

  Buffers &b = c->b;
  b.vfmt = o.precision == PQ_FP64            ? pq::V_C128
           : o.precision == PQ_SPLIT_TF32X3  ? pq::V_C64
           : o.precision == PQ_SPLIT_FP16X3  ? pq::V_F16P
                                             : pq::V_BF16P;
  b.ld = pq::split_planes(b.vfmt) ? (g.n + 7) / 8 * 8 : g.n;  // TMA rows: multiples of 16 bytes
  c->bse_cols = o.bse_tile_cols ? o.bse_tile_cols : 128;  // complex columns per tile of the products
  if (o.q_chunk < 0) {
    delete c;
    return fail(nullptr, PQ_EINVAL, "q_chunk must be >= 0");
  }
  if (o.assembly < 0 || o.assembly > 1) {
    delete c;
    return fail(nullptr, PQ_EINVAL, "assembly must be 0 (tiled) or 1 (general)");
  }
  b.assembly = o.assembly;
  if (o.kernel_level < 0 || o.kernel_level > 2 || o.edge_rule < 0 || o.edge_rule > 1) {
    delete c;
    return fail(nullptr, PQ_EINVAL, "kernel_level must be 0, 1 or 2 and edge_rule 0 or 1");
  }
  if (o.sde < 0 || o.sde > 1) {
    delete c;
    return fail(nullptr, PQ_EINVAL, "sde must be 0 (regulated) or 1 (truncated)");
  }
  b.truncated = o.sde == 1;
  b.first_level = o.kernel_level == 1;
  b.lower_edge = o.edge_rule == 1;

  if (pq::assemble_smem_bytes(g, c->c64) > 200 * 1024) {
    delete c;
    return fail(nullptr, PQ_EINVAL, "NOmega*Nnu = %d too large for one vertex block in shared memory",
                n_Omega * n_nu);
  }

  // device memory: the state Phi, and the operand buffers of q_chunk q-momenta per pass; with
  // fewer than all momenta per pass the Jacobi update needs a second Phi
  const size_t vb = vbytes(c);
  const size_t cs = sizeof(double2);
  const size_t per_q = (size_t)4 * g.n_om * (size_t)g.n * b.ld * (gam_es(b.vfmt) + fv_es(b.vfmt));
  if (o.q_chunk > 0) {
    b.q_chunk = std::min(o.q_chunk, g.nk);
  } else {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      fr = 0;
    }
    const size_t small = (size_t)64 << 20, margin = (size_t)2 << 30;  // tables, and room for the caller
    const size_t avail = fr > margin ? fr - margin : 0;
    if (fr == 0 || vb + per_q * g.nk + small <= avail) {
      b.q_chunk = g.nk;
    } else {
      const size_t left = avail > 2 * vb + small ? avail - 2 * vb - small : 0;
      b.q_chunk = (int)std::max<size_t>(1, std::min<size_t>(g.nk, left / per_q));
    }
  }
  const bool several = b.q_chunk < g.nk;
  const size_t obytes_g = (size_t)b.q_chunk * 4 * g.n_om * (size_t)g.n * b.ld * gam_es(b.vfmt);
  const size_t obytes_f = (size_t)b.q_chunk * 4 * g.n_om * (size_t)g.n * b.ld * fv_es(b.vfmt);
  struct Req {
    void **p;
    size_t bytes;
  } reqs[] = {
      {&b.phi, vb},
      {&b.phi_new, several ? vb : 0},
      {&b.gam, obytes_g},
      {&b.fv, obytes_f},
      {(void **)&b.sigma, cs * g.nk * g.n_ext},
      {(void **)&b.sigma_new, cs * g.nk * g.n_ext},
      {(void **)&b.sigma1, cs * g.nk * g.n_ext},
      {(void **)&b.sigma2, cs * g.nk * g.n_ext},
      {(void **)&b.gtab, cs * g.nk * g.n_g},
      {(void **)&b.xph, cs * g.nQ * (size_t)g.n},
      {(void **)&b.xpp, cs * g.nQ * (size_t)g.n},
      {(void **)&b.gtab32, c->c64 ? sizeof(float2) * g.nk * g.n_g : 0},
      {(void **)&b.xph32, c->c64 ? sizeof(float2) * g.nQ * (size_t)g.n : 0},
      {(void **)&b.xpp32, c->c64 ? sizeof(float2) * g.nQ * (size_t)g.n : 0},
      {(void **)&b.k1, cs * 4 * g.nQ},
      {(void **)&b.k2row, cs * 4 * (size_t)g.n * g.nQ},
      {(void **)&b.k2col, cs * 4 * (size_t)g.n * g.nQ},
      {(void **)&b.krow, pq::split_planes(b.vfmt) ? cs * 4 * (size_t)g.n * g.nQ : 0},
      {(void **)&b.fsc, b.vfmt == pq::V_F16P ? sizeof(float) * pq::FSC_N : 0},
      {(void **)&b.dfpart, cs * (size_t)g.n * g.nk},
      {(void **)&b.scal, 8 * sizeof(double)},
      {(void **)&b.s1_R, cs * g.nk * 2 * (size_t)z.M},
      {(void **)&b.s1_E, cs * 2 * (size_t)z.M * z.ntau},
      {(void **)&b.s1_Ef, cs * (size_t)z.ntau * g.n_ext},
      {(void **)&b.s1_ph, cs * g.nk * g.nk},
      {(void **)&b.s1_phc, cs * g.nk * g.nk},
      {(void **)&b.s1_gkt, cs * g.nk * (size_t)z.ntau},
      {(void **)&b.s1_grt, cs * g.nk * (size_t)z.ntau},
      {(void **)&b.s1_srn, cs * g.nk * g.n_ext},
      {(void **)&b.s1_tau, sizeof(double) * z.ntau},
      {(void **)&b.s2_bph, cs * g.nQ * (size_t)z.nj},
      {(void **)&b.s2_bpp, cs * g.nQ * (size_t)z.nj},
      {(void **)&b.s2_cph, cs * 2 * g.nQ * (size_t)n_nu},
      {(void **)&b.s2_cpp, cs * g.nQ * (size_t)n_nu},
      {(void **)&b.chi, cs * 4 * g.nQ},
      {(void **)&b.chi_part, cs * 4 * (size_t)b.q_chunk * g.n_om * ((g.n + 63) / 64)},
      {(void **)&b.gemm_work, cs * 64 * (size_t)g.nk * std::max(z.ntau, g.n_ext)},
  };
  b.gemm_work_elems = 64LL * g.nk * std::max(z.ntau, g.n_ext);
  // partial sums of chi per pass; also the bubble sums S_ph, S_pp of the truncated scheme
  b.chi_part_elems = std::max(4LL * b.q_chunk * g.n_om * ((g.n + 63) / 64), 2LL * g.nQ);
  size_t need = 0;
  for (auto &r : reqs) need += (r.bytes + 255) & ~(size_t)255;
  for (auto &r : reqs) {
    if (r.bytes == 0) continue;
    *r.p = dalloc(c, r.bytes);
    if (!*r.p) {
      release_all(c);
      delete c;
      return fail(nullptr, PQ_ENOMEM, "device allocation failed: the solve needs %zu bytes", need);
    }
  }

  // imaginary-time quadrature and transforms of Sigma~1
  std::vector<double> gx, gw;
  gauss_legendre(o.tau_order, gx, gw);
  std::vector<double> tau(z.ntau), wt(z.ntau);
  const double h = beta / o.tau_panels;
  for (int p = 0; p < o.tau_panels; ++p)
    for (int i = 0; i < o.tau_order; ++i) {
      tau[p * o.tau_order + i] = p * h + 0.5 * h * (gx[i] + 1.0);
      wt[p * o.tau_order + i] = 0.5 * h * gw[i];
    }
  // E (2M x N_tau complex exponentials) is built on the device from tau; the small tables here
  std::vector<std::complex<double>> Ef((size_t)z.ntau * g.n_ext);
  for (int j = 0; j < z.ntau; ++j)
    for (int e = 0; e < g.n_ext; ++e) {
      double nu = (2.0 * (g.e_lo + e) + 1.0) * M_PI / beta;
      Ef[(size_t)j * g.n_ext + e] = wt[j] * std::exp(std::complex<double>(0.0, nu * tau[j]));
    }
  std::vector<std::complex<double>> ph((size_t)g.nk * g.nk), phc((size_t)g.nk * g.nk);
  for (int r = 0; r < g.nk; ++r)
    for (int k = 0; k < g.nk; ++k) {
      double arg = 2.0 * M_PI * ((double)(r / L) * (k / L) + (double)(r % L) * (k % L)) / L;
      ph[(size_t)r * g.nk + k] = std::exp(std::complex<double>(0.0, arg)) / (double)g.nk;
      phc[(size_t)k * g.nk + r] = std::exp(std::complex<double>(0.0, -arg));
    }
  pq_status s = PQ_OK;
  auto up = [&](void *dst, const void *src, size_t bytes) {
    if (s == PQ_OK && cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
      s = fail(c, PQ_ECUDA, "upload failed: %s", cudaGetErrorString(cudaGetLastError()));
  };
  up(b.s1_Ef, Ef.data(), Ef.size() * cs);
  up(b.s1_ph, ph.data(), ph.size() * cs);
  up(b.s1_phc, phc.data(), phc.size() * cs);
  up(b.s1_tau, tau.data(), tau.size() * sizeof(double));
  if (s == PQ_OK && (pq::launch_e_table(0, (double2 *)b.s1_E, b.s1_tau, 2 * z.M, z.ntau, beta) != cudaSuccess ||
                     cudaStreamSynchronize(0) != cudaSuccess))
    s = fail(c, PQ_ECUDA, "transform table: %s", cudaGetErrorString(cudaGetLastError()));
  if (s == PQ_OK) {
    cudaError_t e1 = cudaMemset(b.phi, 0, vb);
    cudaError_t e2 = cudaMemset(b.sigma, 0, cs * g.nk * g.n_ext);
    cudaError_t e3 = cudaMemset(b.scal, 0, 8 * sizeof(double));
    cudaError_t e4 = b.fsc ? cudaMemset(b.fsc, 0, sizeof(float) * pq::FSC_N) : cudaSuccess;
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess)
      s = fail(c, PQ_ECUDA, "memset failed");
  }
  for (int i = 0; s == PQ_OK && i <= PQ_NSTEPS; ++i)
    if (cudaEventCreate(&c->ev[i]) != cudaSuccess) s = fail(c, PQ_ECUDA, "event create failed");
  if (s == PQ_OK && several && o.time_steps) {
    c->pev.assign(3 * (size_t)num_passes(c), nullptr);
    for (auto &e : c->pev)
      if (s == PQ_OK && cudaEventCreate(&e) != cudaSuccess) s = fail(c, PQ_ECUDA, "event create failed");
  }
  if (s == PQ_OK && pq::split_planes(b.vfmt)) {
    // problem table of the TMA-fed BSE: per pass, and per assignment of the Phi buffers
    CUtensorMap mA, mB;
    CUresult r = pq::make_bse_maps(b.gam, b.fv, g.n, b.ld, 4LL * b.q_chunk * g.n_om, b.vfmt == pq::V_F16P, &mA, &mB);
    if (r != CUDA_SUCCESS) s = fail(c, PQ_ECUDA, "tensor map encoding failed (CUresult %d)", (int)r);
    const int np = num_passes(c);
    std::vector<pq::BseProblem> tab(several ? 2 * np : 1);
    for (size_t i = 0; i < tab.size(); ++i) {
      const int ip = (int)(i % np), sw = (int)(i / np);
      const int nq = std::min(b.q_chunk, g.nk - ip * b.q_chunk);
      pq::BseProblem &e = tab[i];
      e.mapA = mA;
      e.mapB = mB;
      e.tile0 = 0;
      e.n = g.n;
      e.zc = nq * g.n_om;
      e.batch = 4 * e.zc;
      e.pad_ = 0;
      e.phi_cs = g.nQ;
      e.phi_q0 = (long long)ip * b.q_chunk * g.n_om;
      void *cur = sw ? b.phi_new : b.phi, *nxt = several ? (sw ? b.phi : b.phi_new) : b.phi;
      e.phi_in = (const float2 *)cur;
      e.phi_out = (float2 *)nxt;
      e.alpha = (float)g.mix;
      e.n_nu = g.n_nu;
      e.krow = b.krow;
      e.uns = b.vfmt == pq::V_F16P ? b.fsc + pq::FSC_UNS : nullptr;
      e.phimax = b.vfmt == pq::V_F16P ? (unsigned *)(b.fsc + pq::FSC_PHIMAX) : nullptr;
    }
    c->prob_host = tab[0];
    if (s == PQ_OK) {
      c->probs = (pq::BseProblem *)dalloc(c, tab.size() * sizeof(pq::BseProblem));
      if (!c->probs) s = fail(c, PQ_ENOMEM, "device allocation of the BSE problem table failed");
    }
    up(c->probs, tab.data(), tab.size() * sizeof(pq::BseProblem));
  }
  if (s != PQ_OK) {
    g_init_err = c->err;
    pq_destroy(c);
    return s;
  }
  *out = c;
  return PQ_OK;
}

pq_status pq_set_Lambda(pq_ctx *c, int channel, const double *host_c128, int n_lambda) {
  if (!c) return PQ_EINVAL;
  if (c->poisoned) return fail(c, PQ_ESTATE, "context poisoned");
  if (channel < 0 || channel > 3) return fail(c, PQ_EINVAL, "bad channel %d", channel);
  if (!host_c128) return fail(c, PQ_EINVAL, "the table is NULL");
  if (n_lambda < 1 || n_lambda > 1024) return fail(c, PQ_EINVAL, "n_lambda must be in [1, 1024]");
  const size_t cnt = (size_t)(2 * n_lambda + 1) * (2 * n_lambda) * (2 * n_lambda);
  const size_t es = c->c64 ? sizeof(float2) : sizeof(double2);
  void *d = dalloc(c, cnt * es);
  if (!d) return fail(c, PQ_ENOMEM, "device allocation of %zu bytes for the Lambda table failed", cnt * es);
  CK(cudaStreamSynchronize(c->st));
  if (c->c64) {
    std::vector<float2> tmp(cnt);
    for (size_t i = 0; i < cnt; ++i) tmp[i] = make_float2((float)host_c128[2 * i], (float)host_c128[2 * i + 1]);
    CK(cudaMemcpy(d, tmp.data(), cnt * es, cudaMemcpyHostToDevice));
  } else {
    CK(cudaMemcpy(d, host_c128, cnt * es, cudaMemcpyHostToDevice));
  }
  c->b.lam_tab[channel] = d;  // a previous table stays allocated until pq_destroy
  c->b.lam_nl[channel] = n_lambda;
  // bound of |Re|, |Im| of this channel's Lambda (table and constant), for the FP16 scales
  double lm = std::fabs(c->lam[2 * channel]);
  for (size_t i = 0; i < 2 * cnt; ++i) lm = std::max(lm, std::fabs(host_c128[i]));
  c->lam_max[channel] = lm;
  return PQ_OK;
}

pq_status pq_iterate(pq_ctx *c, int max_iter, double tol, int *iters_done, double *last) {
  if (!c) return PQ_EINVAL;
  if (c->poisoned) return fail(c, PQ_ESTATE, "context poisoned by an earlier error: %s", c->err.c_str());
  if (max_iter < 0) return fail(c, PQ_EINVAL, "max_iter < 0");
  if (c->in_batch) return fail(c, PQ_EINVAL, "the context belongs to a batch: iterate it with pq_batch_iterate");
  double d = INFINITY, prev = INFINITY, dref = 0.0;
  int it = 0, grown = 0;
  const int win = c->opt.diverge_window;
  for (; it < max_iter; ++it) {
    pq_status s = run_iteration(c, &d);
    if (s != PQ_OK) {
      if (iters_done) *iters_done = it;
      return s;
    }
    if (d < tol) {
      ++it;
      break;
    }
    grown = d > prev ? grown + 1 : 0;  // consecutive iterations whose max |dSigma| grew
    prev = d;
    if (it < win) dref = std::max(dref, d);  // the changes of the first win iterations of the call
    // diverging: grown win times in a row and 10x above the first changes of this call (a
    // damped iteration oscillates, rising for a while without running away)
    if (win > 0 && grown >= win && d > kDivergeFactor * dref) {
      if (iters_done) *iters_done = it + 1;
      if (last) *last = d;
      return fail(c, PQ_EDIVERGED, "max |dSigma| grew in each of the last %d iterations to %.3e (%.0fx its first values)",
                  win, d, d / dref);
    }
  }
  if (iters_done) *iters_done = it;
  if (last) *last = d;
  return (d < tol) ? PQ_OK : PQ_ENOTCONV;
}

pq_status pq_get_Sigma(const pq_ctx *cc, double *out, size_t len) {
  pq_ctx *c = const_cast<pq_ctx *>(cc);
  if (!c || !out) return PQ_EINVAL;
  if (c->poisoned) return fail(c, PQ_ESTATE, "context poisoned");
  size_t need = (size_t)2 * c->g.nk * c->g.n_ext;
  if (len < need) return fail(c, PQ_EINVAL, "Sigma needs %zu doubles, got %zu", need, len);
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemcpy(out, c->b.sigma, need * sizeof(double), cudaMemcpyDeviceToHost));
  return PQ_OK;
}

static pq_status get_phi_matrix(pq_ctx *c, int channel, int Q, double *out, size_t len) {
  if (!out || channel < 0 || channel > 3 || Q < 0 || Q >= c->g.nQ)
    return fail(c, PQ_EINVAL, "bad channel %d or Q %d", channel, Q);
  const size_t nn = (size_t)c->g.n * c->g.n;
  if (len < 2 * nn) return fail(c, PQ_EINVAL, "matrix needs %zu doubles, got %zu", 2 * nn, len);
  CK(cudaStreamSynchronize(c->st));
  const size_t off = ((size_t)channel * c->g.nQ + Q) * nn;
  if (!c->c64) {
    CK(cudaMemcpy(out, (const double2 *)c->b.phi + off, nn * sizeof(double2), cudaMemcpyDeviceToHost));
  } else {
    std::vector<float2> tmp(nn);
    CK(cudaMemcpy(tmp.data(), (const float2 *)c->b.phi + off, nn * sizeof(float2), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < nn; ++i) {
      out[2 * i] = tmp[i].x;
      out[2 * i + 1] = tmp[i].y;
    }
  }
  return PQ_OK;
}

pq_status pq_get_F(const pq_ctx *cc, int channel, int Q, double *out, size_t len) {
  pq_ctx *c = const_cast<pq_ctx *>(cc);
  if (!c) return PQ_EINVAL;
  if (c->poisoned) return fail(c, PQ_ESTATE, "context poisoned");
  if (c->iterations == 0) return fail(c, PQ_EINVAL, "no iteration has run yet");
  const Grid &g = c->g;
  const pq::Buffers &b = c->b;
  if (!out || channel < 0 || channel > 3 || Q < 0 || Q >= g.nQ)
    return fail(c, PQ_EINVAL, "bad channel %d or Q %d", channel, Q);
  const int nq = std::min(b.q_chunk, g.nk - c->last_qb);
  const int Ql = Q - c->last_qb * g.n_om;
  if (Ql < 0 || Ql >= nq * g.n_om)
    return fail(c, PQ_EINVAL, "F of Q %d is not kept: the last pass held q-momenta %d..%d", Q, c->last_qb,
                c->last_qb + nq - 1);
  const size_t n = g.n, ld = b.ld, nn = n * n;
  if (len < 2 * nn) return fail(c, PQ_EINVAL, "matrix needs %zu doubles, got %zu", 2 * nn, len);
  CK(cudaStreamSynchronize(c->st));
  const size_t slab = (size_t)channel * nq * g.n_om + Ql;
  if (b.vfmt == pq::V_C128) {
    CK(cudaMemcpy(out, (const double2 *)b.fv + slab * nn, nn * sizeof(double2), cudaMemcpyDeviceToHost));
  } else if (b.vfmt == pq::V_C64) {
    std::vector<float2> tmp(nn);
    CK(cudaMemcpy(tmp.data(), (const float2 *)b.fv + slab * nn, nn * sizeof(float2), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < nn; ++i) {
      out[2 * i] = tmp[i].x;
      out[2 * i + 1] = tmp[i].y;
    }
  } else if (b.vfmt == pq::V_F16P) {
    // four FP16 planes (Re h, Im h, Re l, Im l) of the scaled value: (h + l) / scale
    const size_t ps = (size_t)4 * b.q_chunk * g.n_om * n * ld;
    std::vector<uint16_t> tmp(4 * n * ld);
    for (int w = 0; w < 4; ++w)
      CK(cudaMemcpy(tmp.data() + w * n * ld, (const uint16_t *)b.fv + w * ps + slab * n * ld, n * ld * 2,
                    cudaMemcpyDeviceToHost));
    float sb = 1.f;
    CK(cudaMemcpy(&sb, b.fsc + pq::FSC_SB + channel, sizeof sb, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i)
      for (size_t j = 0; j < n; ++j) {
        const size_t e = i * ld + j;
        out[2 * (i * n + j)] = ((double)pq::f16_value(tmp[e]) + pq::f16_value(tmp[2 * n * ld + e])) / sb;
        out[2 * (i * n + j) + 1] = ((double)pq::f16_value(tmp[n * ld + e]) + pq::f16_value(tmp[3 * n * ld + e])) / sb;
      }
  } else {
    // six BF16 planes (Re h, Im h, Re l, Im l, Re r, Im r); element value = h + l + r
    const size_t ps = (size_t)4 * b.q_chunk * g.n_om * n * ld;  // plane stride of the buffer
    std::vector<uint16_t> tmp(6 * n * ld);
    for (int w = 0; w < 6; ++w)
      CK(cudaMemcpy(tmp.data() + w * n * ld, (const uint16_t *)b.fv + w * ps + slab * n * ld, n * ld * 2,
                    cudaMemcpyDeviceToHost));
    auto bf = [](uint16_t h) {
      uint32_t u = (uint32_t)h << 16;
      float f;
      std::memcpy(&f, &u, 4);
      return (double)f;
    };
    for (size_t i = 0; i < n; ++i)
      for (size_t j = 0; j < n; ++j) {
        const size_t e = i * ld + j;
        double re = 0.0, im = 0.0;
        for (int piece = 0; piece < 3; ++piece) {
          re += bf(tmp[(2 * piece) * n * ld + e]);
          im += bf(tmp[(2 * piece + 1) * n * ld + e]);
        }
        out[2 * (i * n + j)] = re;
        out[2 * (i * n + j) + 1] = im;
      }
  }
  return PQ_OK;
}

pq_status pq_get_Phi(const pq_ctx *cc, int channel, int Q, double *out, size_t len) {
  pq_ctx *c = const_cast<pq_ctx *>(cc);
  if (!c) return PQ_EINVAL;
  if (c->poisoned) return fail(c, PQ_ESTATE, "context poisoned");
  return get_phi_matrix(c, channel, Q, out, len);
}

pq_status pq_get_chi(const pq_ctx *cc, int channel, double *out, size_t len) {
  pq_ctx *c = const_cast<pq_ctx *>(cc);
  if (!c || !out) return PQ_EINVAL;
  if (c->poisoned) return fail(c, PQ_ESTATE, "context poisoned");
  if (channel < 0 || channel > 3) return fail(c, PQ_EINVAL, "bad channel %d", channel);
  if (c->iterations == 0) return fail(c, PQ_EINVAL, "no iteration has run yet");
  if (len < (size_t)2 * c->g.nQ) return fail(c, PQ_EINVAL, "chi needs %d doubles", 2 * c->g.nQ);
  if (!c->chi_ready) CK(pq::launch_chi(c->st, c->g, c->b, 0, c->g.nk));
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemcpy(out, c->b.chi + (size_t)channel * c->g.nQ, sizeof(double2) * c->g.nQ, cudaMemcpyDeviceToHost));
  return PQ_OK;
}

pq_status pq_sigma_second_order(pq_ctx *c, const double *sigma_c128, double *out, size_t len) {
  if (!c || !out) return PQ_EINVAL;
  if (c->poisoned) return fail(c, PQ_ESTATE, "context poisoned");
  const size_t need = (size_t)2 * c->g.nk * c->g.n_ext;
  if (len < need) return fail(c, PQ_EINVAL, "Sigma~1 needs %zu doubles, got %zu", need, len);
  pq::Buffers &b = c->b;
  const double2 *src = b.sigma;
  CK(cudaStreamSynchronize(c->st));
  if (sigma_c128) {
    // the last Sigma_new is informational only, so its buffer stages the input
    CK(cudaMemcpy(b.sigma_new, sigma_c128, need * sizeof(double), cudaMemcpyHostToDevice));
    src = b.sigma_new;
  }
  CK(pq::launch_tail_c1(c->st, c->g, src, b.scal + 3));
  CK(pq::launch_sigma1(c->st, c->g, c->z, pq::sigma1_args(b, src, b.scal + 3, b.sigma1)));
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemcpy(out, b.sigma1, need * sizeof(double), cudaMemcpyDeviceToHost));
  return PQ_OK;
}

pq_status pq_set_state(pq_ctx *c, const double *phi, const double *sigma) {
  if (!c) return PQ_EINVAL;
  if (c->poisoned) return fail(c, PQ_ESTATE, "context poisoned");
  if (phi) c->krow_ok = false;  // the row sums belong to the replaced Phi
  CK(cudaStreamSynchronize(c->st));
  if (sigma) CK(cudaMemcpy(c->b.sigma, sigma, sizeof(double2) * c->g.nk * c->g.n_ext, cudaMemcpyHostToDevice));
  if (phi) {
    const long long ne = 4LL * c->g.nQ * c->g.n * c->g.n;
    if (c->b.fsc) {
      // largest |Re|, |Im| per channel of the stored (complex64) Phi: the FP16 scales of the
      // next iteration derive from it
      float mx[4] = {0.f, 0.f, 0.f, 0.f};
      const long long per = ne / 4;
      for (long long i = 0; i < ne; ++i) {
        const float a = std::fabs((float)phi[2 * i]), b2 = std::fabs((float)phi[2 * i + 1]);
        float &m = mx[i / per];
        m = std::max(m, std::max(a, b2));
      }
      CK(cudaMemcpy(c->b.fsc + pq::FSC_PHIMAX, mx, sizeof mx, cudaMemcpyHostToDevice));
    }
    if (!c->c64) {
      CK(cudaMemcpy(c->b.phi, phi, ne * sizeof(double2), cudaMemcpyHostToDevice));
    } else {
      // stage through the F buffer, which the next iteration overwrites
      const long long chunk =
          (long long)b_fv_bytes(c) / (long long)sizeof(double2);
      for (long long o = 0; o < ne; o += chunk) {
        long long cnt = std::min(chunk, ne - o);
        CK(cudaMemcpy(c->b.fv, phi + 2 * o, cnt * sizeof(double2), cudaMemcpyHostToDevice));
        phi_from_c128<<<(unsigned)((cnt + 255) / 256), 256>>>((float2 *)c->b.phi + o, (const double2 *)c->b.fv,
                                                               cnt);
        CK(cudaGetLastError());
        CK(cudaDeviceSynchronize());
      }
    }
  }
  return PQ_OK;
}

pq_status pq_density(pq_ctx *c, double *n_out) {
  if (!c || !n_out) return PQ_EINVAL;
  if (c->poisoned) return fail(c, PQ_ESTATE, "context poisoned");
  if (c->g.lattice != PQ_SQUARE) return fail(c, PQ_EINVAL, "the density is defined for the square lattice");
  double dn = 0.0;
  return density_at(c, c->g.mu, n_out, &dn);
}

pq_status pq_get_mu(const pq_ctx *c, double *mu) {
  if (!c || !mu) return PQ_EINVAL;
  *mu = c->g.mu;
  return PQ_OK;
}

pq_status pq_get_sizes(const pq_ctx *c, long long *o) {
  if (!c || !o) return PQ_EINVAL;
  o[0] = c->g.nk;
  o[1] = c->g.n;
  o[2] = c->g.nQ;
  o[3] = c->g.n_ext;
  o[4] = c->g.n_nu;
  o[5] = c->g.n_om;
  o[6] = (long long)c->bytes;
  o[7] = c->c64 ? 8 : 16;
  return PQ_OK;
}

pq_status pq_step_times(const pq_ctx *c, float *out, int n) {
  if (!c || !out || n < PQ_NSTEPS) return PQ_EINVAL;
  for (int i = 0; i < PQ_NSTEPS; ++i) out[i] = c->times[i];
  return PQ_OK;
}

const char *pq_step_name(int i) { return (i >= 0 && i < PQ_NSTEPS) ? kStepNames[i] : ""; }

pq_status pq_selftest_wait_timeout(pq_ctx *c, int limit_ms) {
  if (!c) return PQ_EINVAL;
  if (c->poisoned) return fail(c, PQ_ESTATE, "context poisoned");
  if (limit_ms < 1 || limit_ms > 10000) return fail(c, PQ_EINVAL, "limit_ms must be in [1, 10000]");
  wait_selftest_kernel<<<1, 1, 0, c->st>>>((uint64_t)limit_ms * 1000000ull, (int *)(c->b.scal + 4));
  CK(cudaGetLastError());
  double h[5];
  CK(cudaMemcpyAsync(h, c->b.scal, sizeof h, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  double d = 0.0;
  return pq::finish_iteration(c, h, &d, false);
}

const char *pq_last_error(const pq_ctx *c) { return c ? c->err.c_str() : g_init_err.c_str(); }

void pq_destroy(pq_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  for (int i = 0; i <= PQ_NSTEPS; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  for (auto e : c->pev)
    if (e) cudaEventDestroy(e);
  release_all(c);
  delete c;
}

}  // extern "C"
