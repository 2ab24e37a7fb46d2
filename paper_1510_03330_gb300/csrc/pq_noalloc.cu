// Second-order self-energy without any device allocation.
//
// Some callers cannot allocate device memory: code that runs while another
// component owns the allocator (a host application that reserves all device
// memory up front, or a plug-in called from inside someone else's solver
// loop), and code that must not block on cudaMalloc's implicit device
// synchronisation.  pq_sigma_second_order_noalloc serves them: it computes
// the same quantity as pq_sigma_second_order, Sigma~1 of G[Sigma], from a
// caller's device input into a caller's device output, and keeps every
// intermediate (the imaginary-time tables and transforms, the split-K
// partials of its products) in one file-scope static device array of fixed
// size.  Each GPU that loads the library holds that array until the process
// exits.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/parquet.h"
#include "pq_common.cuh"
#include "pq_internal.h"

namespace pq {
void set_context_free_error(const char *msg);
}

namespace {

// Limits of the static scratch (double2 elements of each region).
constexpr int kMaxNk = 16;     // momenta: L <= 4
constexpr int kMax2M = 512;    // Matsubara sums of G(tau): 2 * tau_matsubara
constexpr int kMaxTau = 512;   // tau nodes: tau_panels * tau_order
constexpr int kMaxExt = 128;   // extended fermionic range: n_Omega + n_nu - 1
constexpr int kMaxOrder = 32;  // nodes per Gauss-Legendre panel
constexpr long long kWorkElems = 8LL * kMaxNk * kMaxTau;  // split-K partials

constexpr long long kOffE = 0;
constexpr long long kOffEf = kOffE + (long long)kMax2M * kMaxTau;
constexpr long long kOffR = kOffEf + (long long)kMaxTau * kMaxExt;
constexpr long long kOffGkt = kOffR + (long long)kMaxNk * kMax2M;
constexpr long long kOffGrt = kOffGkt + (long long)kMaxNk * kMaxTau;
constexpr long long kOffSrn = kOffGrt + (long long)kMaxNk * kMaxTau;
constexpr long long kOffPh = kOffSrn + (long long)kMaxNk * kMaxExt;
constexpr long long kOffPhc = kOffPh + (long long)kMaxNk * kMaxNk;
constexpr long long kOffWork = kOffPhc + (long long)kMaxNk * kMaxNk;
constexpr long long kOffTau = kOffWork + kWorkElems;     // kMaxTau doubles
constexpr long long kOffC1 = kOffTau + kMaxTau / 2;      // one double
constexpr long long kElems = ((kOffC1 + 1 + 15) / 16) * 16;  // 420,624 elements = 6.73 MB

// The scratch.  In host code this name is only a stand-in for the device
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double2 g_sigma1_scratch[kElems];

struct DeviceSetup {
  bool ready = false;
  double2 *base = nullptr;
};
DeviceSetup g_setup[64];
std::mutex g_setup_mu;

struct TableArgs {
  int nk, L, two_m, ntau, n_ext, e_lo, panels, order;
  double beta;
  double x[kMaxOrder], w[kMaxOrder];
};

// Imaginary-time quadrature and transform tables, written on the device:
// tau_j, E[n][j] = exp(-i nu_n tau_j), Ef[j][e] = w_j exp(i nu_e tau_j),
// ph[r][k] = exp(i k.r)/N, phc[k][r] = exp(-i k.r).
__global__ void tables_kernel(TableArgs t, double2 *E, double2 *Ef, double2 *ph, double2 *phc, double *tau) {
  const long long nE = (long long)t.two_m * t.ntau, nEf = (long long)t.ntau * t.n_ext, nP = (long long)t.nk * t.nk;
  const long long total = nE + nEf + nP;
  const double h = t.beta / t.panels;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    if (i < nE) {
      int a = (int)(i / t.ntau), j = (int)(i % t.ntau);
      int p = j / t.order, q = j % t.order;
      double tj = p * h + 0.5 * h * (t.x[q] + 1.0);
      double nu = (2.0 * (a - t.two_m / 2) + 1.0) * CUDART_PI / t.beta;
      double s, c;
      sincos(-nu * tj, &s, &c);
      E[i] = make_double2(c, s);
      if (a == 0) tau[j] = tj;
    } else if (i < nE + nEf) {
      long long k = i - nE;
      int j = (int)(k / t.n_ext), e = (int)(k % t.n_ext);
      int p = j / t.order, q = j % t.order;
      double tj = p * h + 0.5 * h * (t.x[q] + 1.0);
      double wj = 0.5 * h * t.w[q];
      double nu = (2.0 * (t.e_lo + e) + 1.0) * CUDART_PI / t.beta;
      double s, c;
      sincos(nu * tj, &s, &c);
      Ef[k] = make_double2(wj * c, wj * s);
    } else {
      long long k = i - nE - nEf;
      int r = (int)(k / t.nk), kk = (int)(k % t.nk);
      double arg = 2.0 * CUDART_PI * ((double)(r / t.L) * (kk / t.L) + (double)(r % t.L) * (kk % t.L)) / t.L;
      double s, c;
      sincos(arg, &s, &c);
      ph[(long long)r * t.nk + kk] = make_double2(c / t.nk, s / t.nk);
      phc[(long long)kk * t.nk + r] = make_double2(c, -s);
    }
  }
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_p).
void gauss_legendre_fixed(int p, double *x, double *w) {
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
      dp = p * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    x[p - 1 - i] = z;
    w[p - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

pq_status err(pq_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  pq::set_context_free_error(buf);
  return s;
}

}  // namespace

extern "C" pq_status pq_sigma_second_order_noalloc(int lattice, double beta, double U, double mu, double hop, int L,
                                                   int n_nu, int n_Omega, int tau_panels, int tau_order,
                                                   int tau_matsubara, const double *sigma_dev, double *out_dev,
                                                   void *cuda_stream) {
  if (lattice != PQ_BETHE && lattice != PQ_SQUARE) return err(PQ_EINVAL, "unknown lattice %d", lattice);
  if (!(beta > 0.0) || !std::isfinite(beta)) return err(PQ_EINVAL, "beta must be positive");
  if (L < 1 || (lattice == PQ_BETHE && L != 1)) return err(PQ_EINVAL, "L must be >= 1 (1 for Bethe)");
  if (n_nu < 2 || n_nu % 2 || n_Omega < 1) return err(PQ_EINVAL, "n_nu must be even >= 2 and n_Omega >= 1");
  if (tau_panels < 1 || tau_order < 2 || tau_matsubara < 1) return err(PQ_EINVAL, "bad quadrature sizes");
  if (!sigma_dev || !out_dev) return err(PQ_EINVAL, "sigma_dev and out_dev must be device pointers");
  const int nk = L * L, n_ext = n_Omega + n_nu - 1, ntau = tau_panels * tau_order, two_m = 2 * tau_matsubara;
  if (nk > kMaxNk || two_m > kMax2M || ntau > kMaxTau || n_ext > kMaxExt || tau_order > kMaxOrder)
    return err(PQ_EINVAL,
               "size beyond the static scratch: need L*L <= %d (got %d), 2*tau_matsubara <= %d (got %d), "
               "tau_panels*tau_order <= %d (got %d), n_Omega+n_nu-1 <= %d (got %d), tau_order <= %d (got %d)",
               kMaxNk, nk, kMax2M, two_m, kMaxTau, ntau, kMaxExt, n_ext, kMaxOrder, tau_order);

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return err(PQ_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return err(PQ_EINVAL, "device index %d beyond 64", dev);
  double2 *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_setup[dev].ready) {
      // once per device, with that device current
      e = cudaGetSymbolAddress((void **)&g_setup[dev].base, g_sigma1_scratch);
      if (e != cudaSuccess) return err(PQ_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      g_setup[dev].ready = true;
    }
    base = g_setup[dev].base;
  }

  pq::Grid g{};
  g.lattice = lattice;
  g.L = L;
  g.nk = nk;
  g.n_nu = n_nu;
  g.n_om = n_Omega;
  g.n = nk * n_nu;
  g.nQ = nk * n_Omega;
  g.n_ext = n_ext;
  g.n_lo = -n_nu / 2;
  g.n_hi = n_nu / 2 - 1;
  g.m_lo = -(n_Omega / 2);
  g.m_hi = g.m_lo + n_Omega - 1;
  g.e_lo = g.m_lo + g.n_lo;
  g.e_hi = g.m_hi + g.n_hi;
  g.beta = beta;
  g.T = 1.0 / beta;
  g.U = U;
  g.mu = mu;
  g.hop = hop;
  pq::Sizes z{};
  z.M = tau_matsubara;
  z.ntau = ntau;

  TableArgs t{};
  t.nk = nk;
  t.L = L;
  t.two_m = two_m;
  t.ntau = ntau;
  t.n_ext = n_ext;
  t.e_lo = g.e_lo;
  t.panels = tau_panels;
  t.order = tau_order;
  t.beta = beta;
  gauss_legendre_fixed(tau_order, t.x, t.w);

  cudaStream_t st = (cudaStream_t)cuda_stream;
  pq::Sigma1Args a{};
  a.sigma = (const double2 *)sigma_dev;
  a.out = (double2 *)out_dev;
  a.c1 = (double *)(base + kOffC1);
  a.R = base + kOffR;
  a.gkt = base + kOffGkt;
  a.grt = base + kOffGrt;
  a.srn = base + kOffSrn;
  a.E = base + kOffE;
  a.Ef = base + kOffEf;
  a.ph = base + kOffPh;
  a.phc = base + kOffPhc;
  a.tau = (const double *)(base + kOffTau);
  a.work = base + kOffWork;
  a.work_elems = kWorkElems;

  // every scratch element this call reads is written earlier in the same call
  tables_kernel<<<256, 256, 0, st>>>(t, base + kOffE, base + kOffEf, base + kOffPh, base + kOffPhc,
                                     (double *)(base + kOffTau));
  e = cudaGetLastError();
  if (e != cudaSuccess) return err(PQ_ECUDA, "tables: %s", cudaGetErrorString(e));
  e = pq::launch_tail_c1(st, g, a.sigma, a.c1);
  if (e != cudaSuccess) return err(PQ_ECUDA, "tail: %s", cudaGetErrorString(e));
  e = pq::launch_sigma1(st, g, z, a);
  if (e != cudaSuccess) return err(PQ_ECUDA, "sigma1: %s", cudaGetErrorString(e));
  return PQ_OK;
}
