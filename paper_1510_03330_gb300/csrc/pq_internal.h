// Host-side launchers shared by the translation units of the solver.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "pq_common.cuh"

namespace pq {

// Device buffers of one solve.  Vertex arrays (phi, gam, fv) hold
// 4 * nQ * n * n elements of the storage type (double2 or float2).
struct Buffers {
  void *phi = nullptr;   // reducible vertices Phi_r(Q)[k][k'], the state
  void *gam = nullptr;   // BSE left operand s_r Gamma_r(Q) diag(X_r(Q))
  void *fv = nullptr;    // full vertex F_r(Q)
  double2 *sigma = nullptr;      // [nk][n_ext] state
  double2 *sigma_new = nullptr;  // [nk][n_ext] Sigma of this iteration
  double2 *sigma1 = nullptr;     // [nk][n_ext] Sigma~1
  double2 *sigma2 = nullptr;     // [nk][n_ext] Sigma~2
  double2 *gtab = nullptr;       // [nk][n_g] G on the table range
  double2 *xph = nullptr;        // [nQ][n] (T/N) G(k) G(k+q)
  double2 *xpp = nullptr;        // [nQ][n] (T/N) G(k) G(q-k)
  float2 *gtab32 = nullptr;      // FP32 copies of gtab, xph, xpp for the FP32 assembly of the split paths
  float2 *xph32 = nullptr;
  float2 *xpp32 = nullptr;
  double2 *k1 = nullptr;         // [4][nQ]
  double2 *k2row = nullptr;      // [4][n][nQ]  (row leg k major, transfer fastest)
  double2 *k2col = nullptr;      // [4][n][nQ]
  double2 *dfpart = nullptr;     // [n][nk] dF part of Sigma, one partial per (k, k'-momentum)
  double *scal = nullptr;        // [0] c1 of the Sigma tail, [1] max |dSigma| bits, [2] non-finite flag,
                                 // [3] c1 scratch of pq_sigma_second_order, [4] tensor-core wait timeout flag
  // Sigma~1 in imaginary time
  double2 *s1_R = nullptr;       // [nk][2M] Matsubara remainders
  double2 *s1_E = nullptr;       // [2M][ntau] exp(-i nu_n tau_j)
  double2 *s1_Ef = nullptr;      // [ntau][n_ext] w_j exp(i nu_n tau_j)
  double2 *s1_ph = nullptr;      // [nk][nk] exp(i k.r) / N   (rows r)
  double2 *s1_phc = nullptr;     // [nk][nk] exp(-i k.r)      (rows k)
  double2 *s1_gkt = nullptr;     // [nk][ntau]
  double2 *s1_grt = nullptr;     // [nk][ntau]
  double2 *s1_srn = nullptr;     // [nk][n_ext]
  double *s1_tau = nullptr;      // [ntau]
  // Sigma~2 tables
  double2 *s2_bph = nullptr;     // [nQ][nj] sum_j G(j) G(j+P)
  double2 *s2_bpp = nullptr;     // [nQ][nj] sum_j G(P-j) G(j)
  double2 *s2_cph = nullptr;     // [2][nQ][n_nu] C-weighted ph tables (d-m, m)
  double2 *s2_cpp = nullptr;     // [nQ][n_nu] C-weighted pp table (s+t)
  double2 *chi = nullptr;        // [4][nQ]
  double2 *chi_part = nullptr;   // partial sums of chi over row blocks, one pass of slices
  long long chi_part_elems = 0;
  double2 *gemm_work = nullptr;  // split-K partials of the Sigma~1 transforms
  long long gemm_work_elems = 0;
  // Storage of the BSE operands gam and fv:
  //   V_C128 / V_C64: [r][Q][k][ld] complex of the storage type;
  //   V_BF16P: BF16 planes [plane][r][Q][k][ld]; gam planes (Re h, Re l, Im h, Im l),
  //   fv planes (Re h, Im h, Re l, Im l, Re r, Im r) with x = h + l + r;
  //   V_F16P: FP16 planes of the same order, gam (Re h, Re l, Im h, Im l), fv (Re h, Im h,
  //   Re l, Im l), with x * 2^e = h + l (no third piece).
  const void *lam_tab[4] = {};  // tabulated local Lambda per channel (arithmetic type of the assembly)
  int lam_nl[4] = {};
  double2 *krow = nullptr;       // split planes: edge row sums of Phi accumulated by the BSE epilogue
  // FP16 planes: power-of-two scales of the split operands, [0..3] max |Re|, |Im| of the state's
  // Phi per channel (float bits, accumulated by the products that write it), [4..5] the same of
  // X_ph, X_pp (accumulated by the bubbles), [8..11] scale of Gamma X, [12..15] scale of F,
  // [16..19] 1 / (scale of Gamma X * scale of F), per channel
  float *fsc = nullptr;
  int vfmt = 0;
  int assembly = 0;              // BF16x3 assembly kernel: 0 tiled where the shape allows, 1 general
  bool first_level = false;      // kernel approximation of the fill: K1 only (else K1 + K2)
  bool lower_edge = false;       // K2 from the lower frequency edge alone (else the mean of both edges)
  bool truncated = false;        // Sigma from Eq. PA_Sigma on the box alone (else the regulated Sigma)
  int ld = 0;                    // row stride of gam and fv (elements)
  int q_chunk = 0;               // q-momenta assembled and multiplied per pass
  void *phi_new = nullptr;       // Jacobi target when the transfers run in several passes
};

// V_BF16P: BF16 planes, x = h + l (+ r for F); V_F16P: FP16 planes of the scaled value,
// x * 2^e = h + l, with the power-of-two scale 2^e of the channel in Buffers::fsc.
enum VFmt { V_C128 = 0, V_C64 = 1, V_BF16P = 2, V_F16P = 3 };
inline bool split_planes(int vfmt) { return vfmt == V_BF16P || vfmt == V_F16P; }
enum { FSC_PHIMAX = 0, FSC_XMAX = 4, FSC_SA = 8, FSC_SB = 12, FSC_UNS = 16, FSC_N = 32 };

// One pass of the assembly and the BSE over the transfers Q = (q, m) with
// q-momentum in [qb, qb + nq): the operand buffers hold 4 * nq * NOmega slices.
struct Pass {
  int qb, nq;
  bool fused;       // nq == nk: d/m and s/t outputs of one gather step written together
  bool accumulate;  // add to the dF part of Sigma instead of overwriting it
};

// Pointers of one Sigma~1 evaluation (the context's buffers, or a caller's scratch).
struct Sigma1Args {
  const double2 *sigma;  // [nk][n_ext] input self-energy
  double *c1;            // device scalar: c1 of its 1/(i nu) tail (written)
  double2 *out;          // [nk][n_ext] Sigma~1
  double2 *R, *gkt, *grt, *srn;
  const double2 *E, *Ef, *ph, *phc;
  const double *tau;
  double2 *work;
  long long work_elems;
};

struct Sizes {
  int ntau, M;  // tau nodes, Matsubara cut of G(tau)
  int j_lo, nj; // frequency range of the Sigma~2 bubble tables
};

int zgemm_splits(int M, int N, int K, long long work_elems);
cudaError_t zgemm_fp64_splitk(cudaStream_t st, int M, int N, int K, double2 alpha, const double2 *A, int lda,
                              const double2 *B, int ldb, double2 beta, double2 *C, int ldc, double2 *work,
                              long long work_elems);
cudaError_t zgemm_fp64(cudaStream_t st, int M, int N, int K, double2 alpha, const double2 *A, int lda, long long sA,
                       const double2 *B, int ldb, long long sB, double2 beta, double2 *C, int ldc, long long sC,
                       int batch);

// one-particle steps (pq_onebody.cu)
cudaError_t launch_tail_and_green(cudaStream_t st, const Grid &g, Buffers &b);
cudaError_t launch_bubbles(cudaStream_t st, const Grid &g, Buffers &b);
// FP16 planes: the power-of-two scales of this iteration's operands from the state's vertex
// bound and the bubbles' bound (lam_max: max |Re|, |Im| of Lambda per channel); resets the
// bounds that the bubbles and the products accumulate for the next iteration
cudaError_t launch_split_scales(cudaStream_t st, Buffers &b, const double *lam_max);
cudaError_t launch_sigma1(cudaStream_t st, const Grid &g, const Sizes &z, const Sigma1Args &a);
Sigma1Args sigma1_args(Buffers &b, const double2 *sigma, double *c1, double2 *out);
cudaError_t launch_tail_c1(cudaStream_t st, const Grid &g, const double2 *sigma, double *c1);
// E[a][j] = exp(-i nu_a tau[j]) for the 2M fermionic frequencies nu_a = (2 (a - M) + 1) pi / beta
cudaError_t launch_e_table(cudaStream_t st, double2 *E, const double *tau, int two_m, int ntau, double beta);
// density per site and d density / d mu of G[sigma] at g.mu (square lattice), Matsubara cut M,
// written to out2[0..1] (zeroed first); c1: device scalar of sigma's 1/(i nu) tail
cudaError_t launch_density(cudaStream_t st, const Grid &g, int M, const double2 *sigma, const double *c1,
                           double *out2);
cudaError_t launch_sigma_update(cudaStream_t st, const Grid &g, Buffers &b);
// chi of the slices in the operand buffers (q-momenta [qb, qb + nq))
cudaError_t launch_chi(cudaStream_t st, const Grid &g, Buffers &b, int qb, int nq);

// vertex steps (pq_vertex.cu)
// K1/K2 from the state; with rowsums, K2row from the edge row sums the last BSE accumulated
cudaError_t launch_kernels_extract(cudaStream_t st, const Grid &g, Buffers &b, bool c64, bool rowsums = false);
// truncated scheme: Sigma~1 <- 0, Sigma~2 <- the Lambda^0 part of the box sum (pq_onebody.cu)
cudaError_t launch_sigma_truncated(cudaStream_t st, const Grid &g, Buffers &b);
cudaError_t launch_assemble(cudaStream_t st, const Grid &g, Buffers &b, const double *lam4, const Pass &p);
struct Lam;
// tiled BF16 assembly (pq_assemble_tiled.cu): false / cudaErrorInvalidValue where the shape
// is not served (Nnu % 4 != 0)
bool assemble_tiled_ok(const Grid &g);
cudaError_t launch_assemble_tiled(cudaStream_t st, const Grid &g, Buffers &b, const Lam &lam, const Pass &p,
                                  long long ps, bool tab);
size_t assemble_smem_bytes(const Grid &g, bool c64);

// TF32x3 BSE on the tensor cores from complex64 operands (pq_gemm_tc.cu)
size_t bse_tc_smem_bytes();
cudaError_t launch_bse_split(cudaStream_t st, int n, int batch, const float2 *A, const float2 *B, float2 *Phi,
                             float alpha, int *err);

// BF16x3 BSE from pre-split planes, fed by TMA (pq_bse_tma.cu).  One launch covers the tiles of
// one or more problems (a context's pass, or the solves of a batch), described by a device table.
// GEMM z of a problem reads operand slice z and updates Phi slice
// (z / zc) * phi_cs + phi_q0 + z % zc.
struct BseProblem {
  CUtensorMap mapA;   // Gamma X planes [plane][slice][row][ld]
  CUtensorMap mapB;   // F planes
  long long tile0;    // first tile of this problem within the launch
  int n, batch, zc, pad_;
  long long phi_cs, phi_q0;
  const float2 *phi_in;
  float2 *phi_out;
  float alpha;
  int n_nu;           // fermionic frequencies per momentum block (edge test of the row sums)
  double2 *krow;      // if set: [r][k][Q] += sum of the new Phi row k over the k' frequency edges
  const float *uns;   // if set (FP16 planes): the product of channel r is multiplied by uns[r]
  unsigned *phimax;   // if set: [r] = max of the bits of |Re|, |Im| over the new Phi of channel r
};
size_t bse_tma_smem_bytes(int bnc);
long long bse_tiles(int bnc, int n, int batch);
// f16: FP16 planes (four F planes), else BF16 planes (six F planes)
CUresult make_bse_maps(void *gam_planes, void *fv_planes, int n, int ld, long long slabs, bool f16,
                       CUtensorMap *mapA, CUtensorMap *mapB);
// Tensor map of complex64 Phi [slabs][n][n] as 8-byte words (x = k', y = k, z = slab), boxes of
// box_w x 1 x box_h: the parquet assembly's gathers of a column block over box_h transfers.
CUresult make_phi_rows_map(const void *phi, int n, long long slabs, int box_w, int box_h, CUtensorMap *map);
// bnc: complex output columns per tile (128 or 64); f16: FP16 operand planes, else BF16;
// max_ctas > 0 caps the persistent grid
cudaError_t launch_bse_tma(cudaStream_t st, int bnc, bool f16, const BseProblem *probs, int nprob, long long tiles,
                           int *err, int max_ctas);

// Sigma~2 (pq_sigma2.cu)
cudaError_t launch_sigma2(cudaStream_t st, const Grid &g, const Sizes &z, Buffers &b);

}  // namespace pq
