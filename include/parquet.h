/*
 * parquet.h -- C ABI of the GB300 parquet solver.
 *
 * One context holds one parquet solve of the single-band Hubbard model
 * (Li, Wentzell, Pudleiner, Thunstroem, Held, arXiv:1510.03330) on one GPU:
 * the reducible vertices Phi_r (r = d, m, s, t) on the frequency box, the
 * self-energy Sigma on the extended fermionic range, and the scratch of one
 * iteration.  pq_iterate runs the paper's self-consistent loop (Sec. II):
 * Dyson equation (App. A, Eq. PA_Dyson), bubbles, kernel functions K1/K2
 * (Sec. II.A), parquet equations with the kernel fill (Eq. PA_F, App. A Eqs.
 * PA_Gamma_dm, PA_Gamma_st), the Bethe-Salpeter equations (Eq. PA_F_Phi),
 * the high-frequency regulated Schwinger-Dyson self-energy (Sec. II.B,
 * Eq. PA_Sigma) and linear mixing.
 *
 * Conventions shared by every call:
 *   - complex numbers are (re, im) pairs of doubles, "c128" below;
 *   - k = (k-vector, n) with n fastest: index ik*Nnu + (n - n_lo),
 *     n_lo = -Nnu/2; Q = (q-vector, m): index iq*NOmega + (m - m_lo),
 *     m_lo = -floor(NOmega/2); ik = ix*L + iy for k = 2 pi (ix, iy)/L;
 *   - Sigma is stored on the extended range e in [m_lo+n_lo, m_hi+n_hi]
 *     (NOmega+Nnu-1 frequencies), index ik*n_ext + (e - e_lo);
 *   - every host buffer is owned by the caller; the library copies from or
 *     into it before returning and keeps no pointer to it;
 *   - device memory is owned by the context: allocated in pq_init (through
 *     the caller's allocator if one is given) and released in pq_destroy;
 *   - no call throws; each returns a pq_status and pq_last_error() gives the
 *     message of the last failure on that context;
 *   - one context is used from one host thread at a time; its kernels run
 *     on the stream given in pq_options (the legacy default stream if NULL).
 */
#ifndef PARQUET_GB300_H
#define PARQUET_GB300_H

#include <stddef.h>

#if defined(__GNUC__)
#define PQ_API __attribute__((visibility("default")))
#else
#define PQ_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pq_ctx pq_ctx;

typedef enum {
  PQ_OK = 0,
  PQ_EINVAL = 1,   /* bad argument or size; nothing changed */
  PQ_ENOMEM = 2,   /* device allocation failed; the message gives the bytes */
  PQ_ECUDA = 3,    /* a CUDA call failed; the context is poisoned */
  PQ_ENOTCONV = 4, /* pq_iterate reached max_iter above tol (state is valid) */
  PQ_ETIMEOUT = 5, /* a bounded device wait gave up; the context is poisoned */
  PQ_ENAN = 6,     /* a non-finite Sigma appeared; the context is poisoned */
  PQ_ESTATE = 7,   /* the context is poisoned by an earlier PQ_ECUDA/PQ_ENAN/PQ_ETIMEOUT */
  PQ_EDIVERGED = 8 /* pq_iterate stopped on divergence (pq_options.diverge_window); the state is valid */
} pq_status;

typedef enum { PQ_BETHE = 0, PQ_SQUARE = 1 } pq_lattice;

/* Arithmetic of the vertex storage and the BSE products.
 * PQ_FP64: complex128 vertices, FP64 everywhere.
 * PQ_SPLIT_*: complex64 Phi, parquet assembly in FP32; the BSE runs on the
 * tensor cores as a split-operand product with FP32 accumulation; Dyson, the
 * bubbles, Sigma~1 and Sigma~2 stay FP64.  The parts of Sigma and K1/K2 that
 * read the FP32 vertex are sums of FP32 products kept as compensated FP32
 * (two-sum) accumulators and reduced in FP64: the dF box sum of Eq. PA_Sigma
 * (per assembly thread, one FP32 partial per gather step added into the
 * compensated sum) and the edge sums of K1/K2 (Sec. II.A).
 *   PQ_SPLIT_TF32X3: complex64 operands split into TF32 hi/lo inside the GEMM
 *     (~2^-22 per product);
 *   PQ_SPLIT_BF16X3: the assembly writes the operands as BF16 planes (hi/lo;
 *     F also keeps a third piece), the GEMM reads them by TMA with no
 *     conversion (~2^-16 per product);
 *   PQ_SPLIT_FP16X3: the same with FP16 planes of each channel's operands
 *     scaled by a power of two (chosen every iteration from bounds of the
 *     vertex and the bubbles, so every piece lies in the FP16 range): 11-bit
 *     pieces, ~2^-22 per product at the cost of BF16x3;
 *   both plane formats accumulate the products in chunks of 512 k that are summed
 *   in FP32 registers, so the accumulation error does not grow with n;
 *   PQ_SPLIT_BF16X6 is rejected by pq_init with PQ_EINVAL. */
typedef enum {
  PQ_FP64 = 0,
  PQ_SPLIT_TF32X3 = 1,
  PQ_SPLIT_BF16X3 = 2,
  PQ_SPLIT_BF16X6 = 3,
  PQ_SPLIT_FP16X3 = 4
} pq_precision;

typedef struct {
  int precision;          /* pq_precision; default PQ_FP64 */
  double mix_alpha;       /* weight of the new iterate in linear mixing; default 0.5 */
  int sigma2_box_factor;  /* kernel-term box / vertex box (Sec. II.B); default 3 */
  double hop;             /* t (square) or half-bandwidth D (Bethe); default 1 */
  int tau_panels;         /* Gauss-Legendre panels on [0, beta] for Sigma~1; default 64 */
  int tau_order;          /* nodes per panel; default 16 */
  int tau_matsubara;      /* Matsubara cut M of G(tau): n in [-M, M-1]; default 2048 */
  int time_steps;         /* nonzero: record per-step CUDA-event times (pq_step_times) */
  /* q-momenta whose transfer slices are assembled and multiplied per pass.
   * 0 (default): all of them when the operand buffers of the whole box fit in
   * free device memory, else the largest count that fits next to two copies
   * of Phi.  With fewer than L*L per pass, Gamma and F are rebuilt pass by
   * pass (the operand buffers hold 4*q_chunk*NOmega slices), Phi is double
   * buffered for the Jacobi update, chi is computed during the iteration, and
   * pq_get_F serves only the transfers of the last pass. */
  int q_chunk;
  /* Kernel of the parquet assembly on the BF16x3 path: 0 (default) the tiled kernel,
   * which writes the operand rows in long contiguous runs, wherever Nnu % 4 == 0; 1 the
   * general kernel.  Both write the same operands; the dF part of Sigma is summed in
   * another order. */
  int assembly;
  /* Kernel approximation of the fill and of F~ (Sec. II.A): 0 or 2 (default) second
   * level, K1 + K2; 1 first level, K1 only. */
  int kernel_level;
  /* Frequency edge the second-level kernels are read at: 0 (default) the mean of the
   * lower and upper edges of the box; 1 the lower edge alone (the paper's example of
   * one edge), with K1 at the lower corner. */
  int edge_rule;
  /* Self-energy: 0 (default) the regulated Schwinger-Dyson equation (Sec. II.B:
   * Sigma~1 + Sigma~2 + the box sum of F - F~); 1 Eq. PA_Sigma summed on the vertex box
   * with the vertex cut off at its boundary (zero outside the box), for comparison. */
  int sde;
  /* Complex output columns per tile of the tensor-core products of the plane formats
   * (BF16x3, FP16x3): 0 (default) or 128, or 64 (narrower tiles, more operand traffic per
   * flop: slower on large matrices). */
  int bse_tile_cols;
  /* Divergence detection in pq_iterate: when max |dSigma| has grown in each of the last
   * diverge_window iterations and is more than 10 times the largest max |dSigma| of the
   * first diverge_window iterations of the call (a damped iteration oscillates, rising for
   * a while without running away), stop with
   * PQ_EDIVERGED (the iteration that diverges is kept: the state is valid, e.g. for a
   * restart with stronger mixing).  0 (default): off. */
  int diverge_window;
  /* Filling: 0 (default) keeps mu fixed; a value in (0, 2) (square lattice) is the number of
   * electrons per site (both spins) to hold: every iteration first sets mu, by a Newton search
   * on the FP64 density of the state's G (pq_density), then runs at that mu (pq_get_mu). */
  double target_density;
  void *cuda_stream;      /* cudaStream_t for all work; NULL = legacy default stream */
  /* Optional device allocator: returns 256-byte aligned device memory or NULL.
   * When NULL, cudaMalloc/cudaFree are used. */
  void *(*dev_alloc)(size_t bytes, void *alloc_ctx);
  void (*dev_free)(void *ptr, size_t bytes, void *alloc_ctx);
  void *alloc_ctx;
} pq_options;

/* Fill *opt with the defaults listed above. */
PQ_API void pq_default_options(pq_options *opt);

/* Create a solve.  lattice: pq_lattice; beta > 0; L >= 1 (L = 1 for Bethe);
 * n_nu even >= 2; n_Omega >= 1.  Allocates all device memory (PQ_ENOMEM with
 * the byte count if it does not fit) and sets Phi = 0, Sigma = 0 and
 * Lambda = (U, -U, 2U, 0), the parquet approximation (Sec. II.A).
 * opt may be NULL for the defaults.  On success *out owns the context. */
PQ_API pq_status pq_init(pq_ctx **out, int lattice, double beta, double U, double mu, int L,
                  int n_nu, int n_Omega, const pq_options *opt);

/* Fully irreducible vertex of one channel (0..3 = d, m, s, t), local in
 * momentum (Sec. III.A: Lambda from an impurity calculation on a small frequency
 * box, the full-parquet / parquet-DGammaA input), tabulated as host c128
 * [2 n_lambda + 1 (m)][2 n_lambda (n)][2 n_lambda (n')] with n, n' in
 * [-n_lambda, n_lambda - 1] and m in [-n_lambda, n_lambda], in the channel's own
 * frequency convention (that of F_r^{k k'}(Q)).  Outside the table, and for
 * channels never set, the parquet-approximation value (U, -U, 2U, 0) is used.
 * Applies from the next pq_iterate on.  The table is copied to the device (converted to
 * the storage precision); a later call for the same channel replaces it (the old copy
 * is freed with the context).  Errors: PQ_EINVAL (channel, NULL table, n_lambda
 * outside [1, 1024]), PQ_ENOMEM, PQ_ECUDA. */
PQ_API pq_status pq_set_Lambda(pq_ctx *ctx, int channel, const double *host_c128, int n_lambda);

/* Run up to max_iter iterations; stop after the first one whose
 * max_k |Sigma_new(k) - Sigma(k)| < tol.  Writes the count done and the last
 * max |dSigma| when the pointers are non-NULL.  PQ_ENOTCONV if tol was not
 * reached (the state is still valid); PQ_EDIVERGED if divergence detection
 * (pq_options.diverge_window) stopped it.  One device->host read of a few
 * scalars per iteration. */
PQ_API pq_status pq_iterate(pq_ctx *ctx, int max_iter, double tol, int *iters_done,
                     double *last_max_dsigma);

/* Self-energy of the current state (the mixed Sigma of the regulated
 * Schwinger-Dyson equation, Sec. II.B and App. A Eq. PA_Sigma, that enters the
 * Dyson equation Eq. PA_Dyson of the next iteration), host c128 [L*L][n_ext];
 * len = number of doubles available in out (>= 2*L*L*n_ext). */
PQ_API pq_status pq_get_Sigma(const pq_ctx *ctx, double *out, size_t len);

/* Full vertex F_r(Q) = Gamma_r(Q) + Phi_r(Q) of the last iteration (Eq. PA_F with
 * the parquet equations App. A Eqs. PA_Gamma_dm, PA_Gamma_st, assembled from the
 * state that iteration started from; the right factor of its Bethe-Salpeter
 * equation, Eq. PA_F_Phi), host c128 [n][n], n = L*L*Nnu.  The split paths
 * return the operand they multiplied (FP16x3: (h + l) / 2^e, to 2^-22). */
PQ_API pq_status pq_get_F(const pq_ctx *ctx, int channel, int Q, double *out, size_t len);

/* Reducible vertex Phi_r(Q) of the current state, host c128 [n][n]. */
PQ_API pq_status pq_get_Phi(const pq_ctx *ctx, int channel, int Q, double *out, size_t len);

/* Susceptibility of the last iteration, host c128 [N_Q]:
 * chi_r(Q) = -sum_k X_r(Q,k) - sum_{k,k'} X_r(Q,k) F_r^{k,k'}(Q) X_r(Q,k'),
 * X_ph = (T/N) G(k)G(k+q) for d, m and X_pp = (T/N) G(k)G(q-k) for s, t
 * (App. A, "Notations": chi from F and the bare bubble). */
PQ_API pq_status pq_get_chi(const pq_ctx *ctx, int channel, double *out, size_t len);

/* Second-order self-energy Sigma~1 = -U^2 FFT^-1[G^2(r) G(-r)] (Sec. II.B:
 * the self-energy of the second-order diagram, summed over all frequencies
 * in imaginary time) of G = [G0^-1 - Sigma]^-1 for the given Sigma, host c128
 * [L*L][n_ext] (NULL = the current state), written to out, host c128
 * [L*L][n_ext] (len = doubles available).  The state is not changed. */
PQ_API pq_status pq_sigma_second_order(pq_ctx *ctx, const double *sigma_c128, double *out, size_t len);

/* Replace the state: Phi as host c128 [4][N_Q][n][n] (converted to the
 * storage precision) and Sigma as host c128 [L*L][n_ext]; either may be NULL
 * to keep it. */
PQ_API pq_status pq_set_state(pq_ctx *ctx, const double *phi_c128, const double *sigma_c128);

/* Electron density per site (both spins) of G = [i nu + mu - eps_k - Sigma(k)]^-1 (App. A,
 * Eq. PA_Dyson) for the current Sigma and mu, square lattice:
 * n = (2T/N) sum_k sum_nu G(k, i nu) e^{i nu 0+}, summed in FP64 on the device over
 * n in [-M, M-1] (M = tau_matsubara) with the 1/(i nu) and 1/(i nu)^2 tails of G summed in
 * closed form (1/2 and -beta (eps_k - mu)/4 per spin).  mu is the Hartree-shifted chemical
 * potential of the solve (mu = 0 at half filling).  PQ_EINVAL on the Bethe lattice. */
PQ_API pq_status pq_density(pq_ctx *ctx, double *n_out);

/* The chemical potential of the last iteration (the one pq_init set, unless target_density
 * moves it). */
PQ_API pq_status pq_get_mu(const pq_ctx *ctx, double *mu_out);

/* Sizes: out[0..7] = L*L, n, N_Q, n_ext, Nnu, NOmega, bytes of device memory
 * held, storage bytes per complex vertex element. */
PQ_API pq_status pq_get_sizes(const pq_ctx *ctx, long long *out8);

/* Per-step device times (ms) of the last iteration, when time_steps was set:
 * out[0..PQ_NSTEPS-1] in the order of pq_step_name(i). */
#define PQ_NSTEPS 9
PQ_API pq_status pq_step_times(const pq_ctx *ctx, float *out, int n);
PQ_API const char *pq_step_name(int i);

/* Second-order self-energy without device allocation, for callers that
 * cannot call cudaMalloc: a host program that has handed all device memory
 * to its own allocator, or a plug-in called inside another solver's loop
 * where an allocation (and the device synchronisation it implies) is not
 * allowed.  The paper has no counterpart; this is the Sigma~1 of
 * pq_sigma_second_order computed without a context.
 *   sigma_dev: device c128 [L*L][n_omega+n_nu-1], the self-energy of G (read);
 *   out_dev:   device c128 [L*L][n_omega+n_nu-1], Sigma~1 (written);
 *   the other arguments are those of pq_init and pq_options; cuda_stream is
 *   a cudaStream_t (NULL = legacy default stream).
 * Work is queued on cuda_stream and the call returns without waiting: out_dev
 * is ready when the stream reaches that point.  All intermediates live in one
 * static device array of 6.73 MB that every GPU which loads the library holds
 * until the process exits; sizes beyond it are rejected with PQ_EINVAL:
 * L*L <= 16, 2*tau_matsubara <= 512, tau_panels*tau_order <= 512,
 * n_omega+n_nu-1 <= 128, tau_order <= 32.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  Every call shares the
 * array and leaves its contents behind; each call writes every element it
 * reads before reading it, so nothing has to be cleared, but calls whose
 * work overlaps on the GPU (other streams, other host threads) race on it.
 * Errors: PQ_EINVAL, PQ_ECUDA; pq_last_error(NULL) gives the message. */
PQ_API pq_status pq_sigma_second_order_noalloc(int lattice, double beta, double U, double mu, double hop,
                                               int L, int n_nu, int n_omega, int tau_panels, int tau_order,
                                               int tau_matsubara, const double *sigma_dev, double *out_dev,
                                               void *cuda_stream);

/* ---------------------------------------------------------------- batches
 * A batch iterates several independent solves of uneven size together on one
 * GPU.  Each iteration is one CUDA graph launch: every member's one-particle,
 * kernel-function, self-energy and assembly steps, then ONE persistent grouped
 * kernel over the tiles of the Bethe-Salpeter products of the members with
 * n < 512, then a gather of every member's convergence scalars for a single
 * device->host read.  A member with n >= 512 (its products fill the GPU alone)
 * runs its products in its own launch right after its other steps, as it does
 * outside a batch.
 * Members: contexts made by pq_init with PQ_SPLIT_BF16X3, or all with
 * PQ_SPLIT_FP16X3, and a single pass (q_chunk 0 or >= L*L, and the box fits),
 * on one device and one cuda_stream,
 * none poisoned.  The batch does not own them; they must outlive it, and
 * pq_iterate on a member is refused while it exists (the other calls work
 * between batch iterations).  The paper solves one problem at a time; this is
 * a throughput layer over the same iteration. */
typedef struct pq_batch pq_batch;

typedef struct {
  /* complex output columns per tile of the grouped kernel: 64 or 128; 0 = tune */
  int tile_cols;
  /* order of the members' tiles in the persistent schedule: 0 as given,
   * 1 largest matrix first; -1 = tune */
  int order;
  /* nonzero: record the device time of the grouped kernel and of the whole
   * iteration (pq_batch_times) */
  int time_steps;
} pq_batch_options;

/* Fill *opt with the defaults: tune both choices, no timing. */
PQ_API void pq_batch_default_options(pq_batch_options *opt);

/* Group count contexts.  When a choice is left to tuning, the first iteration
 * of pq_batch_iterate runs untimed (warm-up) and the next ones run the candidate
 * grouped kernels in turn (each a full, real iteration: the candidates compute
 * the same products), keeping the fastest; the graph is captured after that.  Errors: PQ_EINVAL (a
 * member that does not qualify, count < 1), PQ_ENOMEM, PQ_ECUDA;
 * pq_last_error(NULL) gives the message. */
PQ_API pq_status pq_batch_create(pq_batch **out, pq_ctx *const *ctxs, int count, const pq_batch_options *opt);

/* Run n_iter iterations of every member.  max_dsigma, when non-NULL, receives
 * count values: each member's max_k |Sigma_new - Sigma| of the last
 * iteration.  A member's PQ_ENAN or a timed-out device wait (PQ_ETIMEOUT)
 * poisons the batch and the members concerned. */
PQ_API pq_status pq_batch_iterate(pq_batch *b, int n_iter, double *max_dsigma);

/* The grouped kernel's configuration: tile columns, order (as in
 * pq_batch_options; -1 while tuning is not finished, and when no member has
 * n < 512, so that there is no grouped kernel) and, when tuned, the
 * device time in ms of each candidate (tile_cols 128/64 x order 0/1, in that
 * order; 0 where not run) in tuned_ms[4]. */
PQ_API pq_status pq_batch_config(const pq_batch *b, int *tile_cols, int *order, float *tuned_ms);

/* Device times (ms) of the last iteration when time_steps was set: out[0] =
 * the whole iteration (graph launch), out[1] = the grouped BSE kernel (0 when
 * there is none). */
PQ_API pq_status pq_batch_times(const pq_batch *b, float *out2);

/* Message of the last failure on the batch. */
PQ_API const char *pq_batch_last_error(const pq_batch *b);

/* Release the batch (the members stay valid and can be iterated alone).  NULL is a no-op. */
PQ_API void pq_batch_destroy(pq_batch *b);

/* Self-test of the bounded device waits, with no fault: one block waits on an
 * mbarrier that nothing arrives at, for at most limit_ms (1..10000) ms of
 * global time, then sets the context's wait-timeout flag, exactly as the
 * tensor-core and gather pipelines do when one of their waits gives up.  The
 * host side then handles the flag as after an iteration: the call returns
 * PQ_ETIMEOUT and the context is poisoned (later calls: PQ_ESTATE).  For the
 * tests of failure handling; the paper has no counterpart. */
PQ_API pq_status pq_selftest_wait_timeout(pq_ctx *ctx, int limit_ms);

/* Message of the last failure on ctx (or, when ctx is NULL, of the last
 * failed call that has no context: pq_init or pq_sigma_second_order_noalloc). */
PQ_API const char *pq_last_error(const pq_ctx *ctx);

/* Release the context and its device memory.  NULL is a no-op. */
PQ_API void pq_destroy(pq_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* PARQUET_GB300_H */
