// Private definition of a solve context, shared by the translation units of the
// C ABI (pq_api.cu: single solves, pq_batch.cu: batches of solves).
#pragma once

#include <string>
#include <utility>
#include <vector>

#include "../../include/parquet.h"
#include "pq_common.cuh"
#include "pq_internal.h"

struct pq_ctx {
  pq::Grid g{};
  pq::Sizes z{};
  pq_options opt{};
  pq::Buffers b{};
  cudaStream_t st = nullptr;
  bool c64 = false;
  bool poisoned = false;
  double lam[8] = {0};
  std::vector<std::pair<void *, size_t>> allocs;
  size_t bytes = 0;
  std::string err;
  cudaEvent_t ev[PQ_NSTEPS + 1] = {};
  std::vector<cudaEvent_t> pev;  // per-pass marks when the transfers run in several passes
  float times[PQ_NSTEPS] = {0};
  int iterations = 0;
  pq::BseProblem *probs = nullptr;  // device table of the BF16x3 BSE: one entry per pass, for each
                                    // assignment of the two Phi buffers when there are several passes
  bool swapped = false;             // the Phi buffers have traded places an odd number of times
  int last_qb = 0;               // q-momenta whose F the operand buffer holds
  bool chi_ready = false;        // chi computed during the last iteration (several passes)
  pq::BseProblem prob_host{};    // the single-pass entry of the table (for batches)
  bool in_batch = false;         // a batch holds this context: pq_iterate is refused
  bool krow_ok = false;          // split planes: b.krow holds the edge row sums of the current Phi
  double lam_max[4] = {0, 0, 0, 0};  // max |Re|, |Im| of Lambda per channel (FP16 scales)
  int bse_cols = 128;            // complex output columns per tile of the TMA-fed products
};


namespace pq {
// Device work of one iteration queued on the context's stream, without waiting; with
// bse == false the products of a single-pass iteration are left to the caller.
pq_status enqueue_iteration(pq_ctx *c, bool bse, bool timing);
// Host side of the end of an iteration from the context's first five device scalars.
pq_status finish_iteration(pq_ctx *c, const double *h, double *dmax, bool timing);
// Record a failure on c (or, for c == NULL, as the message of the last context-free call).
pq_status fail(pq_ctx *c, pq_status s, const char *fmt, ...);
}  // namespace pq
