// Batches of independent parquet solves on one GPU (C ABI, include/parquet.h).
//
// An iteration of the batch is every member's iteration with the Bethe-Salpeter
// products (Eq. PA_F_Phi) of the small members (n < 512) in ONE persistent grouped launch
// of the TMA-fed split-precision kernel: its problem table lists each member's products
// with the first tile of each, so the small solves share the SMs in one schedule.  A
// member whose matrices fill the GPU alone (n >= 512) runs its products in its own launch
// right after its other steps, as it does alone: grouping such members measured slower
// (three n = 576 members: 27.0 ms grouped against 25.2 ms in three launches, same clocks).
// The whole iteration (members' steps, grouped products, gather of the members'
// convergence scalars and their device->host copy) is captured once as a CUDA
// graph and replayed; the members' steps are captured on four branch streams (the members
// with n >= 512 one after another on the first, the smaller ones round robin on the other
// three), so the graph runs independent small members concurrently.  Two choices of the grouped launch are tuned on the first
// real iterations: the tile width (64 or 128 complex output columns; narrow tiles
// waste less of the MMA on small matrices) and the order of the members in the
// schedule (as given, or largest matrix first so the longest tiles start early).
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pq_ctx.h"

struct pq_batch {
  std::vector<pq_ctx *> m;
  cudaStream_t user_st = nullptr;  // the members' stream
  cudaStream_t st = nullptr;       // the batch's own stream (capturable)
  cudaStream_t br[4] = {};         // branch streams: members' steps run concurrently, round robin
  cudaEvent_t fork = nullptr, join[4] = {};
  pq_batch_options opt{};
  pq::BseProblem *tab[2][2] = {};  // device problem tables [tile 128 / 64][order given / largest first]
  long long tiles[2] = {0, 0};
  const double **scal = nullptr;   // device: the members' scalar arrays
  double *gather = nullptr;        // device: 5 scalars per member + the grouped kernel's flag
  double *host = nullptr;          // pinned copy of gather
  int *err = nullptr;              // device: timeout flag of the grouped kernel
  std::vector<std::pair<int, int>> cand;  // candidate (tile index, order) still to time
  bool warmed = false;             // the untimed first iteration that precedes the tuning ran
  std::vector<int> branch;         // branch stream of each member
  std::vector<char> own;           // the member runs its products in its own launch (n >= kOwnN)
  int ngroup = 0;                  // members whose products are in the grouped launch
  float tuned[4] = {0, 0, 0, 0};
  int tile = -1, order = -1;       // chosen (indices into tab)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev[3] = {};
  float times[2] = {0, 0};
  bool poisoned = false;
  std::string errmsg;
};

namespace {

const int kTileCols[2] = {128, 64};
const int kOwnN = 512;  // members with n >= kOwnN keep their own product launch

pq_status bfail(pq_batch *b, pq_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b) {
    b->errmsg = buf;
    if (s == PQ_ECUDA || s == PQ_ENAN || s == PQ_ETIMEOUT) b->poisoned = true;
  } else {
    pq::fail(nullptr, s, "%s", buf);
  }
  return s;
}

#define BCK(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return bfail(b, PQ_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

__global__ void gather_kernel(const double *const *scal, int count, const int *err, double *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count)
    for (int j = 0; j < 5; ++j) out[5 * i + j] = scal[i][j];
  if (i == 0) out[5 * count] = (double)*err;
}

// Elapsed time between two recorded events; 0 (and no error left behind for the next
// launch check to find) if either was not recorded.
float elapsed(cudaEvent_t a, cudaEvent_t z) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, z) != cudaSuccess) {
    cudaGetLastError();
    ms = 0.f;
  }
  return ms;
}

// Every member's steps, the grouped products with candidate (ti, order), the gather and its copy.
// In a graph capture the timing events become record nodes of the graph (external records);
// a plain record during capture would only order work inside the capture.
pq_status enqueue_all(pq_batch *b, int ti, int order, bool timing, bool in_graph = false) {
  nvtxRangePushA("pq.batch_iteration");
  struct Pop {
    ~Pop() { nvtxRangePop(); }
  } pop;
  auto rec = [&](cudaEvent_t e) {
    return in_graph ? cudaEventRecordWithFlags(e, b->st, cudaEventRecordExternal) : cudaEventRecord(e, b->st);
  };
  if (timing) BCK(rec(b->ev[0]));
  // fork: the members' steps go to the branch streams, joined before the grouped products
  const int nbr = (int)std::min<size_t>(4, b->m.size());
  BCK(cudaEventRecord(b->fork, b->st));
  for (int j = 0; j < nbr; ++j) BCK(cudaStreamWaitEvent(b->br[j], b->fork, 0));
  for (size_t i = 0; i < b->m.size(); ++i) {
    pq_ctx *c = b->m[i];
    cudaStream_t keep = c->st;
    c->st = b->br[b->branch[i] % nbr];
    pq_status s = pq::enqueue_iteration(c, b->own[i] != 0, false);
    c->st = keep;
    if (s != PQ_OK) return bfail(b, s, "member step failed: %s", c->err.c_str());
  }
  for (int j = 0; j < nbr; ++j) {
    BCK(cudaEventRecord(b->join[j], b->br[j]));
    BCK(cudaStreamWaitEvent(b->st, b->join[j], 0));
  }
  if (timing) BCK(rec(b->ev[1]));
  if (b->ngroup > 0)
    BCK(pq::launch_bse_tma(b->st, kTileCols[ti], b->m[0]->b.vfmt == pq::V_F16P, b->tab[ti][order], b->ngroup,
                           b->tiles[ti], b->err, 0));
  if (timing) BCK(rec(b->ev[2]));
  const int n = (int)b->m.size();
  gather_kernel<<<(n + 127) / 128, 128, 0, b->st>>>(b->scal, n, b->err, b->gather);
  BCK(cudaGetLastError());
  BCK(cudaMemcpyAsync(b->host, b->gather, sizeof(double) * (5 * n + 1), cudaMemcpyDeviceToHost, b->st));
  return PQ_OK;
}

pq_status capture(pq_batch *b) {
  BCK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeRelaxed));
  pq_status s = enqueue_all(b, b->tile, b->order, b->opt.time_steps != 0, true);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->st, &g);
  if (s != PQ_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return bfail(b, PQ_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  b->graph = g;
  BCK(cudaGraphInstantiate(&b->exec, g, 0));
  return PQ_OK;
}

void release(pq_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto &e : b->ev)
    if (e) cudaEventDestroy(e);
  for (auto &r : b->tab)
    for (auto &t : r)
      if (t) cudaFree(t);
  if (b->scal) cudaFree((void *)b->scal);
  if (b->gather) cudaFree(b->gather);
  if (b->err) cudaFree(b->err);
  if (b->host) cudaFreeHost(b->host);
  if (b->fork) cudaEventDestroy(b->fork);
  for (auto &e : b->join)
    if (e) cudaEventDestroy(e);
  for (auto &t : b->br)
    if (t) cudaStreamDestroy(t);
  if (b->st) cudaStreamDestroy(b->st);
  for (pq_ctx *c : b->m) c->in_batch = false;
}

}  // namespace

extern "C" {

void pq_batch_default_options(pq_batch_options *o) {
  if (!o) return;
  o->tile_cols = 0;
  o->order = -1;
  o->time_steps = 0;
}

pq_status pq_batch_create(pq_batch **out, pq_ctx *const *ctxs, int count, const pq_batch_options *opt) {
  if (!out) return bfail(nullptr, PQ_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctxs || count < 1) return bfail(nullptr, PQ_EINVAL, "a batch needs at least one context");
  pq_batch_options o;
  pq_batch_default_options(&o);
  if (opt) o = *opt;
  if (o.tile_cols != 0 && o.tile_cols != 64 && o.tile_cols != 128)
    return bfail(nullptr, PQ_EINVAL, "tile_cols must be 0, 64 or 128");
  if (o.order < -1 || o.order > 1) return bfail(nullptr, PQ_EINVAL, "order must be -1, 0 or 1");
  for (int i = 0; i < count; ++i) {
    pq_ctx *c = ctxs[i];
    if (!c) return bfail(nullptr, PQ_EINVAL, "member %d is NULL", i);
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return bfail(nullptr, PQ_EINVAL, "member %d appears twice", i);
    if (c->poisoned) return bfail(nullptr, PQ_EINVAL, "member %d is poisoned", i);
    if (c->in_batch) return bfail(nullptr, PQ_EINVAL, "member %d already belongs to a batch", i);
    if (!pq::split_planes(c->b.vfmt))
      return bfail(nullptr, PQ_EINVAL, "member %d is neither PQ_SPLIT_BF16X3 nor PQ_SPLIT_FP16X3", i);
    if (c->b.vfmt != ctxs[0]->b.vfmt)
      return bfail(nullptr, PQ_EINVAL, "member %d has another operand format than member 0", i);
    if (c->b.q_chunk < c->g.nk) return bfail(nullptr, PQ_EINVAL, "member %d runs in several passes", i);
    if (c->opt.target_density > 0.0)
      return bfail(nullptr, PQ_EINVAL, "member %d holds a fixed density (its mu search waits on the host)", i);
    if (c->st != ctxs[0]->st) return bfail(nullptr, PQ_EINVAL, "member %d uses another stream", i);
  }
  pq_batch *b = new pq_batch();
  b->m.assign(ctxs, ctxs + count);
  b->user_st = ctxs[0]->st;
  b->opt = o;
  auto bad = [&](cudaError_t e, const char *what) {
    if (e == cudaSuccess) return false;
    bfail(nullptr, PQ_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    release(b);
    delete b;
    return true;
  };
  if (bad(cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking), "stream")) return PQ_ECUDA;
  for (auto &t : b->br)
    if (bad(cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking), "stream")) return PQ_ECUDA;
  if (bad(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event")) return PQ_ECUDA;
  for (auto &e : b->join)
    if (bad(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event")) return PQ_ECUDA;
  for (auto &e : b->ev)
    if (bad(cudaEventCreate(&e), "event")) return PQ_ECUDA;
  if (bad(cudaMalloc((void **)&b->scal, sizeof(double *) * count), "alloc")) return PQ_ECUDA;
  if (bad(cudaMalloc((void **)&b->gather, sizeof(double) * (5 * count + 1)), "alloc")) return PQ_ECUDA;
  if (bad(cudaMalloc((void **)&b->err, sizeof(int)), "alloc")) return PQ_ECUDA;
  if (bad(cudaMallocHost((void **)&b->host, sizeof(double) * (5 * count + 1)), "pinned alloc")) return PQ_ECUDA;
  if (bad(cudaMemset(b->err, 0, sizeof(int)), "memset")) return PQ_ECUDA;
  std::vector<const double *> sp(count);
  for (int i = 0; i < count; ++i) sp[i] = ctxs[i]->b.scal;
  if (bad(cudaMemcpy((void *)b->scal, sp.data(), sizeof(double *) * count, cudaMemcpyHostToDevice), "upload"))
    return PQ_ECUDA;
  // problem tables of the grouped members: in the given order, or by decreasing matrix size
  b->own.assign(count, 0);
  std::vector<int> idx;
  for (int i = 0; i < count; ++i) {
    b->own[i] = ctxs[i]->g.n >= kOwnN;
    if (!b->own[i]) idx.push_back(i);
  }
  const int ng = (int)idx.size();
  b->ngroup = ng;
  std::vector<int> big = idx;
  std::stable_sort(big.begin(), big.end(), [&](int x, int y) { return ctxs[x]->g.n > ctxs[y]->g.n; });
  for (int ti = 0; ti < 2 && ng > 0; ++ti) {
    for (int od = 0; od < 2; ++od) {
      const std::vector<int> &ord = od ? big : idx;
      std::vector<pq::BseProblem> t(ng);
      long long tile0 = 0;
      for (int i = 0; i < ng; ++i) {
        t[i] = ctxs[ord[i]]->prob_host;
        t[i].tile0 = tile0;
        tile0 += pq::bse_tiles(kTileCols[ti], t[i].n, t[i].batch);
      }
      b->tiles[ti] = tile0;
      if (bad(cudaMalloc((void **)&b->tab[ti][od], sizeof(pq::BseProblem) * ng), "alloc")) return PQ_ECUDA;
      if (bad(cudaMemcpy(b->tab[ti][od], t.data(), sizeof(pq::BseProblem) * ng, cudaMemcpyHostToDevice),
              "upload"))
        return PQ_ECUDA;
    }
  }
  for (int ti = 0; ti < 2 && ng > 0; ++ti) {
    if (o.tile_cols && kTileCols[ti] != o.tile_cols) continue;
    for (int od = 0; od < 2; ++od) {
      if (o.order >= 0 && od != o.order) continue;
      b->cand.push_back({ti, od});
    }
  }
  if (b->cand.size() == 1) {
    b->tile = b->cand[0].first;
    b->order = b->cand[0].second;
    b->cand.clear();
  }
  // branch streams: the members whose matrices fill the GPU (n >= kOwnN) run their steps and
  // their products one after another on branch 0, where concurrency would only contend for
  // it; the smaller ones are spread over the other branches, so their short kernels overlap
  b->branch.assign(count, 0);
  int next = 0;
  for (int i = 0; i < count; ++i)
    if (!b->own[i]) b->branch[i] = 1 + (next++ % 3);
  for (pq_ctx *c : b->m) c->in_batch = true;
  *out = b;
  return PQ_OK;
}

pq_status pq_batch_iterate(pq_batch *b, int n_iter, double *max_dsigma) {
  if (!b) return PQ_EINVAL;
  if (b->poisoned) return bfail(b, PQ_ESTATE, "batch poisoned by an earlier error: %s", b->errmsg.c_str());
  if (n_iter < 0) return bfail(b, PQ_EINVAL, "n_iter < 0");
  BCK(cudaStreamSynchronize(b->user_st));
  const int n = (int)b->m.size();
  for (int it = 0; it < n_iter; ++it) {
    if (!b->cand.empty() && !b->warmed) {
      // the first iteration runs untimed with the first candidate: the candidates are then
      // timed on equal terms (clocks up, caches and the members' tables warm)
      const auto cnd = b->cand.front();
      pq_status s = enqueue_all(b, cnd.first, cnd.second, false);
      if (s != PQ_OK) return s;
      BCK(cudaStreamSynchronize(b->st));
      b->warmed = true;
    } else if (!b->cand.empty()) {
      // tuning: this iteration runs the next candidate, eagerly, with its grouped launch timed
      const auto cnd = b->cand.front();
      pq_status s = enqueue_all(b, cnd.first, cnd.second, true);
      if (s != PQ_OK) return s;
      BCK(cudaStreamSynchronize(b->st));
      b->tuned[2 * cnd.first + cnd.second] = elapsed(b->ev[1], b->ev[2]);
      b->cand.erase(b->cand.begin());
      if (b->cand.empty()) {
        int best = -1;
        for (int k = 0; k < 4; ++k)
          if (b->tuned[k] > 0.f && (best < 0 || b->tuned[k] < b->tuned[best])) best = k;
        b->tile = best / 2;
        b->order = best % 2;
      }
    } else {
      if (!b->exec) {
        pq_status s = capture(b);
        if (s != PQ_OK) return s;
      }
      BCK(cudaGraphLaunch(b->exec, b->st));
      BCK(cudaStreamSynchronize(b->st));
      if (b->opt.time_steps) {
        b->times[0] = elapsed(b->ev[0], b->ev[2]);
        b->times[1] = elapsed(b->ev[1], b->ev[2]);
      }
    }
    const double *h = b->host;
    if (h[5 * n] != 0.0) {
      for (pq_ctx *c : b->m) {
        c->poisoned = true;
        c->err = "a wait of the batch's grouped tensor-core kernel gave up; the state is invalid";
      }
      return bfail(b, PQ_ETIMEOUT, "a wait of the grouped tensor-core kernel gave up; the states are invalid");
    }
    for (int i = 0; i < n; ++i) {
      double d = 0.0;
      pq_status s = pq::finish_iteration(b->m[i], h + 5 * i, &d, false);
      if (s != PQ_OK) return bfail(b, s, "member %d: %s", i, b->m[i]->err.c_str());
      if (max_dsigma) max_dsigma[i] = d;
    }
  }
  return PQ_OK;
}

pq_status pq_batch_config(const pq_batch *b, int *tile_cols, int *order, float *tuned_ms) {
  if (!b) return PQ_EINVAL;
  if (tile_cols) *tile_cols = b->tile >= 0 ? kTileCols[b->tile] : -1;
  if (order) *order = b->order;
  if (tuned_ms)
    for (int k = 0; k < 4; ++k) tuned_ms[k] = b->tuned[k];
  return PQ_OK;
}

pq_status pq_batch_times(const pq_batch *b, float *out2) {
  if (!b || !out2) return PQ_EINVAL;
  out2[0] = b->times[0];
  out2[1] = b->times[1];
  return PQ_OK;
}

const char *pq_batch_last_error(const pq_batch *b) { return b ? b->errmsg.c_str() : ""; }

void pq_batch_destroy(pq_batch *b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  release(b);
  delete b;
}

}  // extern "C"
