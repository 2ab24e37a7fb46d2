// Split-precision Bethe-Salpeter products fed by TMA from pre-split operand planes.
//
// For every (r, Q) the BSE (App. A, Eq. PA_F_Phi) is one complex n x n x n
// product C = A B with A = s_r Gamma_r(Q) diag(X_r(Q)) and B = F_r(Q), and the
// mixing Phi <- alpha C + (1 - alpha) Phi in the epilogue.  The parquet
// assembly writes both operands already split into 16-bit planes, so this kernel
// does no conversion at all: a real product XY is taken as Xh Yh + Xh Yl + Xl Yh
// on the tensor cores with FP32 accumulation.  Two plane formats:
//   BF16: x = h + l with h = bf16(x), l = bf16(x - h) (F also keeps a third piece
//         for readback);
//   FP16: x 2^e = h + l with 11-bit pieces of the value scaled by the channel's
//         power of two (2^-22 per product instead of 2^-16); the epilogue takes
//         the scales back out exactly.
//
// Complex arithmetic per split product, into one 128 x 256 FP32 accumulator
// (Re C in columns 0..127, Im C in 128..255):
//   D[0:256]   += Ar [Br | Bi]     (N = 256: the Br and Bi planes sit side by side)
//   D[0:128]   += (-Ai) Bi         (N = 128, negated A)
//   D[128:256] += Ai Br            (N = 128)
//
// Accumulation in chunks: the tensor cores add each MMA's products into the FP32
// accumulator with a truncating alignment, so the error of a long accumulation grows
// with the number of updates (1.2e-6 relative on F_t after the 384 updates of n = 1024).
// The MMAs of one tile therefore accumulate KCH stages (512 k) at a time into one of the
// two tensor-memory accumulators, and the epilogue warps add each finished chunk into
// FP32 registers (rounding to nearest) and release the accumulator for the next chunk:
// the error per element is bounded by the chunk length, not by n.  Each epilogue thread
// holds 64 such sums (one row, 32 complex columns), so 128-column tiles take 16 epilogue
// warps and 64-column tiles 8.
//
// Operand layouts in shared memory (written by TMA, read by the MMAs):
//   A plane: 128 rows x 32 k, K-major, 64-byte rows with the 64-byte swizzle;
//   B plane: 32 k x 128 columns, MN-major, two 64-column atoms of 32 rows x 128 B
//            with the 128-byte swizzle; the planes of one stage are ordered
//            Brh, Bih, Brl, Bil so that [Br | Bi] is one N = 256 operand.
//
// Persistent kernel, one CTA per SM, warp-specialised: warp 0 issues the TMA
// loads of a 3-stage ring, warp 1 issues the MMAs, warps 2..9 run the epilogue.
// Tensor memory holds two accumulators, so the epilogue's reading of one chunk, and
// its output of a finished tile, overlap the MMAs of the next chunk.  Every mbarrier
// wait is bounded in time; a wait that gives up sets the error flag and the CTA winds
// down (draining its in-flight copies and MMAs, then freeing tensor memory).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "pq_common.cuh"
#include "pq_internal.h"
#include "pq_tc.cuh"
#include "pq_tma.cuh"

namespace pq {

namespace {

constexpr int BM = 128, BK = 32;
constexpr int A_PLANE = BM * BK * 2;               // 8 KB
constexpr int B_ATOM = BK * 128;                   // 4 KB: 32 k-rows x 64 columns
constexpr int STAGE_A = 4 * A_PLANE;               // Arh Arl Aih Ail
constexpr uint64_t WAIT_NS = 2000000000ull;        // 2 s per wait
constexpr int KCH = 16;                            // stages (of BK k) per accumulator chunk: 512 k

// Tile geometry of the two variants: BNC complex output columns per tile.
template <int BNC>
struct Geo {
  static constexpr int NBA = BNC / 64;             // 64-column atoms per B plane
  static constexpr int B_PLANE = NBA * B_ATOM;
  static constexpr int STAGE = STAGE_A + 4 * B_PLANE;  // + Brh Bih Brl Bil
  static constexpr int NS = BNC == 128 ? 3 : 4;         // 192 KB of stages either way
  // 128-column tiles: one accumulator [Re | Im] per buffer (2 BNC columns); 64-column tiles:
  // two, D1 = Ar [Br | Bi] and D2 = Ai [Br | Bi] (4 BNC columns)
  static constexpr bool TWO_D = BNC == 64;
  // epilogue warps: each holds 32 rows x (BNC / (N_EPI / 4)) complex columns of a tile's sums
  // (64 FP32 values per thread): 8 warps for 64-column tiles, 16 for 128-column tiles
  static constexpr int N_EPI = BNC / 8;
  static constexpr int NTHREADS = 64 + 32 * N_EPI;
  // registers per thread: the most that one CTA of NTHREADS can hold (warps are given
  // registers in groups of four, per thread in multiples of 8)
  static constexpr int MAXREG = (65536 / (((NTHREADS / 32 + 3) / 4) * 4 * 32)) / 8 * 8;
  static constexpr uint32_t ACC_COLS = (TWO_D ? 4 : 2) * BNC;
  static constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;   // two buffers
  static constexpr size_t SMEM = (size_t)NS * STAGE + 1024;
};

// kind::f16 instruction descriptor: F32 accumulator, A and B both BF16 (format 1) or both
// FP16 (format 0), A K-major, B MN-major, M = 128, optional negation of A.
constexpr uint32_t idesc(int n, bool neg_a, bool f16) {
  return (1u << 4) | ((f16 ? 0u : 1u) << 7) | ((f16 ? 0u : 1u) << 10) | ((neg_a ? 1u : 0u) << 13) | (1u << 16) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ uint64_t desc_a(uint32_t addr) { return tc::smem_desc(addr, 16, 512, 4); }
__device__ __forceinline__ uint64_t desc_b(uint32_t addr) { return tc::smem_desc(addr, B_ATOM, 1024, 2); }

struct Tile {
  const BseProblem *p;
  int z, row0, col0, kt;
};

// Problems whose first tile and size the CTA keeps in shared memory (a batch with more
// members searches the table in global memory).  The copies fit in the 1 KB of static
// shared memory the kernel has anyway: with more, the CTA's shared memory passes the
// 196 KB carveout, the next one (228 KB) leaves 28 KB of L1 instead of 60, and the
// products ran 35 % slower.
constexpr int PMAX = 64;

// Tile t of the launch: the problem whose tile range holds t (binary search on tile0, in the
// shared copies t0s/ns when nprob <= PMAX), then GEMM, row block and column block within it
// (columns fastest).  The shared copies keep the search off global memory: the epilogue's
// reads of Phi evict the table from L1, and every role decodes at every tile boundary.
template <int BNC>
__device__ __forceinline__ Tile decode(const BseProblem *__restrict__ probs, const long long *t0s, const int *ns,
                                       int nprob, long long t) {
  const bool sh = nprob <= PMAX;
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((sh ? t0s[mid] : probs[mid].tile0) <= t) lo = mid;
    else hi = mid - 1;
  }
  Tile r;
  r.p = probs + lo;
  const int n = sh ? ns[lo] : r.p->n, ntc = (n + BNC - 1) / BNC, per_z = ((n + BM - 1) / BM) * ntc;
  const long long u = t - (sh ? t0s[lo] : r.p->tile0);
  r.z = (int)(u / per_z);
  const int rem = (int)(u % per_z);
  r.row0 = (rem / ntc) * BM;
  r.col0 = (rem % ntc) * BNC;
  r.kt = (n + BK - 1) / BK;
  return r;
}

template <int BNC, bool F16>
__global__ void __maxnreg__(Geo<BNC>::MAXREG)
    bse_tma_kernel(const BseProblem *__restrict__ probs, int nprob, long long tiles, int *err) {
  using G = Geo<BNC>;
  constexpr int NS = G::NS, STAGE = G::STAGE, B_PLANE = G::B_PLANE;
  constexpr int N_EPI = G::N_EPI;
  constexpr uint32_t ID_PAIR = idesc(2 * BNC, false, F16), ID_ONE = idesc(BNC, false, F16),
                     ID_ONE_N = idesc(BNC, true, F16);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[NS], empty[NS], acc_full[2], acc_empty[2], drain;
  __shared__ uint32_t tslot;
  __shared__ long long t0s[PMAX];
  __shared__ int ns[PMAX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < nprob && i < PMAX; i += blockDim.x) {
    t0s[i] = probs[i].tile0;
    ns[i] = probs[i].n;
  }

  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&acc_full[i], 1);
      tc::mbar_init(&acc_empty[i], 32 * N_EPI);
    }
    tc::mbar_init(&drain, 1);
    tc::mbar_fence_init();
    for (int i = 0; i < nprob && i < 8; ++i) {
      tma::prefetch_map(&probs[i].mapA);
      tma::prefetch_map(&probs[i].mapB);
    }
  }
  if (warp == 1) tc::tmem_alloc(&tslot, G::TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  const uint32_t sbase = tc::smem_u32(sm);
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------ TMA producer
      long long it = 0;
      for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        const Tile T = decode<BNC>(probs, t0s, ns, nprob, t);
        const CUtensorMap *mA = &T.p->mapA, *mB = &T.p->mapB;
        for (int kt = 0; kt < T.kt; ++kt, ++it) {
          const int s = (int)(it % NS);
          if (it >= NS && !tc::mbar_wait_ns(&empty[s], (uint32_t)((it / NS - 1) & 1), WAIT_NS)) {
            ok = false;
            break;
          }
          tma::mbar_expect_tx(&full[s], STAGE);
          const uint32_t st = sbase + (uint32_t)(s * STAGE);
          const int k0 = kt * BK;
#pragma unroll
          for (int p = 0; p < 4; ++p) tma::load4(st + p * A_PLANE, mA, k0, T.row0, T.z, p, &full[s]);
#pragma unroll
          for (int w = 0; w < 4; ++w)
#pragma unroll
            for (int at = 0; at < G::NBA; ++at)
              tma::load4(st + STAGE_A + w * B_PLANE + at * B_ATOM, mB, T.col0 + 64 * at, k0, T.z, w, &full[s]);
        }
      }
      if (!ok) {
        // let the copies already issued land before the CTA exits
        for (long long j = it > NS ? it - NS : 0; j < it; ++j)
          tc::mbar_wait_ns(&full[j % NS], (uint32_t)((j / NS) & 1), WAIT_NS);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------------ MMA issuer
      long long it = 0, ch = 0;  // stages and accumulator chunks of this CTA
      bool issued = false;
      for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        const Tile T = decode<BNC>(probs, t0s, ns, nprob, t);
        const int kch = KCH;  // stages per accumulator chunk
        for (int k0 = 0; k0 < T.kt; k0 += kch, ++ch) {
          const int b = (int)(ch & 1);
          if (ch >= 2) {
            if (!tc::mbar_wait_ns(&acc_empty[b], (uint32_t)(((ch >> 1) - 1) & 1), WAIT_NS)) {
              ok = false;
              break;
            }
            tc::fence_after_sync();
          }
          const uint32_t d = tmem + (uint32_t)b * G::ACC_COLS;
          const int k1 = min(T.kt, k0 + kch);
          for (int kt = k0; kt < k1; ++kt, ++it) {
            const int s = (int)(it % NS);
            if (!tc::mbar_wait_ns(&full[s], (uint32_t)((it / NS) & 1), WAIT_NS)) {
              ok = false;
              break;
            }
            tc::fence_after_sync();
            const uint32_t sa = sbase + (uint32_t)(s * STAGE), sb = sa + STAGE_A;
#pragma unroll
            for (int j = 0; j < 2; ++j) {  // two K = 16 steps per stage
#pragma unroll
              for (int pr = 0; pr < 3; ++pr) {  // (Ah, Bh), (Ah, Bl), (Al, Bh)
                const int al = (pr == 2), bl = (pr == 1);
                const uint64_t ar = desc_a(sa + al * A_PLANE + 32 * j);
                const uint64_t ai = desc_a(sa + (2 + al) * A_PLANE + 32 * j);
                const uint32_t bb = sb + 2 * bl * B_PLANE + 2048 * j;
                const uint32_t acc = (kt > k0 || j || pr) ? 1u : 0u;  // the chunk's first MMA overwrites
                if constexpr (G::TWO_D) {
                  // two N = 2 BNC products on the same [Br | Bi]: fewer shared-memory operand
                  // bytes per flop than N = BNC ones; Re = D1 re - D2 im, Im = D1 im + D2 re
                  mma(d, ar, desc_b(bb), ID_PAIR, acc);            // D1 += Ar [Br | Bi]
                  mma(d + 2 * BNC, ai, desc_b(bb), ID_PAIR, acc);  // D2 += Ai [Br | Bi]
                } else {
                  mma(d, ar, desc_b(bb), ID_PAIR, acc);              // Re += Ar Br, Im += Ar Bi
                  mma(d, ai, desc_b(bb + B_PLANE), ID_ONE_N, 1u);    // Re -= Ai Bi
                  mma(d + BNC, ai, desc_b(bb), ID_ONE, 1u);          // Im += Ai Br
                }
              }
            }
            tc::mma_commit(&empty[s]);
            issued = true;
          }
          if (!ok) break;
          tc::mma_commit(&acc_full[b]);
        }
      }
      if (issued) {
        // all MMAs of this CTA complete before tensor memory is released
        tc::mma_commit(&drain);
        if (!tc::mbar_wait_ns(&drain, 0, WAIT_NS)) ok = false;
      }
    }
  } else {
    // -------------------------------------------------------------- epilogue
    constexpr int CW = BNC / (N_EPI / 4);  // complex columns per epilogue warp (N_EPI / 4 warps per lane quarter)
    constexpr int NP = CW / 16;   // 16-column pieces of them
    const int q = warp & 3, half = (warp - 2) >> 2;  // TMEM lane quarter (warp % 4) and column block
    uint32_t ch = 0;  // accumulator chunks consumed
    // largest |Re|, |Im| of the new Phi per channel, kept per warp while the tiles belong to one
    // problem and added to the problem's bound when they change
    const BseProblem *mp = nullptr;
    float mx0 = 0.f, mx1 = 0.f, mx2 = 0.f, mx3 = 0.f;
    auto flush = [&]() {
      if (mp && mp->phimax) {
        const unsigned am = __activemask();
        for (int o = 16; o > 0; o >>= 1) {
          mx0 = fmaxf(mx0, __shfl_xor_sync(am, mx0, o));
          mx1 = fmaxf(mx1, __shfl_xor_sync(am, mx1, o));
          mx2 = fmaxf(mx2, __shfl_xor_sync(am, mx2, o));
          mx3 = fmaxf(mx3, __shfl_xor_sync(am, mx3, o));
        }
        if (lane == 0) {
          atomicMax(mp->phimax + 0, __float_as_uint(mx0));
          atomicMax(mp->phimax + 1, __float_as_uint(mx1));
          atomicMax(mp->phimax + 2, __float_as_uint(mx2));
          atomicMax(mp->phimax + 3, __float_as_uint(mx3));
        }
      }
      mx0 = mx1 = mx2 = mx3 = 0.f;
    };
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
      const Tile T = decode<BNC>(probs, t0s, ns, nprob, t);
      if (T.p != mp) {
        flush();
        mp = T.p;
      }
      // this thread's row of the tile, columns [CW half, CW half + CW) of Re and Im, summed
      // over the accumulator chunks in FP32 registers
      float cr[NP][16], ci[NP][16];
#pragma unroll
      for (int pc = 0; pc < NP; ++pc)
#pragma unroll
        for (int i = 0; i < 16; ++i) cr[pc][i] = ci[pc][i] = 0.f;
      const int nch = (T.kt + KCH - 1) / KCH;
      for (int c = 0; c < nch; ++c, ++ch) {
        const int b = (int)(ch & 1);
        if (!tc::mbar_wait_ns(&acc_full[b], (uint32_t)((ch >> 1) & 1), WAIT_NS)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)b * G::ACC_COLS;
#pragma unroll
        for (int pc = 0; pc < NP; ++pc) {
#pragma unroll
          for (int h4 = 0; h4 < 16; h4 += 4) {
            const uint32_t col = (uint32_t)(CW * half + 16 * pc + h4);
            float u[4], v[4];
            if constexpr (G::TWO_D) {
              tc::tmem_ld4(tb + col, u);                    // D1: Ar Br
              tc::tmem_ld4(tb + 3 * BNC + col, v);          // D2: Ai Bi
#pragma unroll
              for (int i = 0; i < 4; ++i) cr[pc][h4 + i] += u[i] - v[i];
              tc::tmem_ld4(tb + BNC + col, u);              // D1: Ar Bi
              tc::tmem_ld4(tb + 2 * BNC + col, v);          // D2: Ai Br
#pragma unroll
              for (int i = 0; i < 4; ++i) ci[pc][h4 + i] += u[i] + v[i];
            } else {
              tc::tmem_ld4(tb + col, u);                    // Re
              tc::tmem_ld4(tb + BNC + col, v);              // Im
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                cr[pc][h4 + i] += u[i];
                ci[pc][h4 + i] += v[i];
              }
            }
          }
        }
        tc::fence_before_sync();
        tc::mbar_arrive_cta(&acc_empty[b]);  // the chunk is in registers: the MMAs may reuse it
      }
      if (!ok) break;
      const BseProblem &P = *T.p;
      const int n = P.n, row = T.row0 + 32 * q + lane;
      const int chan = T.z / P.zc;
      const float alpha = P.alpha * (P.uns ? P.uns[chan] : 1.f), beta = 1.0f - P.alpha;
      const long long slab = (long long)chan * P.phi_cs + P.phi_q0 + T.z % P.zc;
      const long long off0 = (slab * n + row) * (long long)n + T.col0 + CW * half;
      // the new Phi of this row at the frequency edges (n' = n_lo, n_hi) of each k' block:
      // summed here, the next iteration's K2row (Sec. II.A) needs no strided reads of Phi
      const int nnu = P.n_nu;
      float rsx = 0.f, rsy = 0.f, mx = 0.f;
      // mixes 16 columns (piece pc) of the product into Phi
      auto out_piece = [&](int pc, const float *vr, const float *vi) {
        const int c0 = T.col0 + CW * half + 16 * pc;  // first column of this piece
        const float2 *pi = P.phi_in + off0 + 16 * pc;
        float2 *po = P.phi_out + off0 + 16 * pc;
        const int lim = n - c0;
        int ph = c0 % nnu;  // frequency index of the column within its k' block
        auto edge = [&](float x, float y) {
          if (ph == 0 || ph == nnu - 1) {
            rsx += x;
            rsy += y;
          }
          ph = ph + 1 == nnu ? 0 : ph + 1;
          mx = fmaxf(mx, fmaxf(fabsf(x), fabsf(y)));
        };
        if (lim >= 16) {
#pragma unroll
          for (int i = 0; i < 16; i += 2) {
            float4 o = *reinterpret_cast<const float4 *>(pi + i);
            o.x = alpha * vr[i] + beta * o.x;
            o.y = alpha * vi[i] + beta * o.y;
            o.z = alpha * vr[i + 1] + beta * o.z;
            o.w = alpha * vi[i + 1] + beta * o.w;
            *reinterpret_cast<float4 *>(po + i) = o;
            edge(o.x, o.y);
            edge(o.z, o.w);
          }
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            if (i < lim) {
              const float2 o = pi[i];
              const float2 v = make_float2(alpha * vr[i] + beta * o.x, alpha * vi[i] + beta * o.y);
              po[i] = v;
              edge(v.x, v.y);
            }
          }
        }
      };
      if (row < n) {
#pragma unroll
        for (int pc = 0; pc < NP; ++pc) out_piece(pc, cr[pc], ci[pc]);
      }
      if (P.krow && row < n) {
        double2 *dst = P.krow + ((long long)chan * n + row) * P.phi_cs + P.phi_q0 + T.z % P.zc;
        atomicAdd(&dst->x, (double)rsx);
        atomicAdd(&dst->y, (double)rsy);
      }
      mx0 = chan == 0 ? fmaxf(mx0, mx) : mx0;
      mx1 = chan == 1 ? fmaxf(mx1, mx) : mx1;
      mx2 = chan == 2 ? fmaxf(mx2, mx) : mx2;
      mx3 = chan == 3 ? fmaxf(mx3, mx) : mx3;
    }
    flush();
  }
  if (!ok) atomicExch(err, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 1) tc::tmem_dealloc(tmem, G::TMEM_COLS);
}

}  // namespace

size_t bse_tma_smem_bytes(int bnc) { return bnc == 64 ? Geo<64>::SMEM : Geo<128>::SMEM; }

long long bse_tiles(int bnc, int n, int batch) {
  return (long long)((n + BM - 1) / BM) * ((n + bnc - 1) / bnc) * batch;
}

// The encoder is a driver entry point; it is looked up through the runtime so that the
// library itself does not link the driver (it loads on hosts without a GPU).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

CUresult make_bse_maps(void *gam_planes, void *fv_planes, int n, int ld, long long slabs, bool f16,
                       CUtensorMap *mapA, CUtensorMap *mapB) {
  const PFN_cuTensorMapEncodeTiled_v12000 cuTensorMapEncodeTiled = tensor_map_encoder();
  if (!cuTensorMapEncodeTiled) return CUDA_ERROR_NOT_FOUND;
  const cuuint64_t row = (cuuint64_t)ld * 2, mat = row * (cuuint64_t)n, plane = mat * (cuuint64_t)slabs;
  const CUtensorMapDataType dt = f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const cuuint32_t es[4] = {1, 1, 1, 1};
  {
    // A: x = k (contiguous), y = row, z = GEMM, w = plane (Arh, Arl, Aih, Ail)
    const cuuint64_t dims[4] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)slabs, 4};
    const cuuint64_t str[3] = {row, mat, plane};
    const cuuint32_t box[4] = {BK, BM, 1, 1};
    CUresult r = cuTensorMapEncodeTiled(mapA, dt, 4, gam_planes, dims, str, box, es,
                                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return r;
  }
  {
    // B: x = column (contiguous), y = k, z = GEMM, w = plane (Brh, Bih, Brl, Bil[, Brr, Bir])
    const cuuint64_t dims[4] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)slabs, f16 ? 4u : 6u};
    const cuuint64_t str[3] = {row, mat, plane};
    const cuuint32_t box[4] = {64, BK, 1, 1};
    return cuTensorMapEncodeTiled(mapB, dt, 4, fv_planes, dims, str, box, es,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
}

CUresult make_phi_rows_map(const void *phi, int n, long long slabs, int box_w, int box_h, CUtensorMap *map) {
  const PFN_cuTensorMapEncodeTiled_v12000 cuTensorMapEncodeTiled = tensor_map_encoder();
  if (!cuTensorMapEncodeTiled) return CUDA_ERROR_NOT_FOUND;
  // x = k' (contiguous complex64 words), y = k, z = (channel, Q)
  const cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)slabs};
  const cuuint64_t str[2] = {(cuuint64_t)n * 8, (cuuint64_t)n * n * 8};
  const cuuint32_t box[3] = {(cuuint32_t)box_w, 1, (cuuint32_t)box_h};
  const cuuint32_t es[3] = {1, 1, 1};
  return cuTensorMapEncodeTiled(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<void *>(phi), dims, str, box, es,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

template <int BNC, bool F16>
static cudaError_t launch_one(cudaStream_t st, unsigned grid, const BseProblem *probs, int nprob, long long tiles,
                              int *err) {
  cudaError_t e = cudaFuncSetAttribute(bse_tma_kernel<BNC, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Geo<BNC>::SMEM);
  if (e != cudaSuccess) return e;
  bse_tma_kernel<BNC, F16><<<grid, Geo<BNC>::NTHREADS, Geo<BNC>::SMEM, st>>>(probs, nprob, tiles, err);
  return cudaGetLastError();
}

cudaError_t launch_bse_tma(cudaStream_t st, int bnc, bool f16, const BseProblem *probs, int nprob, long long tiles,
                           int *err, int max_ctas) {
  if (tiles <= 0 || nprob <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (max_ctas > 0) sms = std::min(sms, max_ctas);
  const unsigned grid = (unsigned)std::min<long long>(tiles, sms);
  if (bnc == 64) return f16 ? launch_one<64, true>(st, grid, probs, nprob, tiles, err)
                            : launch_one<64, false>(st, grid, probs, nprob, tiles, err);
  return f16 ? launch_one<128, true>(st, grid, probs, nprob, tiles, err)
             : launch_one<128, false>(st, grid, probs, nprob, tiles, err);
}

}  // namespace pq
