// Split-precision Bethe-Salpeter products on the tcgen05 tensor cores.
//
// For every (r, Q) the BSE (App. A, Eq. PA_F_Phi) is one complex n x n x n
// product C = A B with A = s_r Gamma_r(Q) diag(X_r(Q)) and B = F_r(Q), both
// complex64, and the mixing Phi <- alpha C + (1 - alpha) Phi in the epilogue.
// Each FP32 operand x is split into TF32 parts x = h + l (h = tf32(x),
// l = tf32(x - h)); a real product X Y is taken as Xh Yh + Xh Yl + Xl Yh with
// FP32 accumulation (the TF32x3 scheme, ~2^-22 relative per product).
//
// Complex arithmetic as two real products into one 128 x 256 accumulator:
// the B tile is staged as 384 K-major rows [-Bi ; Br ; Bi], so
//   D += Ar [Br | Bi]   (B rows 128..383)
//   D += Ai [-Bi | Br]  (B rows 0..255)
// leaves Re C in accumulator columns 0..127 and Im C in 128..255.
//
// One CTA owns a 128 x 128 complex output tile in tensor memory.  All 256
// threads convert and stage the operands (global -> registers -> split ->
// swizzled shared memory), one thread issues the MMAs, and tcgen05.commit
// releases each of the two shared-memory stages back to the producers.
#include "pq_common.cuh"
#include "pq_internal.h"
#include "pq_tc.cuh"

namespace pq {

namespace {

constexpr int BM = 128, BNC = 128, BK = 16, NT = 256;
constexpr int A_PLANE = BM * 64;        // 128 rows x 64 B
constexpr int B_PLANE = 3 * BNC * 64;   // 384 rows x 64 B
constexpr int STAGE = 4 * A_PLANE + 2 * B_PLANE;  // Arh Arl Aih Ail Bh Bl
constexpr int NSTAGE = 2;
constexpr uint32_t TMEM_COLS = 256;
constexpr uint32_t WAIT_TRIES = 1u << 24;

__device__ __forceinline__ void split(float x, float &h, float &l) {
  h = tc::to_tf32(x);
  l = tc::to_tf32(x - h);
}

__global__ void __launch_bounds__(NT, 1) bse_tf32x3_kernel(int n, const float2 *__restrict__ A,
                                                           const float2 *__restrict__ B, float2 *Phi, float alpha,
                                                           int *err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bars[NSTAGE];
  __shared__ uint32_t tslot;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BNC;
  const long long nn = (long long)n * n;
  A += blockIdx.z * nn;
  B += blockIdx.z * nn;
  Phi += blockIdx.z * nn;

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) tc::mbar_init(&bars[s], 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(&tslot, TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  const uint32_t idesc = tc::idesc_tf32(BM, 2 * BNC, false);

  // Producer work split (per stage: A 128 rows x 16 k, B 16 k x 128 columns, complex64).
  // A: thread task (row r, quad kq) holds A[r][4kq .. 4kq+3] (two float4); lanes 0..7 of a
  //    warp take 8 consecutive rows of one quad, so each 8-lane phase of a 16-byte store
  //    covers the 8 distinct 16-byte bank groups of the 64-byte-swizzled layout.
  // B: thread task (column pair p, quad kq) holds B[4kq + j][2p, 2p+1] for j = 0..3 (four
  //    float4) and writes 16-byte runs of K for each of its two columns; the lane map makes
  //    each 8-lane phase hit 8 distinct bank groups.
  const int a_rlo = lane & 7, a_kq = (lane >> 3) & 3;
  const int b_plo = lane & 3, b_kqlo = (lane >> 2) & 1, b_kqhi = (lane >> 3) & 1, b_phi = (lane >> 4) & 1;
  const int b_p = b_plo + 4 * b_phi + 8 * warp, b_kq = b_kqlo + 2 * b_kqhi;
  float4 ra[4], rb[4];
  auto load = [&](int kt) {
    const int k0 = kt * BK;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r = 8 * (warp + 8 * i) + a_rlo, gr = row0 + r, k = k0 + 4 * a_kq;
      const float4 *src = reinterpret_cast<const float4 *>(A + (long long)gr * n + k);
      ra[2 * i] = (gr < n && k < n) ? src[0] : make_float4(0.f, 0.f, 0.f, 0.f);
      ra[2 * i + 1] = (gr < n && k + 2 < n) ? src[1] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int c = col0 + 2 * b_p;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int kr = k0 + 4 * b_kq + j;
      rb[j] = (kr < n && c < n) ? *reinterpret_cast<const float4 *>(B + (long long)kr * n + c)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto stage_store = [&](int s) {
    unsigned char *st = sm + s * STAGE;
    unsigned char *Arh = st, *Arl = st + A_PLANE, *Aih = st + 2 * A_PLANE, *Ail = st + 3 * A_PLANE;
    unsigned char *Bh = st + 4 * A_PLANE, *Bl = Bh + B_PLANE;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r = 8 * (warp + 8 * i) + a_rlo;
      const float4 u = ra[2 * i], v = ra[2 * i + 1];  // (re,im) at k, k+1 and k+2, k+3
      float4 rh, rl, ih, il;
      split(u.x, rh.x, rl.x);
      split(u.z, rh.y, rl.y);
      split(v.x, rh.z, rl.z);
      split(v.z, rh.w, rl.w);
      split(u.y, ih.x, il.x);
      split(u.w, ih.y, il.y);
      split(v.y, ih.z, il.z);
      split(v.w, ih.w, il.w);
      const uint32_t o = tc::sw64_offset(r, 4 * a_kq);
      *reinterpret_cast<float4 *>(Arh + o) = rh;
      *reinterpret_cast<float4 *>(Arl + o) = rl;
      *reinterpret_cast<float4 *>(Aih + o) = ih;
      *reinterpret_cast<float4 *>(Ail + o) = il;
    }
    // columns 2p and 2p+1; the column with parity b_kqlo goes first (bank spread)
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int cc = t ^ b_kqlo;
      const int col = 2 * b_p + cc;
      float4 rh, rl, ih, il;
      const float x0 = cc ? rb[0].z : rb[0].x, x1 = cc ? rb[1].z : rb[1].x;
      const float x2 = cc ? rb[2].z : rb[2].x, x3 = cc ? rb[3].z : rb[3].x;
      const float y0 = cc ? rb[0].w : rb[0].y, y1 = cc ? rb[1].w : rb[1].y;
      const float y2 = cc ? rb[2].w : rb[2].y, y3 = cc ? rb[3].w : rb[3].y;
      split(x0, rh.x, rl.x);
      split(x1, rh.y, rl.y);
      split(x2, rh.z, rl.z);
      split(x3, rh.w, rl.w);
      split(y0, ih.x, il.x);
      split(y1, ih.y, il.y);
      split(y2, ih.z, il.z);
      split(y3, ih.w, il.w);
      const uint32_t o = tc::sw64_offset(col, 4 * b_kq);
      const uint32_t ob = (uint32_t)BNC * 64u;  // one 128-row block
      // rows: [0,128) -Bi, [128,256) Br, [256,384) Bi
      *reinterpret_cast<float4 *>(Bh + o) = make_float4(-ih.x, -ih.y, -ih.z, -ih.w);
      *reinterpret_cast<float4 *>(Bh + ob + o) = rh;
      *reinterpret_cast<float4 *>(Bh + 2 * ob + o) = ih;
      *reinterpret_cast<float4 *>(Bl + o) = make_float4(-il.x, -il.y, -il.z, -il.w);
      *reinterpret_cast<float4 *>(Bl + ob + o) = rl;
      *reinterpret_cast<float4 *>(Bl + 2 * ob + o) = il;
    }
  };

  const int KT = (n + BK - 1) / BK;
  bool ok = true;
  load(0);
  for (int kt = 0; kt < KT; ++kt) {
    const int s = kt % NSTAGE;
    if (kt >= NSTAGE) ok &= tc::mbar_wait(&bars[s], ((kt - NSTAGE) / NSTAGE) & 1, WAIT_TRIES);
    stage_store(s);
    if (kt + 1 < KT) load(kt + 1);
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t st = tc::smem_u32(sm + s * STAGE);
      const uint32_t arh = st, arl = st + A_PLANE, aih = st + 2 * A_PLANE, ail = st + 3 * A_PLANE;
      const uint32_t bh = st + 4 * A_PLANE, bl = bh + B_PLANE;
#pragma unroll
      for (int j = 0; j < BK / 8; ++j) {
        const uint32_t o = 32u * j;
        auto d = [&](uint32_t a) { return tc::smem_desc(a + o, 16, 512, 4); };
        const uint32_t acc0 = (kt > 0 || j > 0) ? 1u : 0u;
        // D += Ar [Br | Bi]: B rows 128..383
        tc::mma_tf32(tmem, d(arh), d(bh + BNC * 64), idesc, acc0);
        tc::mma_tf32(tmem, d(arh), d(bl + BNC * 64), idesc, 1u);
        tc::mma_tf32(tmem, d(arl), d(bh + BNC * 64), idesc, 1u);
        // D += Ai [-Bi | Br]: B rows 0..255
        tc::mma_tf32(tmem, d(aih), d(bh), idesc, 1u);
        tc::mma_tf32(tmem, d(aih), d(bl), idesc, 1u);
        tc::mma_tf32(tmem, d(ail), d(bh), idesc, 1u);
      }
      tc::mma_commit(&bars[s]);
    }
  }
  // the last NSTAGE commits (or fewer) are still outstanding
  for (int kt = (KT > NSTAGE ? KT - NSTAGE : 0); kt < KT; ++kt)
    ok &= tc::mbar_wait(&bars[kt % NSTAGE], (kt / NSTAGE) & 1, WAIT_TRIES);
  tc::fence_after_sync();
  if (!ok) atomicExch(err, 1);

  // epilogue: warp w reads TMEM lanes 32*(w%4) .. +31, columns half (w/4)
  const int q = warp & 3, half = warp >> 2;
  const int row = row0 + 32 * q + lane;
  const float beta = 1.0f - alpha;
#pragma unroll 1
  for (int c = 64 * half; c < 64 * half + 64; c += 16) {
    float cr[16], ci[16];
    tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c, cr);
    tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(BNC + c), ci);
    if (row < n) {
      float2 *p = Phi + (long long)row * n + col0 + c;
      const int lim = n - (col0 + c);
      if (lim >= 16) {
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
          float4 o = *reinterpret_cast<float4 *>(p + i);
          o.x = alpha * cr[i] + beta * o.x;
          o.y = alpha * ci[i] + beta * o.y;
          o.z = alpha * cr[i + 1] + beta * o.z;
          o.w = alpha * ci[i + 1] + beta * o.w;
          *reinterpret_cast<float4 *>(p + i) = o;
        }
      } else {
        for (int i = 0; i < lim; ++i) {
          float2 o = p[i];
          p[i] = make_float2(alpha * cr[i] + beta * o.x, alpha * ci[i] + beta * o.y);
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace

size_t bse_tc_smem_bytes() { return (size_t)NSTAGE * STAGE + 1024; }

cudaError_t launch_bse_tf32x3(cudaStream_t st, int n, int batch, const float2 *A, const float2 *B, float2 *Phi,
                              float alpha, int *err) {
  const size_t sm = bse_tc_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(bse_tf32x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid((n + BNC - 1) / BNC, (n + BM - 1) / BM, batch);
  bse_tf32x3_kernel<<<grid, NT, sm, st>>>(n, A, B, Phi, alpha, err);
  return cudaGetLastError();
}

}  // namespace pq
