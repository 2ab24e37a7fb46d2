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
// One CTA owns a 128 x 128 complex output tile in tensor memory (columns
// 0..255).  All 256 threads convert and stage the operands: the four A split
// planes go from registers straight into tensor memory (tcgen05.st, columns
// 256.. per stage), so the MMAs read A from tensor memory and only B from
// swizzled shared memory -- shared-memory bandwidth is the limit of a TF32
// product otherwise.  One thread issues the MMAs; tcgen05.commit releases each
// of the three stages back to the producers.
#include "pq_common.cuh"
#include "pq_internal.h"
#include "pq_tc.cuh"

namespace pq {

namespace {

constexpr int BM = 128, BNC = 128, BK = 16, NT = 256;
constexpr int B_PLANE = 3 * BNC * 64;   // 384 rows x 64 B
constexpr int STAGE = 2 * B_PLANE;      // Bh Bl
constexpr int NSTAGE = 2;               // split stages (B planes in shared memory, A planes in TMEM)
constexpr int RAW_A = BM * 128;         // raw complex64 A tile: 128 rows x 16 values, 16-byte chunks XOR-swizzled
constexpr int RAW_B_ROW = BNC * 8 + 16; // raw B tile row (128 values) padded by 16 bytes
constexpr int RAW_B = BK * RAW_B_ROW;
constexpr int RAW = RAW_A + RAW_B;
constexpr int NRAW = 3;                 // raw stages: cp.async runs two stages ahead
constexpr uint32_t D_COLS = 2 * BNC;    // accumulator: Re in 0..127, Im in 128..255
constexpr uint32_t A_STAGE_COLS = 4 * BK;  // Arh Arl Aih Ail, BK columns each
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t WAIT_TRIES = 1u << 24;

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}

__device__ __forceinline__ void split(float x, float &h, float &l) {
  h = tc::to_tf32(x);
  l = tc::to_tf32(x - h);
}

__device__ __forceinline__ void cp_async_mbar_arrive(void *bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive(void *bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(tc::smem_u32(bar))
               : "memory");
}

// Warp roles: warps 0..7 (256 threads) fetch, convert and stage operands and run the
// epilogue; warp 8 allocates tensor memory and issues the MMAs.  Stages hand over through
// mbarriers only: raw_full (cp.async landed), raw_empty (raw tile converted),
// split_full (TF32 planes staged), split_empty (MMAs of the stage done, tcgen05.commit).
__global__ void __launch_bounds__(NT + 32, 1) bse_tf32x3_kernel(int n, const float2 *__restrict__ A,
                                                                const float2 *__restrict__ B, float2 *Phi,
                                                                float alpha, int *err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t raw_full[NRAW], raw_empty[NRAW], split_full[NSTAGE], split_empty[NSTAGE], done;
  __shared__ uint32_t tslot;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BNC;
  const long long nn = (long long)n * n;
  A += blockIdx.z * nn;
  B += blockIdx.z * nn;
  Phi += blockIdx.z * nn;
  const int KT = (n + BK - 1) / BK;

  if (tid == 0) {
    for (int i = 0; i < NRAW; ++i) {
      tc::mbar_init(&raw_full[i], NT);
      tc::mbar_init(&raw_empty[i], NT);
    }
    for (int i = 0; i < NSTAGE; ++i) {
      tc::mbar_init(&split_full[i], NT);
      tc::mbar_init(&split_empty[i], 1);
    }
    tc::mbar_init(&done, 1);
    tc::mbar_fence_init();
  }
  if (warp == 8) tc::tmem_alloc(&tslot, TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  bool ok = true;

  if (warp == 8) {
    // ---------------------------------------------------------------- MMA issuer
    const uint32_t idesc = tc::idesc_tf32(BM, 2 * BNC, false);
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % NSTAGE;
      ok &= tc::mbar_wait(&split_full[s], (kt / NSTAGE) & 1, WAIT_TRIES);
      tc::fence_after_sync();
      if (lane == 0) {
        const uint32_t bh = tc::smem_u32(sm + s * STAGE), bl = bh + B_PLANE;
        const uint32_t a = tmem + D_COLS + (uint32_t)s * A_STAGE_COLS;
        const uint32_t arh = a, arl = a + BK, aih = a + 2 * BK, ail = a + 3 * BK;
#pragma unroll
        for (int j = 0; j < BK / 8; ++j) {
          const uint32_t o = 32u * j, ak = 8u * j;
          auto d = [&](uint32_t b) { return tc::smem_desc(b + o, 16, 512, 4); };
          const uint32_t acc0 = (kt > 0 || j > 0) ? 1u : 0u;
          // D += Ar [Br | Bi]: B rows 128..383
          tc::mma_tf32_tmem_a(tmem, arh + ak, d(bh + BNC * 64), idesc, acc0);
          tc::mma_tf32_tmem_a(tmem, arh + ak, d(bl + BNC * 64), idesc, 1u);
          tc::mma_tf32_tmem_a(tmem, arl + ak, d(bh + BNC * 64), idesc, 1u);
          // D += Ai [-Bi | Br]: B rows 0..255
          tc::mma_tf32_tmem_a(tmem, aih + ak, d(bh), idesc, 1u);
          tc::mma_tf32_tmem_a(tmem, aih + ak, d(bl), idesc, 1u);
          tc::mma_tf32_tmem_a(tmem, ail + ak, d(bh), idesc, 1u);
        }
        tc::mma_commit(&split_empty[s]);
        if (kt == KT - 1) tc::mma_commit(&done);
      }
      __syncwarp();
    }
  } else {
    // ---------------------------------------------------------------- producers
    // Operand fetch: cp.async copies the raw complex64 tiles of a stage (A: 128 rows x 128 B,
    // B: 16 rows x 1 KB) in 16-byte chunks, eight consecutive threads per 128-byte line,
    // NRAW - 1 stages ahead of their conversion.
    // A conversion: warp w owns TMEM lanes 32(w%4).. (rows) and k half w/4; each thread
    //    reads its row's 8 values (A chunks are XOR-swizzled by row, so 8 consecutive rows
    //    hit 8 bank groups) and writes 8 columns of each of the four A planes into TMEM.
    // B conversion: thread task (column pair p, quad kq) reads B[4kq + j][2p, 2p+1], j = 0..3
    //    (rows padded so the two kq of an 8-lane phase fall on different bank groups) and
    //    writes 16-byte runs of K of the six B plane rows of its two columns.
    const int a_row = 32 * (warp & 3) + lane, a_kh = warp >> 2;
    const uint32_t a_lane = (uint32_t)(32 * (warp & 3)) << 16;
    const int b_plo = lane & 3, b_kqlo = (lane >> 2) & 1, b_kqhi = (lane >> 3) & 1, b_phi = (lane >> 4) & 1;
    const int b_p = b_plo + 4 * b_phi + 8 * warp, b_kq = b_kqlo + 2 * b_kqhi;
    unsigned char *raw0 = sm + NSTAGE * STAGE;

    auto fetch = [&](int kt) {
      const int r_ = kt % NRAW;
      if (kt >= NRAW) ok &= tc::mbar_wait(&raw_empty[r_], ((kt - NRAW) / NRAW) & 1, WAIT_TRIES);
      unsigned char *ra = raw0 + r_ * RAW, *rb = ra + RAW_A;
      const int k0 = kt * BK;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int e = tid + NT * i;
        const int r = e >> 3, c = e & 7;  // A row, 16-byte chunk (2 complex values)
        const int gr = row0 + r, k = k0 + 2 * c;
        const bool va = gr < n && k < n;
        cp_async16(tc::smem_u32(ra + r * 128 + ((c ^ (r & 7)) << 4)),
                   va ? (const void *)(A + (long long)gr * n + k) : (const void *)A, va);
        const int br = e >> 6, bc = e & 63;  // B row (k), 16-byte chunk (column pair)
        const int gk = k0 + br, col = col0 + 2 * bc;
        const bool vb = gk < n && col < n;
        cp_async16(tc::smem_u32(rb + br * RAW_B_ROW + bc * 16),
                   vb ? (const void *)(B + (long long)gk * n + col) : (const void *)B, vb);
      }
      cp_async_mbar_arrive(&raw_full[r_]);
    };

    for (int kt = 0; kt < NRAW - 1 && kt < KT; ++kt) fetch(kt);
    for (int kt = 0; kt < KT; ++kt) {
      if (kt + NRAW - 1 < KT) fetch(kt + NRAW - 1);
      const int r_ = kt % NRAW, s = kt % NSTAGE;
      ok &= tc::mbar_wait(&raw_full[r_], (kt / NRAW) & 1, WAIT_TRIES);
      if (kt >= NSTAGE) ok &= tc::mbar_wait(&split_empty[s], ((kt - NSTAGE) / NSTAGE) & 1, WAIT_TRIES);
      tc::fence_after_sync();
      const unsigned char *ra = raw0 + r_ * RAW, *rb = ra + RAW_A;
      {
        float rh[8], rl[8], ih[8], il[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int c = 4 * a_kh + i;
          const float4 v = *reinterpret_cast<const float4 *>(ra + a_row * 128 + ((c ^ (a_row & 7)) << 4));
          split(v.x, rh[2 * i], rl[2 * i]);
          split(v.y, ih[2 * i], il[2 * i]);
          split(v.z, rh[2 * i + 1], rl[2 * i + 1]);
          split(v.w, ih[2 * i + 1], il[2 * i + 1]);
        }
        const uint32_t t = tmem + a_lane + D_COLS + (uint32_t)s * A_STAGE_COLS + 8u * a_kh;
        tc::tmem_st8(t, rh);
        tc::tmem_st8(t + BK, rl);
        tc::tmem_st8(t + 2 * BK, ih);
        tc::tmem_st8(t + 3 * BK, il);
      }
      float4 rbv[4];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        rbv[j] = *reinterpret_cast<const float4 *>(rb + (4 * b_kq + j) * RAW_B_ROW + b_p * 16);
      mbar_arrive(&raw_empty[r_]);  // this thread is done reading the raw tile
      unsigned char *Bh = sm + s * STAGE, *Bl = Bh + B_PLANE;
      // columns 2p and 2p+1; the column with parity b_kqlo goes first (bank spread)
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int cc = t ^ b_kqlo;
        const int col = 2 * b_p + cc;
        float4 rh, rl, ih, il;
        const float x0 = cc ? rbv[0].z : rbv[0].x, x1 = cc ? rbv[1].z : rbv[1].x;
        const float x2 = cc ? rbv[2].z : rbv[2].x, x3 = cc ? rbv[3].z : rbv[3].x;
        const float y0 = cc ? rbv[0].w : rbv[0].y, y1 = cc ? rbv[1].w : rbv[1].y;
        const float y2 = cc ? rbv[2].w : rbv[2].y, y3 = cc ? rbv[3].w : rbv[3].y;
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
      tc::tmem_wait_st();
      tc::fence_proxy_async();
      tc::fence_before_sync();
      mbar_arrive(&split_full[s]);
    }

    // ---------------------------------------------------------------- epilogue
    ok &= tc::mbar_wait(&done, 0, WAIT_TRIES);
    tc::fence_after_sync();
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
  }
  if (!ok) atomicExch(err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 8) tc::tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace

size_t bse_tc_smem_bytes() { return (size_t)NSTAGE * STAGE + (size_t)NRAW * RAW + 1024; }

cudaError_t launch_bse_tf32x3(cudaStream_t st, int n, int batch, const float2 *A, const float2 *B, float2 *Phi,
                              float alpha, int *err) {
  const size_t sm = bse_tc_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(bse_tf32x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid((n + BNC - 1) / BNC, (n + BM - 1) / BM, batch);
  bse_tf32x3_kernel<<<grid, NT + 32, sm, st>>>(n, A, B, Phi, alpha, err);
  return cudaGetLastError();
}

}  // namespace pq
