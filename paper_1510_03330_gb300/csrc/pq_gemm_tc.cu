// TF32x3 Bethe-Salpeter products on the tcgen05 tensor cores, from complex64 operands.
//
// For every (r, Q) the BSE (App. A, Eq. PA_F_Phi) is one complex n x n x n
// product C = A B with A = s_r Gamma_r(Q) diag(X_r(Q)) and B = F_r(Q), both
// complex64, and the mixing Phi <- alpha C + (1 - alpha) Phi in the epilogue.
// Each FP32 operand x is split into x = h + l (h TF32, l read as TF32) inside
// this kernel, and a real product XY is taken as Xh Yh + Xh Yl + Xl Yh with FP32
// accumulation (~2^-22 per product).
//
// Complex arithmetic as two real products into one 128 x 256 accumulator:
// the B tile is staged as 384 K-major rows [-Bi ; Br ; Bi], so
//   D += Ar [Br | Bi]   (B rows 128..383)
//   D += Ai [-Bi | Br]  (B rows 0..255)
// leaves Re C in accumulator columns 0..127 and Im C in 128..255.
//
// One CTA owns a 128 x 128 complex output tile in tensor memory (columns
// 0..255).  The A split planes go from registers straight into tensor memory
// (tcgen05.st), so the MMAs read A there and only B from 64-byte-swizzled
// shared memory.  Eight producer warps fetch raw complex64 tiles with cp.async,
// convert them and stage the planes; one warp issues the MMAs; stages hand
// over through mbarriers, and tcgen05.commit releases each stage.  Operand rows
// are 64 bytes: 16 k per stage.
#include "pq_common.cuh"
#include "pq_internal.h"
#include "pq_tc.cuh"

namespace pq {

namespace {

constexpr int BM = 128, BNC = 128, NT = 256;
constexpr int B_BLOCK = BNC * 64;        // 128 K-major rows x 64 B
constexpr int B_PLANE = 3 * B_BLOCK;     // rows [-Bi ; Br ; Bi]
constexpr int NSTAGE = 2;                // split stages (B planes in shared memory, A planes in TMEM)
constexpr uint32_t D_COLS = 2 * BNC;     // accumulator: Re in 0..127, Im in 128..255
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t WAIT_TRIES = 1u << 24;

enum Scheme { TF32X3 = 0 };

template <int SC>
struct Traits;
template <>
struct Traits<TF32X3> {
  static constexpr int BK = 16;    // complex k per stage (16 x 4 B = one 64-byte row)
  static constexpr int KG = 4;     // k per 16-byte chunk of a staged row
  static constexpr int NRAW = 3;   // raw stages: cp.async two stages ahead
  static constexpr uint32_t IDESC = tc::idesc_tf32(BM, 2 * BNC, false);
};

template <int SC>
struct Layout {
  static constexpr int BK = Traits<SC>::BK;
  static constexpr int STAGE = 2 * B_PLANE;            // Bh, Bl
  static constexpr int RAW_A_ROW = BK * 8;             // complex64 bytes per raw A row
  static constexpr int RAW_A = BM * RAW_A_ROW;
  static constexpr int RAW_B_ROW = BNC * 8 + 16;       // padded by 16 bytes
  static constexpr int RAW_B = BK * RAW_B_ROW;
  static constexpr int RAW = RAW_A + RAW_B;
  static constexpr uint32_t A_PLANE_COLS = 16;         // 64 bytes of K per lane
  static constexpr uint32_t A_STAGE_COLS = 4 * A_PLANE_COLS;  // Arh Arl Aih Ail
  static constexpr size_t SMEM = (size_t)NSTAGE * STAGE + (size_t)Traits<SC>::NRAW * RAW + 1024;
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}

// h = tf32(x) exactly; the remainder is left in FP32 and the MMA uses its TF32 bits,
// an error of at most 2^-11 |l| <= 2^-22 |x|
__device__ __forceinline__ void split_tf32(float x, float &h, float &l) {
  h = tc::to_tf32(x);
  l = x - h;
}
__device__ __forceinline__ void mma_tmem_a(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  tc::mma_tf32_tmem_a(d, a, b, idesc, acc);
}

__device__ __forceinline__ void cp_async_mbar_arrive(void *bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// Warp roles: warps 0..7 (256 threads) fetch, convert and stage operands and run the
// epilogue; warp 8 allocates tensor memory and issues the MMAs.  Stages hand over through
// mbarriers only: raw_full (cp.async landed), raw_empty (raw tile converted),
// split_full (split planes staged), split_empty (MMAs of the stage done, tcgen05.commit).
template <int SC>
__global__ void __launch_bounds__(NT + 32, 1) bse_split_kernel(int n, const float2 *__restrict__ A,
                                                               const float2 *__restrict__ B, float2 *Phi,
                                                               float alpha, int *err) {
  using Tr = Traits<SC>;
  using Ly = Layout<SC>;
  constexpr int BK = Tr::BK, KG = Tr::KG, NRAW = Tr::NRAW;
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
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % NSTAGE;
      ok &= tc::mbar_wait(&split_full[s], (kt / NSTAGE) & 1, WAIT_TRIES);
      tc::fence_after_sync();
      if (lane == 0) {
        const uint32_t bh = tc::smem_u32(sm + s * Ly::STAGE), bl = bh + B_PLANE;
        const uint32_t a = tmem + D_COLS + (uint32_t)s * Ly::A_STAGE_COLS;
        const uint32_t arh = a, arl = a + 16, aih = a + 32, ail = a + 48;
#pragma unroll
        for (int j = 0; j < 2; ++j) {  // two k steps of 32 bytes per 64-byte row
          const uint32_t o = 32u * j, ak = 8u * j;
          auto d = [&](uint32_t b) { return tc::smem_desc(b + o, 16, 512, 4); };
          const uint32_t acc0 = (kt > 0 || j > 0) ? 1u : 0u;
          // D += Ar [Br | Bi]: B rows 128..383
          mma_tmem_a(tmem, arh + ak, d(bh + B_BLOCK), Tr::IDESC, acc0);
          mma_tmem_a(tmem, arh + ak, d(bl + B_BLOCK), Tr::IDESC, 1u);
          mma_tmem_a(tmem, arl + ak, d(bh + B_BLOCK), Tr::IDESC, 1u);
          // D += Ai [-Bi | Br]: B rows 0..255
          mma_tmem_a(tmem, aih + ak, d(bh), Tr::IDESC, 1u);
          mma_tmem_a(tmem, aih + ak, d(bl), Tr::IDESC, 1u);
          mma_tmem_a(tmem, ail + ak, d(bh), Tr::IDESC, 1u);
        }
        tc::mma_commit(&split_empty[s]);
        if (kt == KT - 1) tc::mma_commit(&done);
      }
      __syncwarp();
    }
  } else {
    // ---------------------------------------------------------------- producers
    // Operand fetch: cp.async copies the raw complex64 tiles of a stage (A: 128 rows x BK,
    // B: BK rows x 128) in 16-byte chunks, consecutive threads along each line, NRAW - 1
    // stages ahead of their conversion.
    // A conversion: warp w owns TMEM lanes 32(w%4).. (rows) and k half w/4; each thread
    //    reads its row's BK/2 values (A chunks are XOR-swizzled by row, so 8 consecutive rows
    //    hit 8 bank groups) and writes 8 columns of each of the four A planes into TMEM.
    // B conversion: thread task (column pair p, k group g of KG values) reads KG raw rows
    //    (padded so the two g of an 8-lane phase fall on different bank groups) and writes
    //    one 16-byte run of K to each of the six B plane rows of its two columns.
    const int a_row = 32 * (warp & 3) + lane, a_kh = warp >> 2;
    const uint32_t a_lane = (uint32_t)(32 * (warp & 3)) << 16;
    const int b_plo = lane & 3, b_glo = (lane >> 2) & 1, b_ghi = (lane >> 3) & 1, b_phi = (lane >> 4) & 1;
    const int b_p = b_plo + 4 * b_phi + 8 * warp, b_g = b_glo + 2 * b_ghi;
    unsigned char *raw0 = sm + NSTAGE * Ly::STAGE;
    constexpr int ACH = BK / 2;  // 16-byte chunks per raw A row

    // With e = tid + NT * i a thread's chunks are one base plus constant strides:
    // A row (tid / ACH) + i * (NT / ACH), chunk tid % ACH; B row (tid >> 6) + 4 i, chunk tid & 63.
    const int fa_r = tid / ACH, fa_c = tid % ACH, fb_r = tid >> 6, fb_c = tid & 63;
    const uint32_t fa_dst = (uint32_t)(fa_r * Ly::RAW_A_ROW + ((fa_c ^ (fa_r & 7)) << 4));
    const uint32_t fb_dst = (uint32_t)(Ly::RAW_A + fb_r * Ly::RAW_B_ROW + fb_c * 16);
    const float2 *fa_src = A + (long long)(row0 + fa_r) * n + 2 * fa_c;
    const float2 *fb_src = B + (long long)fb_r * n + col0 + 2 * fb_c;
    const uint32_t raw0_s = tc::smem_u32(raw0);
    constexpr int A_RSTEP = NT / ACH;  // rows between a thread's A chunks
    auto fetch = [&](int kt) {
      const int r_ = kt % NRAW;
      if (kt >= NRAW) ok &= tc::mbar_wait(&raw_empty[r_], ((kt - NRAW) / NRAW) & 1, WAIT_TRIES);
      const uint32_t base = raw0_s + (uint32_t)(r_ * Ly::RAW);
      const int k0 = kt * BK;
      const bool ka = k0 + 2 * fa_c < n, cb = col0 + 2 * fb_c < n;
#pragma unroll
      for (int i = 0; i < BK / 4; ++i) {
        const bool va = ka && row0 + fa_r + A_RSTEP * i < n;
        cp_async16(base + fa_dst + (uint32_t)(i * A_RSTEP * Ly::RAW_A_ROW),
                   va ? (const void *)(fa_src + (long long)A_RSTEP * i * n + k0) : (const void *)A, va);
        const bool vb = cb && k0 + fb_r + 4 * i < n;
        cp_async16(base + fb_dst + (uint32_t)(4 * i * Ly::RAW_B_ROW),
                   vb ? (const void *)(fb_src + (long long)(k0 + 4 * i) * n) : (const void *)B, vb);
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
      const unsigned char *ra = raw0 + r_ * Ly::RAW, *rb = ra + Ly::RAW_A;
      // ---- A: this thread's row, BK/2 complex values -> 8 TMEM columns of each plane
      {
        float rh[8], rl[8], ih[8], il[8];  // one value per TMEM column
#pragma unroll
        for (int i = 0; i < BK / 4; ++i) {
          const int c = a_kh * (BK / 4) + i;
          const float4 v = *reinterpret_cast<const float4 *>(ra + a_row * Ly::RAW_A_ROW + ((c ^ (a_row & 7)) << 4));
          split_tf32(v.x, rh[2 * i], rl[2 * i]);
          split_tf32(v.y, ih[2 * i], il[2 * i]);
          split_tf32(v.z, rh[2 * i + 1], rl[2 * i + 1]);
          split_tf32(v.w, ih[2 * i + 1], il[2 * i + 1]);
        }
        const uint32_t t = tmem + a_lane + D_COLS + (uint32_t)s * Ly::A_STAGE_COLS + 8u * a_kh;
        tc::tmem_st8(t, rh);
        tc::tmem_st8(t + 16, rl);
        tc::tmem_st8(t + 32, ih);
        tc::tmem_st8(t + 48, il);
      }
      // ---- B: KG rows x two columns
      float4 rbv[KG];
#pragma unroll
      for (int j = 0; j < KG; ++j)
        rbv[j] = *reinterpret_cast<const float4 *>(rb + (KG * b_g + j) * Ly::RAW_B_ROW + b_p * 16);
      tc::mbar_arrive_cta(&raw_empty[r_]);  // this thread is done reading the raw tile
      unsigned char *Bh = sm + s * Ly::STAGE, *Bl = Bh + B_PLANE;
      // columns 2p and 2p+1; the column with parity b_glo goes first (bank spread)
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int cc = t ^ b_glo;
        const int col = 2 * b_p + cc;
        uint4 rh, rl, ih, il, nih, nil;
        {
          float h[4], l[4], hi[4], li[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            split_tf32(cc ? rbv[j].z : rbv[j].x, h[j], l[j]);
            split_tf32(cc ? rbv[j].w : rbv[j].y, hi[j], li[j]);
          }
          rh = make_uint4(__float_as_uint(h[0]), __float_as_uint(h[1]), __float_as_uint(h[2]), __float_as_uint(h[3]));
          rl = make_uint4(__float_as_uint(l[0]), __float_as_uint(l[1]), __float_as_uint(l[2]), __float_as_uint(l[3]));
          ih = make_uint4(__float_as_uint(hi[0]), __float_as_uint(hi[1]), __float_as_uint(hi[2]),
                          __float_as_uint(hi[3]));
          il = make_uint4(__float_as_uint(li[0]), __float_as_uint(li[1]), __float_as_uint(li[2]),
                          __float_as_uint(li[3]));
          nih = make_uint4(ih.x ^ 0x80000000u, ih.y ^ 0x80000000u, ih.z ^ 0x80000000u, ih.w ^ 0x80000000u);
          nil = make_uint4(il.x ^ 0x80000000u, il.y ^ 0x80000000u, il.z ^ 0x80000000u, il.w ^ 0x80000000u);
        }
        const uint32_t o = (uint32_t)col * 64u + ((uint32_t)(b_g ^ ((col >> 1) & 3)) << 4);
        // rows: [0,128) -Bi, [128,256) Br, [256,384) Bi
        *reinterpret_cast<uint4 *>(Bh + o) = nih;
        *reinterpret_cast<uint4 *>(Bh + B_BLOCK + o) = rh;
        *reinterpret_cast<uint4 *>(Bh + 2 * B_BLOCK + o) = ih;
        *reinterpret_cast<uint4 *>(Bl + o) = nil;
        *reinterpret_cast<uint4 *>(Bl + B_BLOCK + o) = rl;
        *reinterpret_cast<uint4 *>(Bl + 2 * B_BLOCK + o) = il;
      }
      tc::tmem_wait_st();
      tc::fence_proxy_async();
      tc::fence_before_sync();
      tc::mbar_arrive_cta(&split_full[s]);
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

size_t bse_tc_smem_bytes() { return Layout<TF32X3>::SMEM; }

cudaError_t launch_bse_split(cudaStream_t st, int n, int batch, const float2 *A, const float2 *B, float2 *Phi,
                             float alpha, int *err) {
  const size_t sm = bse_tc_smem_bytes();
  dim3 grid((n + BNC - 1) / BNC, (n + BM - 1) / BM, batch);
  cudaError_t e = cudaFuncSetAttribute(bse_split_kernel<TF32X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  bse_split_kernel<TF32X3><<<grid, NT + 32, sm, st>>>(n, A, B, Phi, alpha, err);
  return cudaGetLastError();
}

}  // namespace pq
