// FP64 complex GEMM on the CUDA cores (DFMA), batched:
//   C[b] = alpha * A[b] * B[b] + beta * C[b],  A: M x K, B: K x N, C: M x N,
// row-major complex128 with leading dimensions and batch strides in elements.
// It carries the FP64 Bethe-Salpeter products Phi_r(Q) = [s_r Gamma_r X_r](Q) F_r(Q)
// (App. A, Eq. PA_F_Phi) with the linear mixing in the epilogue
// (alpha = mixing weight, beta = 1 - alpha, C = the old Phi), and the small
// transforms of the imaginary-time route to Sigma~1 (Sec. II.B).
#include "pq_common.cuh"
#include "pq_internal.h"

namespace pq {

namespace {
constexpr int BM = 64, BN = 64, BK = 8, NT = 256;

// kchunk > 0: split-K, blockIdx.z = split index, the split covers
// k in [z*kchunk, min(K, (z+1)*kchunk)) and writes its partial to C + z*sC.
__global__ void __launch_bounds__(NT) zgemm_kernel(int M, int N, int K, double2 alpha, const double2 *__restrict__ A,
                                                   int lda, long long sA, const double2 *__restrict__ B, int ldb,
                                                   long long sB, double2 beta, double2 *C, int ldc, long long sC,
                                                   int kchunk) {
  __shared__ double2 As[BK][BM];
  __shared__ double2 Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  if (kchunk > 0) {
    const int kb = blockIdx.z * kchunk;
    A += kb;
    B += (long long)kb * ldb;
    K = min(K - kb, kchunk);
  } else {
    A += blockIdx.z * sA;
    B += blockIdx.z * sB;
  }
  C += blockIdx.z * sC;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);

  for (int k0 = 0; k0 < K; k0 += BK) {
    // A tile: BM rows x BK cols, 2 elements per thread
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      int e = tid + t * NT;
      int r = e / BK, c = e % BK;
      int gr = row0 + r, gc = k0 + c;
      As[c][r] = (gr < M && gc < K) ? A[(long long)gr * lda + gc] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      int e = tid + t * NT;
      int r = e / BN, c = e % BN;
      int gr = k0 + r, gc = col0 + c;
      Bs[r][c] = (gr < K && gc < N) ? B[(long long)gr * ldb + gc] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cfma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  const bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gr = row0 + ty + 16 * i;
    if (gr >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gc = col0 + tx + 16 * j;
      if (gc >= N) continue;
      double2 *cp = C + (long long)gr * ldc + gc;
      double2 v = cmul(alpha, acc[i][j]);
      if (use_beta) v = cfma(beta, *cp, v);
      *cp = v;
    }
  }
}
}  // namespace

cudaError_t zgemm_fp64(cudaStream_t st, int M, int N, int K, double2 alpha, const double2 *A, int lda, long long sA,
                       const double2 *B, int ldb, long long sB, double2 beta, double2 *C, int ldc, long long sC,
                       int batch) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
  zgemm_kernel<<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, 0);
  return cudaGetLastError();
}

namespace {
__global__ void splitk_reduce(int M, int N, int splits, double2 alpha, const double2 *__restrict__ W, double2 beta,
                              double2 *C, int ldc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * N) return;
  double2 s = make_double2(0.0, 0.0);
  for (int z = 0; z < splits; ++z) s = s + W[(long long)z * M * N + i];
  double2 *cp = C + (long long)(i / N) * ldc + i % N;
  double2 v = cmul(alpha, s);
  if (beta.x != 0.0 || beta.y != 0.0) v = cfma(beta, *cp, v);
  *cp = v;
}
}  // namespace

int zgemm_splits(int M, int N, int K, long long work_elems) {
  long long tiles = (long long)((N + BN - 1) / BN) * ((M + BM - 1) / BM);
  long long want = (4 * 152 + tiles - 1) / tiles;          // about four CTAs per SM
  long long kcap = (K + 4 * BK - 1) / (4 * BK);             // at least four k-steps per split
  long long wcap = work_elems / ((long long)M * N);
  long long s = want < kcap ? want : kcap;
  if (s > wcap) s = wcap;
  return s < 1 ? 1 : (int)s;
}

cudaError_t zgemm_fp64_splitk(cudaStream_t st, int M, int N, int K, double2 alpha, const double2 *A, int lda,
                              const double2 *B, int ldb, double2 beta, double2 *C, int ldc, double2 *work,
                              long long work_elems) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  int splits = zgemm_splits(M, N, K, work_elems);
  if (splits <= 1) return zgemm_fp64(st, M, N, K, alpha, A, lda, 0, B, ldb, 0, beta, C, ldc, 0, 1);
  int kchunk = (K + splits - 1) / splits;
  splits = (K + kchunk - 1) / kchunk;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
  zgemm_kernel<<<grid, NT, 0, st>>>(M, N, K, make_double2(1.0, 0.0), A, lda, 0, B, ldb, 0, make_double2(0.0, 0.0),
                                    work, N, (long long)M * N, kchunk);
  splitk_reduce<<<(M * N + 255) / 256, 256, 0, st>>>(M, N, splits, alpha, work, beta, C, ldc);
  return cudaGetLastError();
}

}  // namespace pq
