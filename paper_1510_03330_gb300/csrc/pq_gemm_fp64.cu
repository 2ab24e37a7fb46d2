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

__global__ void __launch_bounds__(NT) zgemm_kernel(int M, int N, int K, double2 alpha, const double2 *__restrict__ A,
                                                   int lda, long long sA, const double2 *__restrict__ B, int ldb,
                                                   long long sB, double2 beta, double2 *C, int ldc, long long sC) {
  __shared__ double2 As[BK][BM];
  __shared__ double2 Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  A += blockIdx.z * sA;
  B += blockIdx.z * sB;
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
  zgemm_kernel<<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
  return cudaGetLastError();
}

}  // namespace pq
