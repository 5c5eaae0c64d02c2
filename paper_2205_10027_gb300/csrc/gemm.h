// Dense products of the pISTA path: the argument block shared by the FP64 (CUDA-core)
// and the split-precision tensor-core GEMMs.
#pragma once
#include <algorithm>
#include "common.cuh"

namespace glasso {

// Which k-range a 64-row x 64-column (or larger) output tile needs.
enum KRule : int {
  KR_FULL = 0,    // all of [0, K)
  KR_LO_COL = 1,  // [col0, K): B is lower triangular (B[k][j] = 0 for k < j)
  KR_LO_ROW = 2,  // [row0, K): op(A) is upper triangular (A = X^T with X lower)
  KR_HI_ROW = 3,  // [0, row0 + tile): A is lower triangular (A[i][k] = 0 for k > i)
  KR_HI_COL = 4   // [0, col0 + tile): op(B) is upper triangular (op(B)[k][j] = 0 for k > j)
};

// C = alpha op(A) op(B) + beta C.  op(A)[i][k] = transA ? A[k*lda+i] : A[i*lda+k];
// op(B)[k][j] = transB ? B[j*ldb+k] : B[k*ldb+j].  Row-major, batch strides sA/sB/sC.
// lower != 0: only the tiles on or below the diagonal are computed and, in diagonal tiles,
// only entries with column <= row are written.  beta == 0: C is not read.
// flag != nullptr: the kernel does nothing when *flag == 0 (an earlier failed pivot).
struct GemmArgs {
  const double* A;
  const double* B;
  double* C;
  int64_t lda, ldb, ldc;
  int64_t sA, sB, sC;
  int M, N, K;
  double alpha, beta;
  int transA, transB, lower, krule;
  const int* flag;
};

inline GemmArgs gemm_args(const double* A, int64_t lda, int transA, const double* B, int64_t ldb,
                          int transB, double* C, int64_t ldc, int M, int N, int K, double alpha,
                          double beta) {
  GemmArgs g{};
  g.A = A; g.B = B; g.C = C;
  g.lda = lda; g.ldb = ldb; g.ldc = ldc;
  g.M = M; g.N = N; g.K = K;
  g.alpha = alpha; g.beta = beta;
  g.transA = transA; g.transB = transB;
  return g;
}

void gemm_f64(const GemmArgs& a, int batch, cudaStream_t st);

// Products with max(M, N) <= kSmallGemm and K <= 256 run, in the split-precision modes, on
// the FP32 CUDA-core kernel (gemm_f32.cu): at that size a tensor-core product is dominated by
// its fixed costs.  M, N multiples of 64, C distinct from A and B.
constexpr int kSmallGemm = 256;
bool gemm_f32_supported(const GemmArgs& a);
void gemm_f32(const GemmArgs& a, cudaStream_t st);

}  // namespace glasso
