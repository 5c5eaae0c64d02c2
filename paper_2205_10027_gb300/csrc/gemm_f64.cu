// FP64 GEMM on the CUDA cores, with the structure the pISTA path needs:
// lower-triangle-only outputs (symmetric results, the Cholesky trailing update) and
// k-ranges that skip the known zero blocks of triangular operands (triangular inverse,
// L^{-T} L^{-1}).  GB300 runs FP64 at about 2 FMA/clock/SM, so a modest register-blocked
// tile already keeps the FP64 pipe busy; the tensor-core path lives in gemm_tc.cu.
#include "gemm.h"

namespace glasso {

namespace {
constexpr int BM = 64, BN = 64, BK = 16, THREADS = 256;

// C[M,N] = alpha * op(A)[M,K] op(B)[K,N] + beta * C  for one 64x64 output tile per block.
__global__ void __launch_bounds__(THREADS) k_gemm_f64(const __grid_constant__ GemmArgs p) {
  dep_wait();
  dep_release();
  if (p.flag && *p.flag == 0) return;  // an earlier step failed (non-PD pivot)
  const int tm = blockIdx.y, tn = blockIdx.x;
  if (p.lower && tm < tn) return;
  const int64_t z = blockIdx.z;
  const double* __restrict__ A = p.A + z * p.sA;
  const double* __restrict__ B = p.B + z * p.sB;
  double* __restrict__ C = p.C + z * p.sC;
  const int row0 = tm * BM, col0 = tn * BN;

  int k_lo = 0, k_hi = p.K;
  if (p.krule == KR_LO_COL) k_lo = col0;
  else if (p.krule == KR_LO_ROW) k_lo = row0;
  else if (p.krule == KR_HI_ROW) k_hi = min(p.K, row0 + BM);
  else if (p.krule == KR_HI_COL) k_hi = min(p.K, col0 + BN);

  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = k_lo; k0 < k_hi; k0 += BK) {
    // stage op(A)[row0:row0+64, k0:k0+16] as As[k][m]
#pragma unroll
    for (int r = 0; r < (BM * BK) / THREADS; ++r) {
      const int e = tid + r * THREADS;
      if (!p.transA) {
        const int m = e >> 4, k = e & 15;  // 16 consecutive k of one row per 16 threads
        As[k][m] = A[(int64_t)(row0 + m) * p.lda + (k0 + k)];
      } else {
        const int k = e >> 6, m = e & 63;  // op(A)[m][k] = A[k][m]: rows of A are contiguous in m
        As[k][m] = A[(int64_t)(k0 + k) * p.lda + (row0 + m)];
      }
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / THREADS; ++r) {
      const int e = tid + r * THREADS;
      if (!p.transB) {
        const int k = e >> 6, n = e & 63;
        Bs[k][n] = B[(int64_t)(k0 + k) * p.ldb + (col0 + n)];
      } else {
        const int n = e >> 4, k = e & 15;  // op(B)[k][n] = B[n][k]
        Bs[k][n] = B[(int64_t)(col0 + n) * p.ldb + (k0 + k)];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tx + 16 * j;
      if (p.lower && c > r) continue;
      double* dst = C + (int64_t)r * p.ldc + c;
      const double v = p.alpha * acc[i][j];
      *dst = (p.beta == 0.0) ? v : fma(p.beta, *dst, v);
    }
  }
}
}  // namespace

void gemm_f64(const GemmArgs& a, int batch, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0) return;
  if (a.M % BM || a.N % BN || a.K % BK)
    throw Error(1, "gemm_f64: M, N must be multiples of 64 and K of 16");
  dim3 grid(a.N / BN, a.M / BM, batch);
  launch_dependent(k_gemm_f64, grid, THREADS, 0, st, a);
}

}  // namespace glasso
