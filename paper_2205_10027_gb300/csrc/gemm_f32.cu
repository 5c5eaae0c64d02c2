// Small dense products of the split-precision modes on the CUDA cores in FP32 arithmetic.
//
// The recursive factorisation issues hundreds of products with M, N <= 640 (its lowest
// levels); a tensor-core product of that size is dominated by fixed costs (operand split
// launch, TMEM allocation, pipeline fill, epilogue), while the CUDA cores finish it in a few
// microseconds.  FP64 operands are converted to FP32 when staged in shared memory (integer
// conversion), products accumulate in FP32 - the accuracy of the split products they
// replace - and the result is stored in FP64.  Same structure options as the other GEMMs
// (transposes, lower-triangle output, k-ranges of triangular operands, failure flag).
#include "gemm.h"

namespace glasso {

namespace {
// TILE x TILE output per block, BK = 16, 256 threads with (TILE / 16)^2 outputs each.
template <int TILE>
__global__ void __launch_bounds__(256) k_gemm_f32(const __grid_constant__ GemmArgs p) {
  constexpr int BK = 16, R = TILE / 16;
  if (p.flag && *p.flag == 0) return;
  const int tm = blockIdx.y, tn = blockIdx.x;
  const int row0 = tm * TILE, col0 = tn * TILE;
  if (p.lower && row0 + TILE <= col0) return;
  const double* __restrict__ A = p.A;
  const double* __restrict__ B = p.B;
  double* __restrict__ C = p.C;

  int k_lo = 0, k_hi = p.K;
  if (p.krule == KR_LO_COL) k_lo = col0;
  else if (p.krule == KR_LO_ROW) k_lo = row0;
  else if (p.krule == KR_HI_ROW) k_hi = min(p.K, row0 + TILE);
  else if (p.krule == KR_HI_COL) k_hi = min(p.K, col0 + TILE);
  k_lo = k_lo / BK * BK;

  __shared__ float As[BK][TILE + 1];
  __shared__ float Bs[BK][TILE + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = 0.f;

  for (int k0 = k_lo; k0 < k_hi; k0 += BK) {
    // stage op(A)[row0 .. + TILE, k0 .. + 16] as As[k][m] and op(B)[k0 .., col0 ..] as Bs[k][n]
#pragma unroll
    for (int r = 0; r < (TILE * BK) / 256; ++r) {
      const int e = tid + r * 256;
      if (!p.transA) {
        const int m = e >> 4, k = e & 15;  // 16 consecutive k of one row per 16 threads
        As[k][m] = f64_to_f32(A[(int64_t)(row0 + m) * p.lda + (k0 + k)]);
      } else {
        const int k = e / TILE, m = e % TILE;  // op(A)[m][k] = A[k][m]: contiguous in m
        As[k][m] = f64_to_f32(A[(int64_t)(k0 + k) * p.lda + (row0 + m)]);
      }
      if (!p.transB) {
        const int k = e / TILE, n = e % TILE;
        Bs[k][n] = f64_to_f32(B[(int64_t)(k0 + k) * p.ldb + (col0 + n)]);
      } else {
        const int n = e >> 4, k = e & 15;  // op(B)[k][n] = B[n][k]
        Bs[k][n] = f64_to_f32(B[(int64_t)(col0 + n) * p.ldb + (k0 + k)]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float a[R], b[R];
#pragma unroll
      for (int i = 0; i < R; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < R; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

  const float al = (float)p.alpha, be = (float)p.beta;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int r = row0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int c = col0 + tx + 16 * j;
      if (p.lower && c > r) continue;
      double* dst = C + (int64_t)r * p.ldc + c;
      const float v = al * acc[i][j];
      *dst = f32_to_f64(p.beta == 0.0 ? v : fmaf(be, f64_to_f32(*dst), v));
    }
  }
}
}  // namespace

bool gemm_f32_supported(const GemmArgs& a) {
  return a.M > 0 && a.N > 0 && a.K > 0 && a.M % 32 == 0 && a.N % 32 == 0 && a.K % 16 == 0 &&
         std::max(a.M, a.N) <= kSmallGemm && a.C != a.A && a.C != a.B;
}

void gemm_f32(const GemmArgs& a, cudaStream_t st) {
  if (!gemm_f32_supported(a)) throw Error(1, "gemm_f32: unsupported shape or in-place product");
  if (a.M % 64 == 0 && a.N % 64 == 0 && (int64_t)a.M * a.N >= 256 * 256) {
    k_gemm_f32<64><<<dim3(a.N / 64, a.M / 64), 256, 0, st>>>(a);
  } else {
    k_gemm_f32<32><<<dim3(a.N / 32, a.M / 32), 256, 0, st>>>(a);
  }
  LAUNCH_CHECK();
}

}  // namespace glasso
