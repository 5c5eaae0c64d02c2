// Small dense products of the split-precision modes on the CUDA cores in FP32 arithmetic.
//
// The recursive factorisation issues hundreds of products with M, N, K <= 256 (its lowest
// levels); a tensor-core product of that size is dominated by fixed costs (operand split
// launch, TMEM allocation, pipeline fill, epilogue), while the CUDA cores finish it in a few
// microseconds.  FP64 operands are converted to FP32 when staged in shared memory (integer
// conversion), products accumulate in FP32 - the accuracy of the split products they
// replace - and the result is stored in FP64 (added to an FP64 C in FP64 when beta != 0).  Same structure options as the other GEMMs
// (transposes, lower-triangle output, k-ranges of triangular operands, failure flag).
#include <mutex>
#include "gemm.h"

namespace glasso {

namespace {
constexpr int TILE = 32;          // output tile per block (small tiles: many blocks per product)
constexpr int KMAX = 256;         // largest k-range staged at once

// Stage rows [r0, r0 + TILE) x k-range [k_lo, k_lo + kn) of an operand into S[r][k] (pitch
// kp), converting to FP32.  KFAST: the operand is stored as G[r][k] (k contiguous); else as
// G[k][r] (r contiguous).  Each thread issues its loads in batches of 16 or 32 independent
// ones before converting any, so a block keeps its whole tile in flight.
template <bool KFAST>
__device__ __forceinline__ void stage_operand(const double* __restrict__ G, int64_t ld, int r0, int k_lo, int kn,
                                              float* S, int kp, int warp, int lane) {
  if (KFAST) {
    // warp w: rows w + 8 i (i < 4); lanes: k = lane + 32 q (q < 8 covers kn <= 256)
    double v[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int r = warp + 8 * i, k = lane + 32 * q;
        v[i][q] = k < kn ? G[(int64_t)(r0 + r) * ld + k_lo + k] : 0.0;
      }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int r = warp + 8 * i, k = lane + 32 * q;
        if (k < kn) S[r * kp + k] = f64_to_f32(v[i][q]);
      }
  } else {
    // warp w: k = k0 + w + 8 i (i < 16); lanes: r = lane
    for (int k0 = 0; k0 < kn; k0 += 128) {
      double v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int k = k0 + warp + 8 * i;
        v[i] = k < kn ? G[(int64_t)(k_lo + k) * ld + r0 + lane] : 0.0;
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int k = k0 + warp + 8 * i;
        if (k < kn) S[lane * kp + k] = f64_to_f32(v[i]);
      }
    }
  }
}

// One TILE x TILE output tile per block, 256 threads with 2 x 2 outputs each (rows ty + 16 i,
// columns tx + 16 j).  The tile's whole k-range of op(A) and op(B) is staged at once in
// shared memory as As[m][k] and Bs[n][k] (row pitch kn + 1, odd, so that both the staging
// stores and the strided reads hit distinct banks): a product this small is latency-bound,
// so every global load of the block is issued before the first multiply.
__global__ void __launch_bounds__(256) k_gemm_f32(const __grid_constant__ GemmArgs p) {
  dep_wait();
  dep_release();
  if (p.flag && *p.flag == 0) return;
  const int row0 = blockIdx.y * TILE, col0 = blockIdx.x * TILE;
  if (p.lower && row0 + TILE <= col0) return;
  int k_lo = 0, k_hi = p.K;
  if (p.krule == KR_LO_COL) k_lo = col0;
  else if (p.krule == KR_LO_ROW) k_lo = row0;
  else if (p.krule == KR_HI_ROW) k_hi = min(p.K, row0 + TILE);
  else if (p.krule == KR_HI_COL) k_hi = min(p.K, col0 + TILE);
  const int kn = max(k_hi - k_lo, 0), kp = kn + 1;
  extern __shared__ float sm[];
  float* As = sm;              // [TILE][kp]: As[m][k] = op(A)[row0 + m][k_lo + k]
  float* Bs = sm + TILE * kp;  // [TILE][kp]: Bs[n][k] = op(B)[k_lo + k][col0 + n]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // op(A)[m][k] is A[m][k] (k contiguous) or A[k][m]; op(B)[k][n] is B[n][k] or B[k][n]
  if (!p.transA) stage_operand<true>(p.A, p.lda, row0, k_lo, kn, As, kp, warp, lane);
  else stage_operand<false>(p.A, p.lda, row0, k_lo, kn, As, kp, warp, lane);
  if (p.transB) stage_operand<true>(p.B, p.ldb, col0, k_lo, kn, Bs, kp, warp, lane);
  else stage_operand<false>(p.B, p.ldb, col0, k_lo, kn, Bs, kp, warp, lane);
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  constexpr int R = TILE / 16;
  float acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = 0.f;
  const float* a0 = As + ty * kp;
  const float* b0 = Bs + tx * kp;
#pragma unroll 4
  for (int k = 0; k < kn; ++k) {
    float a[R], b[R];
#pragma unroll
    for (int i = 0; i < R; ++i) a[i] = a0[16 * i * kp + k];
#pragma unroll
    for (int j = 0; j < R; ++j) b[j] = b0[16 * j * kp + k];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
  }
  // alpha acc in FP32; a beta != 0 update (the factorisation's trailing updates) is added to
  // the FP64 C in FP64, so the Schur complement loses nothing beyond the product's own error
  // (the C entries are all loaded before the first store, so their latencies overlap)
  const float al = (float)p.alpha;
  double cv[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
      cv[i][j] = (p.beta != 0.0 && !(p.lower && c > r)) ? p.C[(int64_t)r * p.ldc + c] : 0.0;
    }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int r = row0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int c = col0 + tx + 16 * j;
      if (p.lower && c > r) continue;
      const double v = f32_to_f64(al * acc[i][j]);
      p.C[(int64_t)r * p.ldc + c] = p.beta == 0.0 ? v : fma(p.beta, cv[i][j], v);
    }
  }
}

constexpr size_t smem_for(int K) { return (size_t)2 * TILE * (K + 1) * sizeof(float); }
}  // namespace

bool gemm_f32_supported(const GemmArgs& a) {
  return a.M > 0 && a.N > 0 && a.K > 0 && a.M % TILE == 0 && a.N % TILE == 0 && a.K <= KMAX &&
         std::max(a.M, a.N) <= kSmallGemm && a.C != a.A && a.C != a.B;
}

void gemm_f32(const GemmArgs& a, cudaStream_t st) {
  if (!gemm_f32_supported(a)) throw Error(1, "gemm_f32: unsupported shape or in-place product");
  static std::once_flag once;
  std::call_once(once, [] {
    CUDA_CHECK(cudaFuncSetAttribute(k_gemm_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_for(KMAX)));
  });
  launch_dependent(k_gemm_f32, dim3(a.N / TILE, a.M / TILE), 256, smem_for(a.K), st, a);
}

}  // namespace glasso
