// Recursive blocked Cholesky factorisation that also builds the inverse of its factor, with
// the PD test and log det the line search needs (Sec. 4.3.2, eq. t_cond_pd; the log det of
// eq. sparse_obj), and W = A^{-1} = X^T X from X = L^{-1} (eq. grad_hessian needs W).
//
// Splitting the matrix in halves puts almost all of the work in a few large products
// (K up to np/2), which is what the tensor cores need; the leaves are 64 x 64 (FP64) or
// 128 x 128 (FP32, split-precision modes) blocks that one CTA factors and inverts.  Layout: np x np row-major, np a multiple of 128; the factor
// overwrites the lower triangle of A in place, X is written in full (zero upper).
#include <mutex>
#include "factor.h"

namespace glasso {

namespace {
constexpr int NB = kNb;        // leaf size of the FP64 form (64)
constexpr int NB32 = 128;      // leaf size of the split-precision forms (FP32 leaves)

// Factor the NB x NB diagonal block at Ablk (leading dimension ld) in place, write the
// inverse of its factor to Xblk (leading dimension ld, zero upper), 2 sum log L_jj to
// *ld_part, and clear *pd on a pivot that is not finite and positive.  T is the arithmetic
// type: double for the FP64 form, float for the split-precision forms (whose products carry
// FP32-level error anyway); storage and the log det are FP64 in both.
//
// Blocked by 32 columns so that barriers are few: warp 0 factors each 32 x 32 diagonal block
// with one row per lane in registers (pivots and columns travel by shuffles), then the rows
// below solve against it one row per thread, and all warps apply the rank-32 update.  The
// inverse inverts the diagonal 32 x 32 blocks one warp each (one column per lane), then fills
// the block rows below: X_ij = -X_ii (sum_{j<=k<i} L_ik X_kj).
template <typename T, int NB, int PT>
__global__ void __launch_bounds__(PT) k_potrf_diag(double* Ablk, int64_t ld, double* Xblk,
                                                   double* ld_part, int* pd) {
  constexpr int LDS = NB + 1;  // padded shared row
  constexpr int P = NB / 32;   // 32-column panels
  constexpr int NW = PT / 32;
  static_assert(NB % 32 == 0 && NW >= P, "one warp per diagonal block in the inverse");
  if (*pd == 0) return;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* a = reinterpret_cast<T*>(sm_raw);  // [NB][LDS]
  T* x = a + NB * LDS;                  // [NB][LDS]
  __shared__ double red[32];
  __shared__ int fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < NB * NB; e += PT) {
    const int i = e / NB, c = e % NB;
    a[i * LDS + c] = (c <= i) ? from_f64<T>(Ablk[(int64_t)i * ld + c]) : (T)0;
    x[i * LDS + c] = (T)0;
  }
  if (tid == 0) fail = 0;
  __syncthreads();

  for (int p = 0; p < P; ++p) {
    const int o = 32 * p;
    // (1) 32 x 32 diagonal block, lane r holding row o + r
    if (warp == 0) {
      T row[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) row[c] = (c <= lane) ? a[(o + lane) * LDS + o + c] : (T)0;
      bool bad = false;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const T d = __shfl_sync(0xffffffffu, row[j], j);
        if (!(d > (T)0) || !isfinite(d)) bad = true;
        const T piv = sqrt(d);
        if (lane == j) row[j] = piv;
        if (lane > j) row[j] = row[j] / piv;
#pragma unroll
        for (int c = j + 1; c < 32; ++c) {
          const T lcj = __shfl_sync(0xffffffffu, row[j], c);
          if (lane >= c) row[c] -= row[j] * lcj;
        }
      }
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c <= lane) a[(o + lane) * LDS + o + c] = row[c];
      if (lane == 0 && bad) fail = 1;
    }
    __syncthreads();
    if (fail) break;
    // (2) rows below: l_i = a_i L_pp^{-T}, one row per thread (forward substitution)
    for (int i = o + 32 + tid; i < NB; i += PT) {
      T* ri = a + i * LDS + o;
      for (int j = 0; j < 32; ++j) {
        const T* lj = a + (o + j) * LDS + o;
        T s = ri[j];
        for (int k = 0; k < j; ++k) s -= ri[k] * lj[k];
        ri[j] = s / lj[j];
      }
    }
    __syncthreads();
    // (3) rank-32 update of the trailing lower triangle; warp w takes rows o+32+w, +NW, ...
    for (int i = o + 32 + warp; i < NB; i += NW) {
      const T* ri = a + i * LDS + o;
      for (int c = o + 32 + lane; c <= i; c += 32) {
        const T* rc = a + c * LDS + o;
        T s = (T)0;
#pragma unroll 8
        for (int k = 0; k < 32; ++k) s += ri[k] * rc[k];
        a[i * LDS + c] -= s;
      }
    }
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) *pd = 0;
    return;
  }
  // inverse: diagonal blocks, one warp each, one column per lane
  if (warp < P) {
    const int o = 32 * warp, c = lane;
    for (int r = 0; r < 32; ++r) {
      if (r < c) continue;
      T s = (r == c) ? (T)1 : (T)0;
      for (int k = c; k < r; ++k) s -= a[(o + r) * LDS + o + k] * x[(o + k) * LDS + o + c];
      x[(o + r) * LDS + o + c] = s / a[(o + r) * LDS + o + r];
    }
  }
  __syncthreads();
  // block rows below: X_ij = -X_ii (sum_{j<=k<i} L_ik X_kj) for j < i, through the upper
  // (unused) half of a as scratch is not safe; use x's own block (i, j) for the sum first
  for (int bi = 1; bi < P; ++bi) {
    // S_ij = sum_k L_ik X_kj into x block (bi, j) for all j < bi
    for (int e = tid; e < bi * 32 * 32; e += PT) {
      const int j = e / 1024, r = (e / 32) % 32, c = e % 32;
      const int gi = 32 * bi + r, gj = 32 * j + c;
      T s = (T)0;
      for (int k = 32 * j; k < 32 * bi; ++k) s += a[gi * LDS + k] * x[k * LDS + gj];
      x[gi * LDS + gj] = s;
    }
    __syncthreads();
    // X_ij = -X_ii S_ij, computed into registers first (S is overwritten in place)
    T v[(NB * 32 + PT - 1) / PT];
    int cnt = 0;
    for (int e = tid; e < bi * 32 * 32; e += PT, ++cnt) {
      const int j = e / 1024, r = (e / 32) % 32, c = e % 32;
      const int gi = 32 * bi + r, gj = 32 * j + c;
      T s = (T)0;
      for (int k = 0; k <= r; ++k) s += x[gi * LDS + 32 * bi + k] * x[(32 * bi + k) * LDS + gj];
      v[cnt] = -s;
    }
    __syncthreads();
    cnt = 0;
    for (int e = tid; e < bi * 32 * 32; e += PT, ++cnt) {
      const int j = e / 1024, r = (e / 32) % 32, c = e % 32;
      x[(32 * bi + r) * LDS + 32 * j + c] = v[cnt];
    }
    __syncthreads();
  }
  const double lsum = (tid < NB) ? log((double)a[tid * LDS + tid]) : 0.0;
  const double tot = block_sum(lsum, red);
  for (int e = tid; e < NB * NB; e += PT) {
    const int i = e / NB, c = e % NB;
    Ablk[(int64_t)i * ld + c] = (c <= i) ? to_f64(a[i * LDS + c]) : 0.0;
    Xblk[(int64_t)i * ld + c] = to_f64(x[i * LDS + c]);
  }
  if (tid == 0) *ld_part = 2.0 * tot;
}

// out = sum of parts[0..n) in index order (one thread: n is at most a few hundred).
__global__ void k_sum_parts(const double* parts, int n, const int* pd, double* out) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += parts[i];
  *out = (*pd) ? s : NAN;
}

// dst[rows x cols] := src[rows x cols] (both with leading dimension ld), unless *flag == 0.
__global__ void k_copy_block(const double* __restrict__ src, double* __restrict__ dst, int64_t ld,
                             int rows, int cols, const int* flag) {
  if (*flag == 0) return;
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
    for (int c = threadIdx.x; c < cols; c += blockDim.x) dst[r * ld + c] = src[r * ld + c];
}

// Upper triangle of M := transpose of its lower triangle (32 x 32 tiles through shared).
__global__ void k_mirror_lower(double* M, int64_t ld, int np) {
  __shared__ double t[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;  // source tile (bi, bj) with bi > bj is lower
  if (bi < bj) return;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) t[r][tx] = M[(int64_t)(bi * 32 + r) * ld + bj * 32 + tx];
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int gi = bj * 32 + r, gj = bi * 32 + tx;  // destination (upper) entry
    if (gj > gi) M[(int64_t)gi * ld + gj] = t[tx][r];
  }
}
}  // namespace

namespace {
struct Ctx {
  bool fp32_leaf;  // split-precision modes: FP32 leaves of NB32 rows, in-place panel products
  int leaf;
  double* A;
  double* X;
  double* T;
  int64_t ld;
  double* ld_parts;
  int* pd;
  const GemmFn* gemm;
  cudaStream_t st;
  size_t smem;
};

// Factor the diagonal block [o, o + s) of A in place and write X = L^{-1} there:
//   L11 X11 from the first half; L21 = A21 X11^T; A22 -= L21 L21^T; L22 X22 from the second
//   half; X21 = -X22 (L21 X11).
void chol_inv_rec(const Ctx& c, int o, int s) {
  if (s == c.leaf) {
    double* Ab = c.A + (int64_t)o * c.ld + o;
    double* Xb = c.X + (int64_t)o * c.ld + o;
    if (c.fp32_leaf)
      k_potrf_diag<float, NB32, 4 * NB32><<<1, 4 * NB32, c.smem, c.st>>>(Ab, c.ld, Xb, c.ld_parts + o / c.leaf, c.pd);
    else
      k_potrf_diag<double, NB, 4 * NB><<<1, 4 * NB, c.smem, c.st>>>(Ab, c.ld, Xb, c.ld_parts + o / c.leaf, c.pd);
    LAUNCH_CHECK();
    return;
  }
  const int s1 = ((s / c.leaf + 1) / 2) * c.leaf, s2 = s - s1;
  chol_inv_rec(c, o, s1);
  const int64_t ld = c.ld;
  double* A21 = c.A + (int64_t)(o + s1) * ld + o;
  double* A22 = c.A + (int64_t)(o + s1) * ld + o + s1;
  const double* X11 = c.X + (int64_t)o * ld + o;
  const double* X22 = c.X + (int64_t)(o + s1) * ld + o + s1;
  double* X21 = c.X + (int64_t)(o + s1) * ld + o;
  // L21 = A21 X11^T (X11^T upper triangular).  The tensor-core product reads its operands
  // from the split copies made before it starts, so it may overwrite A21 in place; the FP64
  // kernel reads A21 tile by tile and goes through T.
  GemmArgs a = gemm_args(A21, ld, 0, X11, ld, 1, c.fp32_leaf ? A21 : c.T, ld, s2, s1, s1, 1.0, 0.0);
  a.krule = KR_HI_COL;
  a.flag = c.pd;
  (*c.gemm)(a, GemmRole::Panel, c.st);
  if (!c.fp32_leaf) {
    k_copy_block<<<std::min(s2, 1024), 256, 0, c.st>>>(c.T, A21, ld, s2, s1, c.pd);
    LAUNCH_CHECK();
  }
  // A22 -= L21 L21^T on the lower triangle
  GemmArgs b = gemm_args(A21, ld, 0, A21, ld, 1, A22, ld, s2, s2, s1, -1.0, 1.0);
  b.lower = 1;
  b.flag = c.pd;
  (*c.gemm)(b, GemmRole::Trailing, c.st);
  chol_inv_rec(c, o + s1, s2);
  // X21 = -X22 (L21 X11)
  GemmArgs d = gemm_args(A21, ld, 0, X11, ld, 0, c.T, ld, s2, s1, s1, 1.0, 0.0);
  d.krule = KR_LO_COL;
  d.flag = c.pd;
  (*c.gemm)(d, GemmRole::Inverse, c.st);
  GemmArgs e = gemm_args(X22, ld, 0, c.T, ld, 0, X21, ld, s2, s1, s2, -1.0, 0.0);
  e.krule = KR_HI_ROW;
  e.flag = c.pd;
  (*c.gemm)(e, GemmRole::Inverse, c.st);
}
}  // namespace

void cholesky_inverse(double* A, double* X, int64_t ld, int np, double* T, double* ld_parts, int* pd,
                      double* logdet, const GemmFn& gemm, cudaStream_t st, bool fp32_leaf, int panel) {
  const int leaf = fp32_leaf ? NB32 : NB;
  const size_t smem = 2 * (size_t)leaf * (leaf + 1) * (fp32_leaf ? sizeof(float) : sizeof(double));
  static std::once_flag once;  // not repeated inside a stream capture
  std::call_once(once, [] {
    CUDA_CHECK(cudaFuncSetAttribute(k_potrf_diag<float, NB32, 4 * NB32>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(2 * NB32 * (NB32 + 1) * sizeof(float))));
    CUDA_CHECK(cudaFuncSetAttribute(k_potrf_diag<double, NB, 4 * NB>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(2 * NB * (NB + 1) * sizeof(double))));
  });
  CUDA_CHECK(cudaMemsetAsync(X, 0, sizeof(double) * ld * np, st));
  Ctx c{fp32_leaf, leaf, A, X, T, ld, ld_parts, pd, &gemm, st, smem};
  if (panel <= 0) {
    chol_inv_rec(c, 0, np);
  } else {
    // right-looking over panels of `panel` columns: each diagonal block is factored (and
    // inverted) recursively, then L21 = A21 X_kk^T and A22 -= L21 L21^T are single large
    // products; the off-diagonal blocks of X are left to inverse_merge
    for (int o = 0; o < np; o += panel) {
      const int s = std::min(panel, np - o);
      chol_inv_rec(c, o, s);
      const int rem = np - o - s;
      if (rem <= 0) break;
      double* A21 = A + (int64_t)(o + s) * ld + o;
      double* A22 = A + (int64_t)(o + s) * ld + o + s;
      const double* Xkk = X + (int64_t)o * ld + o;
      GemmArgs a = gemm_args(A21, ld, 0, Xkk, ld, 1, fp32_leaf ? A21 : T, ld, rem, s, s, 1.0, 0.0);
      a.krule = KR_HI_COL;
      a.flag = pd;
      gemm(a, GemmRole::Panel, st);
      if (!fp32_leaf) {
        k_copy_block<<<std::min(rem, 1024), 256, 0, st>>>(T, A21, ld, rem, s, pd);
        LAUNCH_CHECK();
      }
      GemmArgs b = gemm_args(A21, ld, 0, A21, ld, 1, A22, ld, rem, rem, s, -1.0, 1.0);
      b.lower = 1;
      b.flag = pd;
      gemm(b, GemmRole::Trailing, st);
    }
  }
  k_sum_parts<<<1, 32, 0, st>>>(ld_parts, np / leaf, pd, logdet);
  LAUNCH_CHECK();
}

void inverse_merge(const double* L, double* X, int64_t ld, int np, double* T, int panel, const GemmFn& gemm,
                   cudaStream_t st) {
  // X = L^{-1} from its diagonal panel blocks, bottom-up: [[X11, 0], [X21, X22]] with
  // X21 = -X22 (L21 X11)
  for (int w = panel; w < np; w *= 2) {
    for (int b0 = 0; b0 + w < np; b0 += 2 * w) {
      const int s2 = std::min(w, np - b0 - w);
      const double* L21 = L + (int64_t)(b0 + w) * ld + b0;
      const double* X11 = X + (int64_t)b0 * ld + b0;
      const double* X22 = X + (int64_t)(b0 + w) * ld + b0 + w;
      double* X21 = X + (int64_t)(b0 + w) * ld + b0;
      GemmArgs a = gemm_args(L21, ld, 0, X11, ld, 0, T, ld, s2, w, w, 1.0, 0.0);
      a.krule = KR_LO_COL;
      gemm(a, GemmRole::Inverse, st);
      GemmArgs b = gemm_args(X22, ld, 0, T, ld, 0, X21, ld, s2, w, s2, -1.0, 0.0);
      b.krule = KR_HI_ROW;
      gemm(b, GemmRole::Inverse, st);
    }
  }
}

void mirror_lower(double* M, int64_t ld, int np, cudaStream_t st) {
  dim3 grid(np / 32, np / 32);
  k_mirror_lower<<<grid, dim3(32, 8), 0, st>>>(M, ld, np);
  LAUNCH_CHECK();
}

void inverse_from_inverse_factor(const double* X, int64_t ld, int np, double* W, const GemmFn& gemm,
                                 cudaStream_t st) {
  // W = X^T X (lower triangle), then mirrored
  GemmArgs w = gemm_args(X, ld, 1, X, ld, 0, W, ld, np, np, np, 1.0, 0.0);
  w.lower = 1;
  w.krule = KR_LO_ROW;
  gemm(w, GemmRole::Inverse, st);
  mirror_lower(W, ld, np, st);
}

}  // namespace glasso
