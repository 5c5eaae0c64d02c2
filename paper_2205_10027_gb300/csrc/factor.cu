// Recursive blocked Cholesky factorisation that also builds the inverse of its factor, with
// the PD test and log det the line search needs (Sec. 4.3.2, eq. t_cond_pd; the log det of
// eq. sparse_obj), and W = A^{-1} = X^T X from X = L^{-1} (eq. grad_hessian needs W).
//
// Splitting the matrix in halves puts almost all of the work in a few large products
// (K up to np/2), which is what the tensor cores need; the leaves are 64 x 64 blocks that
// one CTA factors and inverts.  Layout: np x np row-major, np a multiple of 128; the factor
// overwrites the lower triangle of A in place, X is written in full (zero upper).
#include <mutex>
#include "factor.h"

namespace glasso {

namespace {
constexpr int NB = kNb;        // 64
constexpr int PT = 256;        // threads of the panel kernel
constexpr int LDS = NB + 1;    // padded shared row

// Factor the 64 x 64 diagonal block at Ablk (leading dimension ld) in place, write the
// inverse of its factor to Xblk (leading dimension ld, zero upper), 2 sum log L_jj to
// *ld_part, and clear *pd on a pivot that is not finite and positive.  T is the arithmetic
// type: double for the FP64 form, float for the split-precision forms (whose products carry
// FP32-level error anyway); storage and the log det are FP64 in both.
template <typename T>
__global__ void __launch_bounds__(PT) k_potrf_diag(double* Ablk, int64_t ld, double* Xblk,
                                                   double* ld_part, int* pd) {
  if (*pd == 0) return;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* a = reinterpret_cast<T*>(sm_raw);  // [NB][LDS]
  T* x = a + NB * LDS;                  // [NB][LDS]
  __shared__ double red[32];
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += PT) {
    const int i = e / NB, c = e % NB;
    a[i * LDS + c] = (c <= i) ? (T)Ablk[(int64_t)i * ld + c] : (T)0;
    x[i * LDS + c] = (T)0;
  }
  __syncthreads();
  bool fail = false;
  for (int j = 0; j < NB; ++j) {
    // every thread reads the same pivot, so the decision is uniform without a flag
    const T d = a[j * LDS + j];
    if (!(d > (T)0) || !isfinite((double)d)) { fail = true; break; }
    const T piv = sqrt(d);
    __syncthreads();  // all reads of a[j][j] before it is overwritten
    if (tid == 0) a[j * LDS + j] = piv;
    for (int i = j + 1 + tid; i < NB; i += PT) a[i * LDS + j] /= piv;
    __syncthreads();
    const int m = NB - j - 1;  // trailing (m x m) lower block
    for (int e = tid; e < m * m; e += PT) {
      const int i = j + 1 + e / m, c = j + 1 + e % m;
      if (c <= i) a[i * LDS + c] -= a[i * LDS + j] * a[c * LDS + j];
    }
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) *pd = 0;
    return;
  }
  // X = L^{-1} row by row: X_ii = 1/L_ii, X_ic = -(sum_{c<=k<i} L_ik X_kc) / L_ii.  Thread t
  // handles column c = t / 4 and every fourth k; the four partial sums meet by shuffles.
  {
    const int c = tid >> 2, part = tid & 3;
    for (int i = 0; i < NB; ++i) {
      T s = (T)0;
      if (c < i)
        for (int k = c + part; k < i; k += 4) s += a[i * LDS + k] * x[k * LDS + c];
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      if (part == 0) {
        if (c == i) x[i * LDS + c] = (T)1 / a[i * LDS + i];
        else if (c < i) x[i * LDS + c] = -s / a[i * LDS + i];
      }
      __syncthreads();
    }
  }
  const double lsum = (tid < NB) ? log((double)a[tid * LDS + tid]) : 0.0;
  const double tot = block_sum(lsum, red);
  for (int e = tid; e < NB * NB; e += PT) {
    const int i = e / NB, c = e % NB;
    Ablk[(int64_t)i * ld + c] = (c <= i) ? (double)a[i * LDS + c] : 0.0;
    Xblk[(int64_t)i * ld + c] = (double)x[i * LDS + c];
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
  bool fp32_leaf;
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
  if (s == NB) {
    double* Ab = c.A + (int64_t)o * c.ld + o;
    double* Xb = c.X + (int64_t)o * c.ld + o;
    if (c.fp32_leaf)
      k_potrf_diag<float><<<1, PT, c.smem, c.st>>>(Ab, c.ld, Xb, c.ld_parts + o / NB, c.pd);
    else
      k_potrf_diag<double><<<1, PT, c.smem, c.st>>>(Ab, c.ld, Xb, c.ld_parts + o / NB, c.pd);
    LAUNCH_CHECK();
    return;
  }
  const int s1 = ((s / NB + 1) / 2) * NB, s2 = s - s1;
  chol_inv_rec(c, o, s1);
  const int64_t ld = c.ld;
  double* A21 = c.A + (int64_t)(o + s1) * ld + o;
  double* A22 = c.A + (int64_t)(o + s1) * ld + o + s1;
  const double* X11 = c.X + (int64_t)o * ld + o;
  const double* X22 = c.X + (int64_t)(o + s1) * ld + o + s1;
  double* X21 = c.X + (int64_t)(o + s1) * ld + o;
  // L21 = A21 X11^T (X11^T upper triangular), through T
  GemmArgs a = gemm_args(A21, ld, 0, X11, ld, 1, c.T, ld, s2, s1, s1, 1.0, 0.0);
  a.krule = KR_HI_COL;
  a.flag = c.pd;
  (*c.gemm)(a, GemmRole::Panel, c.st);
  k_copy_block<<<std::min(s2, 1024), 256, 0, c.st>>>(c.T, A21, ld, s2, s1, c.pd);
  LAUNCH_CHECK();
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
                      double* logdet, const GemmFn& gemm, cudaStream_t st, bool fp32_leaf) {
  const size_t smem = 2 * NB * LDS * (fp32_leaf ? sizeof(float) : sizeof(double));
  static std::once_flag once;  // not repeated inside a stream capture
  std::call_once(once, [] {
    CUDA_CHECK(cudaFuncSetAttribute(k_potrf_diag<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(2 * NB * LDS * sizeof(float))));
    CUDA_CHECK(cudaFuncSetAttribute(k_potrf_diag<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(2 * NB * LDS * sizeof(double))));
  });
  CUDA_CHECK(cudaMemsetAsync(X, 0, sizeof(double) * ld * np, st));
  Ctx c{fp32_leaf, A, X, T, ld, ld_parts, pd, &gemm, st, smem};
  chol_inv_rec(c, 0, np);
  k_sum_parts<<<1, 32, 0, st>>>(ld_parts, np / NB, pd, logdet);
  LAUNCH_CHECK();
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
