// Blocked Cholesky factorisation with PD test and log det (the line-search checks of
// Sec. 4.3.2, eq. t_cond_pd, and the log det of eq. sparse_obj), and W = A^{-1} from the
// factor (eq. grad_hessian needs W): a bottom-up blocked triangular inverse X = L^{-1}
// followed by W = X^T X.
//
// Layout: np x np row-major, np a multiple of 128; the factor overwrites the lower
// triangle in place; the inverses of the 64 x 64 diagonal blocks are kept in a compact
// buffer (np/64 blocks of 64*64) because the triangular inverse starts from them.
#include "factor.h"

namespace glasso {

namespace {
constexpr int NB = kNb;        // 64
constexpr int PT = 256;        // threads of the panel kernel
constexpr int LDS = NB + 1;    // padded shared row

// Factor the 64 x 64 diagonal block at Ablk (leading dimension ld) in place, write the
// inverse of its factor to Dinv (64 x 64, row-major, zero upper), 2 sum log L_jj to
// *ld_part, and clear *pd on a pivot that is not finite and positive.
__global__ void __launch_bounds__(PT) k_potrf_diag(double* Ablk, int64_t ld, double* Dinv,
                                                   double* ld_part, int* pd) {
  if (*pd == 0) return;
  extern __shared__ double sm[];
  double* a = sm;               // [NB][LDS]
  double* x = sm + NB * LDS;    // [NB][LDS]
  __shared__ int fail;
  __shared__ double red[32];
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += PT) {
    const int i = e / NB, c = e % NB;
    a[i * LDS + c] = (c <= i) ? Ablk[(int64_t)i * ld + c] : 0.0;
  }
  if (tid == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < NB; ++j) {
    if (tid == 0) {
      const double d = a[j * LDS + j];
      if (!(d > 0.0) || !isfinite(d)) fail = 1;
      a[j * LDS + j] = sqrt(d);
    }
    __syncthreads();
    if (fail) break;
    const double piv = a[j * LDS + j];
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
  // inverse of the lower-triangular factor, one column per thread (forward substitution)
  if (tid < NB) {
    const int c = tid;
    for (int i = 0; i < c; ++i) x[i * LDS + c] = 0.0;
    x[c * LDS + c] = 1.0 / a[c * LDS + c];
    for (int i = c + 1; i < NB; ++i) {
      double s = 0.0;
      for (int k = c; k < i; ++k) s = fma(a[i * LDS + k], x[k * LDS + c], s);
      x[i * LDS + c] = -s / a[i * LDS + i];
    }
  }
  double lsum = (tid < NB) ? log(a[tid * LDS + tid]) : 0.0;
  const double tot = block_sum(lsum, red);
  __syncthreads();
  for (int e = tid; e < NB * NB; e += PT) {
    const int i = e / NB, c = e % NB;
    Ablk[(int64_t)i * ld + c] = (c <= i) ? a[i * LDS + c] : 0.0;
    Dinv[e] = x[i * LDS + c];
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

// Copy the 64 x 64 diagonal-block inverses into the diagonal blocks of X.
__global__ void k_place_diag(const double* Dinv, double* X, int64_t ld) {
  const int b = blockIdx.x;
  const double* src = Dinv + (int64_t)b * NB * NB;
  double* dst = X + (int64_t)b * NB * ld + (int64_t)b * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) dst[(int64_t)(e / NB) * ld + e % NB] = src[e];
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

void cholesky_f64(double* A, int64_t ld, int np, double* Dinv, double* ld_parts, int* pd,
                  double* logdet, const GemmFn& gemm, cudaStream_t st) {
  const int nblk = np / NB;
  static bool attr_set = false;
  const size_t smem = 2 * NB * LDS * sizeof(double);
  if (!attr_set) {
    CUDA_CHECK(cudaFuncSetAttribute(k_potrf_diag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    attr_set = true;
  }
  for (int k = 0; k < nblk; ++k) {
    const int64_t o = (int64_t)k * NB;
    k_potrf_diag<<<1, PT, smem, st>>>(A + o * ld + o, ld, Dinv + o * NB, ld_parts + k, pd);
    LAUNCH_CHECK();
    const int rem = np - (int)o - NB;
    if (rem <= 0) break;
    double* L21 = A + (o + NB) * ld + o;
    // L21 = A21 * Dinv^T, in place (one tile column covers all 64 columns of the panel)
    GemmArgs t = gemm_args(L21, ld, 0, Dinv + o * NB, NB, 1, L21, ld, rem, NB, NB, 1.0, 0.0);
    t.flag = pd;
    gemm(t, GemmRole::Panel, st);
    // A22 -= L21 L21^T on the lower triangle
    GemmArgs u = gemm_args(L21, ld, 0, L21, ld, 1, A + (o + NB) * ld + o + NB, ld, rem, rem, NB,
                           -1.0, 1.0);
    u.lower = 1;
    u.flag = pd;
    gemm(u, GemmRole::Trailing, st);
  }
  k_sum_parts<<<1, 32, 0, st>>>(ld_parts, nblk, pd, logdet);
  LAUNCH_CHECK();
}

void mirror_lower(double* M, int64_t ld, int np, cudaStream_t st) {
  dim3 grid(np / 32, np / 32);
  k_mirror_lower<<<grid, dim3(32, 8), 0, st>>>(M, ld, np);
  LAUNCH_CHECK();
}

void inverse_from_factor(const double* L, const double* Dinv, int64_t ld, int np, double* X,
                         double* T, double* W, const GemmFn& gemm, cudaStream_t st) {
  CUDA_CHECK(cudaMemsetAsync(X, 0, sizeof(double) * ld * np, st));
  k_place_diag<<<np / NB, 256, 0, st>>>(Dinv, X, ld);
  LAUNCH_CHECK();
  // X = L^{-1}, bottom-up: [[X11, 0], [X21, X22]] with X21 = -X22 L21 X11
  for (int s = NB; s < np; s *= 2) {
    for (int b0 = 0; b0 + s < np; b0 += 2 * s) {
      const int s2 = std::min(s, np - b0 - s);
      const double* L21 = L + (int64_t)(b0 + s) * ld + b0;
      const double* X11 = X + (int64_t)b0 * ld + b0;
      const double* X22 = X + (int64_t)(b0 + s) * ld + b0 + s;
      double* X21 = X + (int64_t)(b0 + s) * ld + b0;
      GemmArgs a = gemm_args(L21, ld, 0, X11, ld, 0, T, ld, s2, s, s, 1.0, 0.0);
      a.krule = KR_LO_COL;
      gemm(a, GemmRole::Inverse, st);
      GemmArgs b = gemm_args(X22, ld, 0, T, ld, 0, X21, ld, s2, s, s2, -1.0, 0.0);
      b.krule = KR_HI_ROW;
      gemm(b, GemmRole::Inverse, st);
    }
  }
  // W = X^T X (lower triangle), then mirrored
  GemmArgs w = gemm_args(X, ld, 1, X, ld, 0, W, ld, np, np, np, 1.0, 0.0);
  w.lower = 1;
  w.krule = KR_LO_ROW;
  gemm(w, GemmRole::Inverse, st);
  mirror_lower(W, ld, np, st);
}

}  // namespace glasso
