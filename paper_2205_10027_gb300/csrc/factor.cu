// Recursive blocked Cholesky factorisation that also builds the inverse of its factor, with
// the PD test and log det the line search needs (Sec. 4.3.2, eq. t_cond_pd; the log det of
// eq. sparse_obj), and W = A^{-1} = X^T X from X = L^{-1} (eq. grad_hessian needs W).
//
// Splitting the matrix in halves puts almost all of the work in a few large products
// (K up to np/2), which is what the tensor cores need; the leaves are diagonal blocks that one
// CTA factors and inverts: 64 x 64 in FP64 (the FP64 form), 64 x 64 with an FP64 Cholesky and
// an FP32 inverse (the split-precision forms), or, as an option of the split-precision forms,
// 128 x 128 in FP32.  Layout: np x np row-major, np a multiple of 128; the factor overwrites
// the lower triangle of A in place, X is written in full (zero upper).
#include <mutex>
#include "factor.h"

namespace glasso {

namespace {
constexpr int NB = kNb;        // leaf size of the FP64 form (64)
constexpr int NB32 = 128;      // leaf size of the split-precision forms

// Factor the NB x NB diagonal block at Ablk (leading dimension ld) in place, write the
// inverse of its factor to the lower triangle of Xblk (leading dimension ld; the caller has
// zeroed X), 2 sum log L_jj to *ld_part, and clear *pd on a pivot that is not finite and
// positive.  T is the arithmetic type: double for the FP64 form, float for the
// split-precision forms (whose products carry FP32-level error anyway); storage and the log
// det are FP64 in both.
//
// One CTA, blocked by 32-column panels p, two barriers per panel:
//  (1) warp 0 factors the 32 x 32 diagonal block L_pp, one row per lane in registers, and in
//      the same sweep applies the inverse elementary column transforms to an identity held
//      the same way, which leaves X_pp = L_pp^{-1};
//  (2) all warps: the rows below, L_ip = A_ip X_pp^T (dot products of length 32), and the
//      first half of block row p of X, T_pj = sum_{j<=k<p} L_pk X_kj (into the unused upper
//      triangle of the block);
//  (3) all warps: the rank-32 update of the trailing lower triangle, and X_pj = -X_pp T_pj.
// Work items are 8 rows x 32 columns (one column per lane), so each shared-memory load of a
// row segment is a 16-byte broadcast reused by the 8 accumulators of a lane.
template <typename T>
__device__ __forceinline__ void lds4(const T* p, T& v0, T& v1, T& v2, T& v3);
template <>
__device__ __forceinline__ void lds4<float>(const float* p, float& v0, float& v1, float& v2, float& v3) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v0 = q.x; v1 = q.y; v2 = q.z; v3 = q.w;
}
template <>
__device__ __forceinline__ void lds4<double>(const double* p, double& v0, double& v1, double& v2, double& v3) {
  const double2 q0 = reinterpret_cast<const double2*>(p)[0];
  const double2 q1 = reinterpret_cast<const double2*>(p)[1];
  v0 = q0.x; v1 = q0.y; v2 = q1.x; v3 = q1.y;
}
__device__ __forceinline__ float rsqrt_t(float v) { return rsqrtf(v); }
__device__ __forceinline__ double rsqrt_t(double v) { return rsqrt(v); }

// acc[q] += sum_{k in [k0, k1)} R[(r0 + q) * LDS + k] * c[k]  for q < 8, with c[k] supplied
// by the caller as a per-lane register row (k relative to 0) or a strided shared column.
template <typename T, int LDS>
__device__ __forceinline__ void rows8_times_regs(const T* R, int r0, int koff, const T (&c)[32], T (&acc)[8]) {
#pragma unroll
  for (int k = 0; k < 32; k += 4) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      T v0, v1, v2, v3;
      lds4(R + (r0 + q) * LDS + koff + k, v0, v1, v2, v3);
      acc[q] = fma(v0, c[k], acc[q]);
      acc[q] = fma(v1, c[k + 1], acc[q]);
      acc[q] = fma(v2, c[k + 2], acc[q]);
      acc[q] = fma(v3, c[k + 3], acc[q]);
    }
  }
}

// Step J of the 32 x 32 diagonal-block sweep in one warp (lane l holds row l of the block
// in r and row l of the running inverse in xr): pivot d = L_JJ^2, column J of L, the inverse
// elementary transform E_J^{-1} on xr, and the right-looking update of columns > J.  Written
// as a template recursion so that every register index is a compile-time constant.
// Entries of r above the diagonal (r[c], c > lane) are scratch: they take updates that are
// never read back, which keeps every update a plain multiply-add (no per-lane predicate).
template <typename T, int J>
__device__ __forceinline__ void diag_steps(T (&r)[32], T (&xr)[32], int lane, bool& bad) {
  if constexpr (J < 32) {
    constexpr unsigned FULL = 0xffffffffu;
    const T d = __shfl_sync(FULL, r[J], J);  // pivot after the updates of columns < J
    bad |= !(d > T(0)) || isinf(d);
    const T s = rsqrt_t(d);  // 1 / L_JJ
    r[J] = (lane == J) ? d * s : r[J] * s;  // column J of L (valid for lanes >= J)
    // xr <- E_J^{-1} xr: row J scaled by 1 / L_JJ, rows below minus L_iJ (row J)
    const T sj = (lane == J) ? s : T(1);
#pragma unroll
    for (int c = 0; c <= J; ++c) xr[c] *= sj;
    const T m = (lane > J) ? -r[J] : T(0);
#pragma unroll
    for (int c = 0; c <= J; ++c) xr[c] = fma(m, __shfl_sync(FULL, xr[c], J), xr[c]);
    // right-looking update of columns > J (rows >= c are the valid ones)
    const T mr = -r[J];
#pragma unroll
    for (int c = J + 1; c < 32; ++c) r[c] = fma(mr, __shfl_sync(FULL, r[J], c), r[c]);
    diag_steps<T, J + 1>(r, xr, lane, bad);
  }
}

template <typename T, int NB, int PT>
__global__ void __launch_bounds__(PT) k_leaf_chol_inv(double* Ablk, int64_t ld, double* Xblk,
                                                      double* ld_part, int* pd) {
  constexpr int LDS = NB + 4;  // row pitch: rows start on 16-byte boundaries
  constexpr int P = NB / 32;
  constexpr int NW = PT / 32;
  constexpr unsigned FULL = 0xffffffffu;
  static_assert(NB % 32 == 0 && PT % 32 == 0, "shape");
  dep_wait();
  dep_release();
  if (*pd == 0) return;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* a = reinterpret_cast<T*>(sm_raw);  // [NB][LDS]: L (lower); T_pj scratch above the diagonal
  T* x = a + NB * LDS;                  // [NB][LDS]: X = L^{-1} (lower, zero above)
  __shared__ double red[32];
  __shared__ int fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  {
    // every thread issues all of its loads (lower triangle only) before converting any
    constexpr int PER = NB * NB / PT, BATCH = PER < 16 ? PER : 16;
    static_assert(NB * NB % PT == 0 && PER % BATCH == 0, "load split");
#pragma unroll
    for (int u0 = 0; u0 < PER; u0 += BATCH) {
      double v[BATCH];
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        const int e = tid + (u0 + u) * PT, i = e / NB, c = e % NB;
        v[u] = (c <= i) ? Ablk[(int64_t)i * ld + c] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        const int e = tid + (u0 + u) * PT, i = e / NB, c = e % NB;
        a[i * LDS + c] = from_f64<T>(v[u]);
        x[i * LDS + c] = T(0);
      }
    }
  }
  if (tid == 0) fail = 0;
  __syncthreads();

  for (int p = 0; p < P; ++p) {
    const int o = 32 * p;
    const int m = NB - o - 32;  // trailing rows
    // ---- (1) L_pp and X_pp in warp 0
    if (warp == 0) {
      T r[32], xr[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        r[c] = (c <= lane) ? a[(o + lane) * LDS + o + c] : T(0);
        xr[c] = (c == lane) ? T(1) : T(0);
      }
      bool bad = false;
      diag_steps<T, 0>(r, xr, lane, bad);
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        if (c <= lane) {
          a[(o + lane) * LDS + o + c] = r[c];
          x[(o + lane) * LDS + o + c] = xr[c];
        }
      }
      if (__any_sync(FULL, bad) && lane == 0) fail = 1;
    }
    __syncthreads();
    if (fail) break;
    // ---- (2) rows below: L_ip = A_ip X_pp^T;  T_pj = sum_{j<=k<p} L_pk X_kj
    {
      const int n_rows = m / 8, n_t = 4 * p;
      for (int t = warp; t < n_rows + n_t; t += NW) {
        T acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = T(0);
        if (t < n_rows) {
          T xrow[32];  // row `lane` of X_pp
#pragma unroll
          for (int k = 0; k < 32; k += 4)
            lds4(x + (o + lane) * LDS + o + k, xrow[k], xrow[k + 1], xrow[k + 2], xrow[k + 3]);
          const int r0 = o + 32 + 8 * t;
          rows8_times_regs<T, LDS>(a, r0, o, xrow, acc);
          __syncwarp();
#pragma unroll
          for (int q = 0; q < 8; ++q) a[(r0 + q) * LDS + o + lane] = acc[q];
        } else {
          const int u = t - n_rows, j = u / 4, r0 = 8 * (u % 4);
          // rows o + r0 .. + 7 of L against column 32 j + lane of X, k over [32 j, o)
          for (int k0 = 32 * j; k0 < o; k0 += 32) {
            T col[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) col[k] = x[(k0 + k) * LDS + 32 * j + lane];
            rows8_times_regs<T, LDS>(a, o + r0, k0, col, acc);
          }
#pragma unroll
          for (int q = 0; q < 8; ++q) a[(32 * j + r0 + q) * LDS + o + lane] = acc[q];
        }
      }
    }
    __syncthreads();
    // ---- (3) trailing update A_ic -= sum_k L_ik L_ck (o+32 <= c <= i);  X_pj = -X_pp T_pj
    {
      int n_upd = 0;
      for (int q = 0; q < m / 32; ++q) n_upd += (m - 32 * q) / 8;
      const int n_x = 4 * p;
      for (int t = warp; t < n_upd + n_x; t += NW) {
        T acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = T(0);
        if (t < n_upd) {
          int chunk = 0, rem = t;
          while (rem >= (m - 32 * chunk) / 8) { rem -= (m - 32 * chunk) / 8; ++chunk; }
          const int c = o + 32 + 32 * chunk + lane;
          const int r0 = o + 32 + 32 * chunk + 8 * rem;
          T lc[32];  // row c of the panel: L_c,o..o+31
#pragma unroll
          for (int k = 0; k < 32; k += 4) lds4(a + c * LDS + o + k, lc[k], lc[k + 1], lc[k + 2], lc[k + 3]);
          rows8_times_regs<T, LDS>(a, r0, o, lc, acc);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (c <= r0 + q) a[(r0 + q) * LDS + c] -= acc[q];
        } else {
          const int u = t - n_upd, j = u / 4, r0 = 8 * (u % 4);
          T col[32];  // column 32 j + lane of T_pj (stored at rows 32 j.., columns o..)
#pragma unroll
          for (int k = 0; k < 32; ++k) col[k] = a[(32 * j + k) * LDS + o + lane];
          rows8_times_regs<T, LDS>(x, o + r0, o, col, acc);  // X_pp is zero above its diagonal
#pragma unroll
          for (int q = 0; q < 8; ++q) x[(o + r0 + q) * LDS + 32 * j + lane] = -acc[q];
        }
      }
    }
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) *pd = 0;
    return;
  }
  const double lsum = (tid < NB) ? log(to_f64(a[tid * LDS + tid])) : 0.0;
  const double tot = block_sum(lsum, red);
  for (int e = tid; e < NB * NB; e += PT) {
    const int i = e / NB, c = e % NB;
    Ablk[(int64_t)i * ld + c] = (c <= i) ? to_f64(a[i * LDS + c]) : 0.0;
    if (c <= i) Xblk[(int64_t)i * ld + c] = to_f64(x[i * LDS + c]);
  }
  if (tid == 0) *ld_part = 2.0 * tot;
}

// dynamic shared memory of k_leaf_chol_inv: two NB x (NB + 4) arrays
constexpr size_t leaf_smem(int nb, size_t elt) { return 2 * (size_t)nb * (nb + 4) * elt; }

// ---- 128 x 128 leaf of the split-precision forms: FP64 Cholesky panels, FP32 inverse ----
// The diagonal block is factored as two 64 x 64 FP64 Cholesky panels (the pivots, the PD test
// and the log det are FP64 arithmetic on the FP64 Schur complement) joined inside the CTA by
// the block's own small products: L21 = A21 X11^T and X21 = -X22 (L21 X11) in FP32 (the
// accuracy of the split-precision products they stand beside), and the trailing update
// A22 -= L21 L21^T formed in FP32 and subtracted from the FP64 A22 in FP64.  The inverse
// X = L^{-1}, which only feeds split-precision products, is formed in FP32.
//
// On this part the FP64 pipe issues one warp instruction per 64 cycles per sub-partition and
// an FP64 divide takes ~430 cycles, so each FP64 panel keeps its serial chain short: the
// right-looking update is kept unscaled (a_ic -= a_ij a_cj / d_j, L recovered at the end as
// a_ij / sqrt(d_j)), one lane of warp 0 runs the pivot chain d_{j+1} = a_{j+1,j+1} -
// a_{j+1,j}^2 / d_j one column ahead, and the six warps on the other three sub-partitions
// apply the update of column j to the rest of the trailing triangle meanwhile.
constexpr int L64 = 64, L64P = 65;     // panel size, FP64 row pitch (odd: conflict-free columns)
constexpr int F64P = 68;               // FP32 row pitch: rows 16-byte aligned for float4 loads
constexpr int LEAF128_THREADS = 256;
constexpr size_t leaf128_smem() {
  return 3 * (size_t)L64 * L64P * sizeof(double) + 5 * (size_t)L64 * F64P * sizeof(float);
}

// 1 / d in FP64 for a pivot d > 0: the PTX approximate reciprocal y (relative error e0 well
// below 2^-16), refined by one step of the third-order iteration for the reciprocal,
// e = 1 - d y, y <- y (1 + e + e^2) (the error becomes O(e0^3), below FP64 rounding): three
// dependent FP64 operations, where two Newton steps take four and a correctly rounded divide
// longer still.  On this part each dependent FP64 operation costs ~64 cycles, and the pivot
// chain is the leaf's critical path.
// A pivot is usable when it is a positive finite number: tested on the bit pattern with
// integer operations, which keeps FP64 compares (one FP64 instruction each) off the chain.
__device__ __forceinline__ bool pivot_ok(double d) {
  const long long b = __double_as_longlong(d);
  return b > 0 && ((b >> 52) & 0x7FF) != 0x7FF;  // sign clear, not +0, not Inf or NaN
}

// The divide for pivots outside [2^-960, 2^960], kept out of line so that the compiler cannot
// evaluate it speculatively on the chain (a divide is a long sequence of FP64 operations).
__device__ __noinline__ double pivot_reciprocal_slow(double d) { return 1.0 / d; }

__device__ __forceinline__ double pivot_reciprocal(double d) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
  const double e = fma(-d, y, 1.0);
  double r = fma(y, fma(e, e, e), y);
  // the range test on the exponent field runs on the integer pipe alongside the FP64
  // operations instead of before them
  const int ex = (int)((__double_as_longlong(d) >> 52) & 0x7FF);
  if (ex < 63 || ex > 1983) r = pivot_reciprocal_slow(d);
  return r;
}

// The lower triangle of a 64 x 64 block in column-major order, (i, c) packed as i | c << 8:
// the entries of columns > j are the suffix starting at col_start(j + 1).  k_leaf128 copies
// the list into shared memory (lanes read consecutive entries).
constexpr int kTri64N = L64 * (L64 + 1) / 2;
__device__ uint16_t g_tri64[kTri64N];
__device__ __forceinline__ int col_start(int c) { return c * L64 - c * (c - 1) / 2; }

// FP64 Cholesky of the 64 x 64 lower triangle in a (pitch L64P), all 256 threads.  On return a
// holds L (lower), piv[j] = L_jj^2, and *fail != 0 on a pivot that is not finite and positive.
// inv and tcol are 64-entry shared scratch, tri the column-major list of the triangle, fs a
// 64 x 33 FP32 shared scratch.
//
// The panel is factored as four 16-column micro-panels.  Inside a micro-panel the update is
// FP64 and right-looking, kept unscaled (a_ic -= a_ij a_cj / d_j; L is a_ij / sqrt(d_j) at the
// end): step j, one lane of warp 0 forms the next pivot d_{j+1} = a_{j+1,j+1} - a_{j+1,j}^2 / d_j
// (the chain) while the six warps on the other sub-partitions update the micro-panel's
// remaining columns, all rows, as a flat list so that each FP64 instruction runs 32 lanes.  A
// finished micro-panel's contribution to the columns right of it is one FP32 product
// (l_ik = a_ik / d_k times a_ck, 16 terms) subtracted from the FP64 entries in FP64, the way
// the recursion above applies its trailing updates; so every pivot is FP64 arithmetic on an
// FP64 Schur complement, and the FP64 pipe (one warp instruction per 64 cycles per
// sub-partition here) carries only the micro-panels' own updates.
constexpr int kMicro = 16;
__device__ void chol64_f64(double* a, double* piv, double* inv, double* tcol, const uint16_t* tri, float* fs,
                           int* fail) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // update warps: the six on sub-partitions 1-3 (warp w runs on w % 4); warp 0 runs the chain
  const int uw = warp == 1 ? 0 : warp == 2 ? 1 : warp == 3 ? 2 : warp == 5 ? 3 : warp == 6 ? 4 : warp == 7 ? 5 : -1;
  double rinv = 0.0;  // thread 0: 1 / d of the last pivot (the chain keeps it in a register)
  for (int c0 = 0; c0 < L64; c0 += kMicro) {
    const int c1 = c0 + kMicro;  // the micro-panel is columns [c0, c1)
    // its first pivot: every contribution of the columns left of it is in place
    if (tid == 0) {
      const double d = a[c0 * L64P + c0];
      if (!pivot_ok(d)) *fail = 1;
      piv[c0] = d;
      rinv = pivot_reciprocal(d);
      inv[c0] = rinv;
    }
    __syncthreads();
    for (int j = c0; j < c1; ++j) {
      if (tid == 0 && j + 1 < c1) {
        // the pivot chain, one column ahead
        const double aj = a[(j + 1) * L64P + j];
        const double d = fma(-aj * rinv, aj, a[(j + 1) * L64P + j + 1]);
        if (!pivot_ok(d)) *fail = 1;
        rinv = pivot_reciprocal(d);
        a[(j + 1) * L64P + j + 1] = d;
        piv[j + 1] = d;
        inv[j + 1] = rinv;
      } else if (uw >= 0 && j + 1 < c1) {
        // t_i = a_ij / d_j for the rows below, then a_ic -= t_i a_cj over the micro-panel's
        // columns > j, all rows, except the diagonal (j+1, j+1) that the chain has updated
        if (uw < 2) {
          const int i = j + 1 + 32 * uw + lane;
          if (i < L64) tcol[i] = a[i * L64P + j] * inv[j];
        }
        asm volatile("bar.sync 1, 192;" ::: "memory");
        // two entries per lane per pass, all loads issued before the FP64 operations (the
        // entries are distinct and column j is read-only in this step)
        constexpr int span = 192;
        const int e0 = col_start(j + 1) + 1, e1 = col_start(c1);
        for (int e = e0 + 32 * uw + lane; e < e1; e += 2 * span) {
          const int e2 = e + span;
          const uint16_t p0 = tri[e], p1 = e2 < e1 ? tri[e2] : tri[e];
          const int i0 = p0 & 0xff, q0 = p0 >> 8, i1 = p1 & 0xff, q1 = p1 >> 8;
          const double t0 = tcol[i0], t1 = tcol[i1];
          const double u0 = a[q0 * L64P + j], u1 = a[q1 * L64P + j];
          const double v0 = a[i0 * L64P + q0], v1 = a[i1 * L64P + q1];
          a[i0 * L64P + q0] = fma(-t0, u0, v0);
          if (e2 < e1) a[i1 * L64P + q1] = fma(-t1, u1, v1);
        }
      }
      __syncthreads();
    }
    if (*fail) break;
    if (c1 < L64) {
      // the micro-panel's contribution to the trailing block: FP32 copies of l_ik = a_ik / d_k
      // (fs[r][k]) and of a_ik (fs[r][16 + k]) for rows r = i - c1, then
      // a_ic -= sum_k l_ik a_ck for c1 <= c <= i, formed in FP32, subtracted in FP64
      const int rows = L64 - c1;
      for (int e = tid; e < rows * kMicro; e += LEAF128_THREADS) {
        const int r = e / kMicro, k = e % kMicro;
        const double u = a[(c1 + r) * L64P + c0 + k];
        fs[r * 33 + k] = f64_to_f32(u * inv[c0 + k]);
        fs[r * 33 + kMicro + k] = f64_to_f32(u);
      }
      __syncthreads();
      const int ntri = rows * (rows + 1) / 2;
      for (int e = tid; e < ntri; e += LEAF128_THREADS) {
        // entry e of the trailing lower triangle in row-major order: row r, column q <= r
        int r = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
        while (r * (r + 1) / 2 > e) --r;
        while ((r + 1) * (r + 2) / 2 <= e) ++r;
        const int q = e - r * (r + 1) / 2;
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < kMicro; ++k) acc = fmaf(fs[r * 33 + k], fs[q * 33 + kMicro + k], acc);
        a[(c1 + r) * L64P + c1 + q] -= f32_to_f64(acc);
      }
      __syncthreads();
    }
  }
  if (*fail) return;
  // L_ij = a_ij / sqrt(d_j) (i > j), L_jj = sqrt(d_j)
  if (tid < L64) tcol[tid] = rsqrt(piv[tid]);
  __syncthreads();
  for (int e = tid; e < L64 * L64; e += LEAF128_THREADS) {
    const int i = e >> 6, c = e & 63;
    if (c <= i) a[i * L64P + c] = (c == i ? piv[c] : a[i * L64P + c]) * tcol[c];
  }
  __syncthreads();
}

// One joining level of the recursive-doubling inverse: for every pair of W x W diagonal blocks
// [[X11, 0], [X21, X22]] of X, X21 = -X22 (L21 X11), the two W x W products of all pairs formed
// at once (T in tmp).  Thread layout: 8W threads per pair, each with one column j and the W / 8
// rows ib, ib + 8, ...; the k-loops run the full width W (the upper triangles of X and L hold
// zeros, so the sums equal the triangular ones) with float4 loads along k.
template <int W>
__device__ __forceinline__ void trinv_join(const float* l, float* x, float* tmp) {
  constexpr int R = W / 8;  // rows per thread
  const int tid = threadIdx.x;
  const int pair = tid / (8 * W), rem = tid % (8 * W), j = rem % W, ib = rem / W;
  const int o = 2 * W * pair;
  float acc[R];
  // T = L21 X11
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.f;
#pragma unroll
  for (int k = 0; k < W; k += 4) {
    const float b0 = x[(o + k) * F64P + o + j], b1 = x[(o + k + 1) * F64P + o + j];
    const float b2 = x[(o + k + 2) * F64P + o + j], b3 = x[(o + k + 3) * F64P + o + j];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4 a4 = *reinterpret_cast<const float4*>(l + (o + W + ib + 8 * r) * F64P + o + k);
      acc[r] = fmaf(a4.x, b0, acc[r]);
      acc[r] = fmaf(a4.y, b1, acc[r]);
      acc[r] = fmaf(a4.z, b2, acc[r]);
      acc[r] = fmaf(a4.w, b3, acc[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) tmp[(o + W + ib + 8 * r) * F64P + o + j] = acc[r];
  __syncthreads();
  // X21 = -X22 T
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.f;
#pragma unroll
  for (int k = 0; k < W; k += 4) {
    const float b0 = tmp[(o + W + k) * F64P + o + j], b1 = tmp[(o + W + k + 1) * F64P + o + j];
    const float b2 = tmp[(o + W + k + 2) * F64P + o + j], b3 = tmp[(o + W + k + 3) * F64P + o + j];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4 a4 = *reinterpret_cast<const float4*>(x + (o + W + ib + 8 * r) * F64P + o + W + k);
      acc[r] = fmaf(a4.x, b0, acc[r]);
      acc[r] = fmaf(a4.y, b1, acc[r]);
      acc[r] = fmaf(a4.z, b2, acc[r]);
      acc[r] = fmaf(a4.w, b3, acc[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) x[(o + W + ib + 8 * r) * F64P + o + j] = -acc[r];
  __syncthreads();
}

// X = L^{-1} in FP32 for the 64 x 64 lower-triangular L (FP32 copy l, pitch F64P, zero upper
// triangle), all 256 threads, by recursive doubling: the eight 8 x 8 diagonal blocks are
// inverted by forward substitution (one column per thread, 1 / l_ii from rdiag, the FP64
// reciprocal square roots of the pivots), then blocks of width 8, 16, 32 are joined pairwise
// (trinv_join).  The critical path is the 8-row substitution and three levels of short
// products instead of 64 dependent rows.  x must be zero on entry (its upper triangle is left
// so); tmp is 64 x 64 (pitch F64P) scratch.
__device__ void trinv64_f32(const float* l, const double* rdiag, float* x, float* tmp) {
  const int tid = threadIdx.x;
  if (tid < L64) {
    // diagonal block b = tid / 8, its column c = tid % 8: rows o + c .. o + 7
    const int o = tid & ~7, c = tid & 7;
    float xr[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      float sacc = 0.f;
#pragma unroll
      for (int k = 0; k < r; ++k) sacc = fmaf(l[(o + r) * F64P + o + k], xr[k], sacc);
      xr[r] = (r < c) ? 0.f : ((r == c ? 1.f : 0.f) - sacc) * (float)rdiag[o + r];
    }
#pragma unroll
    for (int r = 0; r < 8; ++r)
      if (r >= c) x[(o + r) * F64P + o + c] = xr[r];
  }
  __syncthreads();
  trinv_join<8>(l, x, tmp);
  trinv_join<16>(l, x, tmp);
  trinv_join<32>(l, x, tmp);
}

// acc[q][p] = sum_k A(row q, k) B(k, col p) over k < 64 for the thread's 16 outputs, A(i, k) at
// a[i * F64P + k]; B(k, j) at b[k * F64P + j], or at b[j * F64P + k] when BT (a transpose).
// Rows are mm_row(q) = (tid >> 4) + 16 q; columns mm_col<BT>(p) = (tid & 15) + 16 p when BT
// (the 16 lanes' B rows then fall in distinct bank groups), 4 (tid & 15) + p otherwise (one
// float4 of a B row).  Every operand is read as float4 along k or along the B row.
__device__ __forceinline__ int mm_row(int q) { return (threadIdx.x >> 4) + 16 * q; }
template <bool BT>
__device__ __forceinline__ int mm_col(int p) { return BT ? (threadIdx.x & 15) + 16 * p : 4 * (threadIdx.x & 15) + p; }
template <bool BT>
__device__ __forceinline__ void mm64_4x4(const float* a, const float* b, float (&acc)[4][4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int p = 0; p < 4; ++p) acc[q][p] = 0.f;
#pragma unroll 4
  for (int k = 0; k < L64; k += 4) {
    float av[4][4], bv[4][4];  // av[q][kk] = A(row q, k + kk); bv[kk][p] = B(k + kk, col p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(a + mm_row(q) * F64P + k);
      av[q][0] = v.x; av[q][1] = v.y; av[q][2] = v.z; av[q][3] = v.w;
    }
    if (BT) {
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const float4 v = *reinterpret_cast<const float4*>(b + mm_col<true>(p) * F64P + k);
        bv[0][p] = v.x; bv[1][p] = v.y; bv[2][p] = v.z; bv[3][p] = v.w;
      }
    } else {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const float4 v = *reinterpret_cast<const float4*>(b + (k + kk) * F64P + mm_col<false>(0));
        bv[kk][0] = v.x; bv[kk][1] = v.y; bv[kk][2] = v.z; bv[kk][3] = v.w;
      }
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[q][p] = fmaf(av[q][kk], bv[kk][p], acc[q][p]);
  }
}

__global__ void __launch_bounds__(LEAF128_THREADS, 1) k_leaf128(double* Ablk, int64_t ld, double* Xblk, double* ld_part,
                                                         int* pd) {
  dep_wait();
  dep_release();
  if (*pd == 0) return;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  constexpr int M = L64 * L64P, MF = L64 * F64P;
  double* a11 = reinterpret_cast<double*>(sm_raw);  // FP64 panels: A11 -> L11, A21 -> L21, A22 -> L22
  double* a21 = a11 + M;
  double* a22 = a21 + M;
  float* f0 = reinterpret_cast<float*>(a22 + M);    // L11 (FP32), then L21 (FP32)
  float* f1 = f0 + MF;                               // X11
  float* f2 = f1 + MF;                               // A21 (FP32), then L22 (FP32), then X21
  float* f3 = f2 + MF;                               // X22
  float* f4 = f3 + MF;                               // T = L21 X11
  __shared__ double piv[2 * L64], inv[L64], tcol[L64];
  __shared__ double red[32];
  __shared__ uint16_t tri[kTri64N];
  __shared__ int fail;
  const int tid = threadIdx.x;
  for (int e = tid; e < kTri64N; e += LEAF128_THREADS) tri[e] = g_tri64[e];
  {
    // every thread issues its 48 loads (16 per 64 x 64 panel) before storing any
    constexpr int PER = L64 * L64 / LEAF128_THREADS;   // 16
    double v11[PER], v21[PER], v22[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + u * LEAF128_THREADS, i = e >> 6, c = e & 63;
      v11[u] = (c <= i) ? Ablk[(int64_t)i * ld + c] : 0.0;
      v21[u] = Ablk[(int64_t)(L64 + i) * ld + c];
      v22[u] = (c <= i) ? Ablk[(int64_t)(L64 + i) * ld + L64 + c] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + u * LEAF128_THREADS, i = e >> 6, c = e & 63;
      a11[i * L64P + c] = v11[u];
      a21[i * L64P + c] = v21[u];
      a22[i * L64P + c] = v22[u];
    }
  }
  if (tid == 0) fail = 0;
  __syncthreads();
  // ---- first panel: L11 (FP64), X11 = L11^{-1} (FP32)
  chol64_f64(a11, piv, inv, tcol, tri, f0, &fail);
  if (fail) {
    if (tid == 0) *pd = 0;
    return;
  }
  for (int e = tid; e < L64 * L64; e += LEAF128_THREADS) {
    const int i = e >> 6, c = e & 63;
    f0[i * F64P + c] = f64_to_f32(a11[i * L64P + c]);
    f2[i * F64P + c] = f64_to_f32(a21[i * L64P + c]);
    f1[i * F64P + c] = 0.f;
    f3[i * F64P + c] = 0.f;
  }
  __syncthreads();
  trinv64_f32(f0, tcol, f1, f4);
  // ---- L21 = A21 X11^T (FP32), kept in FP64 (a21) and FP32 (f0)
  {
    float acc[4][4];
    mm64_4x4<true>(f2, f1, acc);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        a21[mm_row(q) * L64P + mm_col<true>(p)] = f32_to_f64(acc[q][p]);
        f0[mm_row(q) * F64P + mm_col<true>(p)] = acc[q][p];
      }
  }
  __syncthreads();
  // ---- A22 -= L21 L21^T: FP32 product, FP64 subtraction (lower triangle)
  {
    float acc[4][4];
    mm64_4x4<true>(f0, f0, acc);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int p = 0; p < 4; ++p)
        if (mm_col<true>(p) <= mm_row(q)) a22[mm_row(q) * L64P + mm_col<true>(p)] -= f32_to_f64(acc[q][p]);
  }
  // ---- T = L21 X11 (FP32), independent of the second panel
  {
    float acc[4][4];
    mm64_4x4<false>(f0, f1, acc);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int p = 0; p < 4; ++p) f4[mm_row(q) * F64P + mm_col<false>(p)] = acc[q][p];
  }
  __syncthreads();
  // ---- second panel: L22 (FP64), X22 (FP32)
  chol64_f64(a22, piv + L64, inv, tcol, tri, f2, &fail);
  if (fail) {
    if (tid == 0) *pd = 0;
    return;
  }
  for (int e = tid; e < L64 * L64; e += LEAF128_THREADS) {
    const int i = e >> 6, c = e & 63;
    f2[i * F64P + c] = f64_to_f32(a22[i * L64P + c]);
  }
  __syncthreads();
  trinv64_f32(f2, tcol, f3, f0);
  // ---- X21 = -X22 T (FP32)
  {
    float acc[4][4];
    mm64_4x4<false>(f3, f4, acc);
    __syncthreads();  // every thread has read f2 (L22) before it is overwritten
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int p = 0; p < 4; ++p) f2[mm_row(q) * F64P + mm_col<false>(p)] = -acc[q][p];
  }
  // ---- log det = sum of log pivots (FP64)
  const double lsum = (tid < 2 * L64) ? log(piv[tid]) : 0.0;
  const double tot = block_sum(lsum, red);   // its barriers also order the writes above
  __syncthreads();
  for (int e = tid; e < L64 * L64; e += LEAF128_THREADS) {
    const int i = e >> 6, c = e & 63;
    double* Ar0 = Ablk + (int64_t)i * ld;
    double* Ar1 = Ablk + (int64_t)(L64 + i) * ld;
    double* Xr0 = Xblk + (int64_t)i * ld;
    double* Xr1 = Xblk + (int64_t)(L64 + i) * ld;
    Ar0[c] = (c <= i) ? a11[i * L64P + c] : 0.0;   // L11 (zero upper)
    Ar0[L64 + c] = 0.0;                            // upper off-diagonal block
    Ar1[c] = a21[i * L64P + c];                    // L21
    Ar1[L64 + c] = (c <= i) ? a22[i * L64P + c] : 0.0;   // L22
    if (c <= i) Xr0[c] = f32_to_f64(f1[i * F64P + c]);   // X11
    Xr1[c] = f32_to_f64(f2[i * F64P + c]);                // X21
    if (c <= i) Xr1[L64 + c] = f32_to_f64(f3[i * F64P + c]);   // X22
  }
  if (tid == 0) *ld_part = tot;
}

// The leaf is launched with nearly all of an SM's shared memory (more than it uses), so that
// no other block with shared memory is placed beside it: the concurrent tier-2 kernels and
// the sparse products are FP64-bound, and FP64 instructions of a neighbour on the pivot
// chain's sub-partition would delay every pivot.
size_t leaf128_launch_smem() {
  static const size_t v = [] {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return leaf128_smem();
    const size_t reserve = optin > 16384 ? (size_t)optin - 8192 : 0;  // room for the static part
    return std::max(leaf128_smem(), reserve);
  }();
  return v;
}

// out = sum of parts[0..n) in index order (one thread: n is at most a few hundred).
__global__ void k_sum_parts(const double* parts, int n, const int* pd, double* out) {
  dep_wait();
  dep_release();
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += parts[i];
  *out = (*pd) ? s : NAN;
}

// dst[rows x cols] := src[rows x cols] (both with leading dimension ld), unless *flag == 0.
__global__ void k_copy_block(const double* __restrict__ src, double* __restrict__ dst, int64_t ld,
                             int rows, int cols, const int* flag) {
  dep_wait();
  dep_release();
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
// The column-major list of the 64 x 64 lower triangle for k_leaf128's FP64 updates, written
// to each device once, from the host thread that first factors on it (the first
// factorisation of an engine runs directly, never inside a stream capture).
void tri64_tables_once() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  CUDA_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0 || dev >= 64 || done[dev]) return;
  uint16_t t[kTri64N];
  int e = 0;
  for (int c = 0; c < L64; ++c)
    for (int i = c; i < L64; ++i) t[e++] = (uint16_t)(i | (c << 8));
  CUDA_CHECK(cudaMemcpyToSymbol(g_tri64, t, sizeof(t)));
  done[dev] = true;
}

struct Ctx {
  bool split;      // split-precision modes: in-place panel products on the tensor cores
  LeafKind kind;   // which leaf kernel factors the diagonal blocks
  int leaf;
  double* A;
  double* X;
  double* T;
  double* T2;      // a second small-product scratch region of T (columns np - 256 ..), or null
  int64_t ld;
  double* ld_parts;
  int* pd;
  const GemmFn* gemm;
  cudaStream_t st;
  size_t smem;
  const SideStream* side;
};

// The recursion splits a block of s rows (a multiple of the leaf) into halves of whole leaves.
int split_point(int s, int leaf) { return ((s / leaf + 1) / 2) * leaf; }

// Factor the diagonal block [o, o + s) of A in place and write X = L^{-1} there:
//   L11 X11 from the first half; L21 = A21 X11^T; A22 -= L21 L21^T; L22 X22 from the second
//   half; X21 = -X22 (L21 X11).
void chol_inv_rec(const Ctx& c, int o, int s) {
  if (s == c.leaf) {
    double* Ab = c.A + (int64_t)o * c.ld + o;
    double* Xb = c.X + (int64_t)o * c.ld + o;
    double* part = c.ld_parts + o / c.leaf;
    switch (c.kind) {
      case LeafKind::F64Chol:
        launch_dependent(k_leaf128, 1, LEAF128_THREADS, c.smem, c.st, Ab, c.ld, Xb, part, c.pd);
        break;
      case LeafKind::F32:
        launch_dependent(k_leaf_chol_inv<float, NB32, 4 * NB32>, 1, 4 * NB32, c.smem, c.st, Ab, c.ld, Xb, part, c.pd);
        break;
      default:
        launch_dependent(k_leaf_chol_inv<double, NB, 4 * NB>, 1, 4 * NB, c.smem, c.st, Ab, c.ld, Xb, part, c.pd);
    }
    return;
  }
  const int s1 = split_point(s, c.leaf), s2 = s - s1;
  chol_inv_rec(c, o, s1);
  const int64_t ld = c.ld;
  double* A21 = c.A + (int64_t)(o + s1) * ld + o;
  double* A22 = c.A + (int64_t)(o + s1) * ld + o + s1;
  const double* X11 = c.X + (int64_t)o * ld + o;
  const double* X22 = c.X + (int64_t)(o + s1) * ld + o + s1;
  double* X21 = c.X + (int64_t)(o + s1) * ld + o;
  // L21 = A21 X11^T (X11^T upper triangular).  The tensor-core product reads its operands
  // from the split copies made before it starts, so it may overwrite A21 in place; the
  // CUDA-core kernels (FP64, and FP32 for small products) read A21 tile by tile and go
  // through T.
  const bool in_place = c.split && std::max(s1, s2) > kSmallGemm;
  GemmArgs a = gemm_args(A21, ld, 0, X11, ld, 1, in_place ? A21 : c.T, ld, s2, s1, s1, 1.0, 0.0);
  a.krule = KR_HI_COL;
  a.flag = c.pd;
  (*c.gemm)(a, GemmRole::Panel, c.st);
  if (!in_place) {
    launch_dependent(k_copy_block, std::min(s2, 1024), 256, 0, c.st, c.T, A21, ld, s2, s1, c.pd);
  }
  // X21 = -X22 (L21 X11).  With a side stream, the first factor L21 X11 is formed on the side
  // stream right away: it needs only L21 and X11, so it overlaps the trailing update and the
  // whole right half.  In-place tensor-core products put it into X21; a small node whose
  // right half is one leaf puts it into T2 (a node with a deeper right half would see its
  // children's side products reuse T2 before its own last product reads it).
  const bool fork = in_place && c.side && c.side->st;
  const bool fork_small = !in_place && c.side && c.side->st && c.T2 && s2 == c.leaf;
  if (fork || fork_small) {
    CUDA_CHECK(cudaEventRecord(c.side->fork, c.st));
    CUDA_CHECK(cudaStreamWaitEvent(c.side->st, c.side->fork, 0));
    GemmArgs d = gemm_args(A21, ld, 0, X11, ld, 0, fork ? X21 : c.T2, ld, s2, s1, s1, 1.0, 0.0);
    d.krule = KR_LO_COL;
    d.flag = c.pd;
    (*c.gemm)(d, GemmRole::Inverse, c.side->st);
  }
  // A22 -= L21 L21^T on the lower triangle
  GemmArgs b = gemm_args(A21, ld, 0, A21, ld, 1, A22, ld, s2, s2, s1, -1.0, 1.0);
  b.lower = 1;
  b.flag = c.pd;
  (*c.gemm)(b, GemmRole::Trailing, c.st);
  chol_inv_rec(c, o + s1, s2);
  if (fork) {
    // join: everything the side stream holds so far (this node's product among it)
    CUDA_CHECK(cudaEventRecord(c.side->join, c.side->st));
    CUDA_CHECK(cudaStreamWaitEvent(c.st, c.side->join, 0));
    // X21 := -X22 X21 in place (the tensor-core product reads split copies of its operands)
    GemmArgs e = gemm_args(X22, ld, 0, X21, ld, 0, X21, ld, s2, s1, s2, -1.0, 0.0);
    e.krule = KR_HI_ROW;
    e.flag = c.pd;
    (*c.gemm)(e, GemmRole::Inverse, c.st);
    return;
  }
  if (fork_small) {
    CUDA_CHECK(cudaEventRecord(c.side->join, c.side->st));
    CUDA_CHECK(cudaStreamWaitEvent(c.st, c.side->join, 0));
    GemmArgs e = gemm_args(X22, ld, 0, c.T2, ld, 0, X21, ld, s2, s1, s2, -1.0, 0.0);
    e.krule = KR_HI_ROW;
    e.flag = c.pd;
    (*c.gemm)(e, GemmRole::Inverse, c.st);
    return;
  }
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
                      double* logdet, const GemmFn& gemm, cudaStream_t st, bool split, LeafKind kind,
                      int panel, const SideStream* side) {
  const int leaf = kind == LeafKind::F64 ? NB : NB32;
  const size_t smem = kind == LeafKind::F64Chol ? leaf128_launch_smem()
                      : kind == LeafKind::F32   ? leaf_smem(NB32, sizeof(float))
                                                : leaf_smem(NB, sizeof(double));
  static std::once_flag once;  // not repeated inside a stream capture
  std::call_once(once, [] {
    CUDA_CHECK(cudaFuncSetAttribute(k_leaf_chol_inv<float, NB32, 4 * NB32>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)leaf_smem(NB32, sizeof(float))));
    CUDA_CHECK(cudaFuncSetAttribute(k_leaf_chol_inv<double, NB, 4 * NB>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)leaf_smem(NB, sizeof(double))));
    CUDA_CHECK(cudaFuncSetAttribute(k_leaf128, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)leaf128_launch_smem()));
  });
  tri64_tables_once();
  CUDA_CHECK(cudaMemsetAsync(X, 0, sizeof(double) * ld * np, st));
  // T2 = columns np - 256 .. np - 1 of T's first rows: disjoint from the top-left 256 x 256
  // corner the main stream's small products use, when np >= 512
  double* T2 = np >= 2 * kSmallGemm ? T + (np - kSmallGemm) : nullptr;
  Ctx c{split, kind, leaf, A, X, T, T2, ld, ld_parts, pd, &gemm, st, smem, panel <= 0 ? side : nullptr};
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
      GemmArgs a = gemm_args(A21, ld, 0, Xkk, ld, 1, split ? A21 : T, ld, rem, s, s, 1.0, 0.0);
      a.krule = KR_HI_COL;
      a.flag = pd;
      gemm(a, GemmRole::Panel, st);
      if (!split) {
        k_copy_block<<<std::min(rem, 1024), 256, 0, st>>>(T, A21, ld, rem, s, pd);
        LAUNCH_CHECK();
      }
      GemmArgs b = gemm_args(A21, ld, 0, A21, ld, 1, A22, ld, rem, rem, s, -1.0, 1.0);
      b.lower = 1;
      b.flag = pd;
      gemm(b, GemmRole::Trailing, st);
    }
  }
  launch_dependent(k_sum_parts, 1, 32, 0, st, ld_parts, np / leaf, pd, logdet);
}

void factorisation_products(int np, bool split, LeafKind kind, std::vector<GemmArgs>& out) {
  const int leaf = kind == LeafKind::F64 ? NB : NB32;
  // mirrors chol_inv_rec: the panel, trailing and two inverse products of every inner node,
  // with the operand layout and in-place flags the recursion gives them (pointers are dummies
  // whose equality encodes aliasing)
  std::vector<std::pair<int, int>> stack{{0, np}};
  const double* P = reinterpret_cast<const double*>(16);
  const double* Q = reinterpret_cast<const double*>(32);
  double* C = reinterpret_cast<double*>(48);
  while (!stack.empty()) {
    const int s = stack.back().second;
    stack.pop_back();
    if (s <= leaf) continue;
    const int s1 = split_point(s, leaf), s2 = s - s1;
    const bool in_place = split && std::max(s1, s2) > kSmallGemm;
    GemmArgs a = gemm_args(P, np, 0, Q, np, 1, in_place ? const_cast<double*>(P) : C, np, s2, s1, s1, 1.0, 0.0);
    a.krule = KR_HI_COL;
    out.push_back(a);
    GemmArgs b = gemm_args(P, np, 0, P, np, 1, C, np, s2, s2, s1, -1.0, 1.0);
    b.lower = 1;
    out.push_back(b);
    GemmArgs d = gemm_args(P, np, 0, Q, np, 0, C, np, s2, s1, s1, 1.0, 0.0);
    d.krule = KR_LO_COL;
    out.push_back(d);
    GemmArgs e = gemm_args(Q, np, 0, in_place ? C : P, np, 0, C, np, s2, s1, s2, -1.0, 0.0);
    e.krule = KR_HI_ROW;
    out.push_back(e);
    stack.push_back({0, s1});
    stack.push_back({0, s2});
  }
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
  // W = X^T X (lower triangle; the caller mirrors it)
  GemmArgs w = gemm_args(X, ld, 1, X, ld, 0, W, ld, np, np, np, 1.0, 0.0);
  w.lower = 1;
  w.krule = KR_LO_ROW;
  gemm(w, GemmRole::Inverse, st);
}

}  // namespace glasso
