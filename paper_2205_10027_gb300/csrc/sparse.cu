// Sparsity-aware sandwich products (the products A X A of eq. b with A = Theta in CSR form).
//
// Theta keeps a few to a few tens of nonzeros per row along the iteration, so A X and
// (A X)^T A cost O(nnz n) FP64 multiply-adds instead of the O(n^3) of a dense product, and
// they are exact FP64 products (no split-precision error).  Y = A X A is formed as
// T = (A X)^T = X A (the first product stored transposed; X and A are symmetric), then
// Y = A T on the tiles that meet the lower triangle.
#include "sparse.h"
#include "../../include/glasso.h"

namespace glasso {

namespace {
constexpr int kRowsPerBlock = 8;  // one warp per row in the CSR passes

// Whether entry o of A (of A - Am when Am is given) is stored: A_o != 0, or A_o != Am_o, both
// decided on the bit patterns with integer instructions only (an FP64 compare or subtraction
// costs one FP64 instruction per warp, and these passes read every entry of the n x n block).
// Shifting out the sign bit makes -0 a zero; two patterns that differ and are not both zeros
// are two different numbers (or a NaN), whose difference is nonzero, so the count is the
// count of nonzero A - Am and stays within nnz(A) + nnz(Am).
__device__ __forceinline__ bool stored(const double* __restrict__ A, const double* __restrict__ Am, int64_t o) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(A[o]);
  if (!Am) return (a << 1) != 0;
  const unsigned long long b = (unsigned long long)__double_as_longlong(Am[o]);
  return a != b && ((a | b) << 1) != 0;
}

// counts[i] = nonzeros of row i of the n x n block (0 for the padding rows)
__global__ void k_row_counts(const double* __restrict__ A, const double* __restrict__ Am, int64_t ld, int64_t n,
                             int np, int* counts) {
  const int i = blockIdx.x * kRowsPerBlock + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= np) return;
  int c = 0;
  if (i < n) {
    for (int64_t j0 = 0; j0 < n; j0 += 32) {
      const int64_t j = j0 + lane;
      const bool nz = j < n && stored(A, Am, (int64_t)i * ld + j);
      c += __popc(__ballot_sync(0xffffffffu, nz));
    }
  }
  if (lane == 0) counts[i] = c;
}

// rowptr = exclusive prefix sum of counts (np + 1 entries), one block of 1024 threads: each
// thread sums a contiguous chunk, the chunk sums are scanned in shared memory, then each
// thread writes its chunk's prefixes.
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ counts, int np, int64_t* rowptr) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int chunk = (np + 1023) / 1024;
  const int b = t * chunk, e = min(np, b + chunk);
  int64_t s = 0;
  for (int i = b; i < e; ++i) s += counts[i];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {  // inclusive Hillis-Steele scan
    const int64_t v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int64_t run = t > 0 ? part[t - 1] : 0;
  for (int i = b; i < e; ++i) {
    rowptr[i] = run;
    run += counts[i];
  }
  if (t == 1023) rowptr[np] = part[1023];
}

// col / val of row i at rowptr[i] .. in column order (ballot compaction, one warp per row)
__global__ void k_csr_fill(const double* __restrict__ A, const double* __restrict__ Am, int64_t ld, int64_t n,
                           const int64_t* __restrict__ rowptr, int* __restrict__ col,
                           double* __restrict__ val) {
  const int i = blockIdx.x * kRowsPerBlock + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= n) return;
  int64_t base = rowptr[i];
  for (int64_t j0 = 0; j0 < n; j0 += 32) {
    const int64_t j = j0 + lane;
    const bool nz = j < n && stored(A, Am, (int64_t)i * ld + j);
    const unsigned m = __ballot_sync(0xffffffffu, nz);
    if (nz) {
      // the difference is formed only for stored entries (one FP64 instruction per warp that
      // holds any)
      const int64_t o = (int64_t)i * ld + j;
      const int64_t pos = base + __popc(m & ((1u << lane) - 1u));
      col[pos] = (int)j;
      val[pos] = Am ? A[o] - Am[o] : A[o];
    }
    base += __popc(m);
  }
}

// One 32-row x 64-column tile of A B per block: warp w takes rows w, w + 8, ..., its lanes
// columns c0 + lane and c0 + 32 + lane; the tile is staged in shared memory so that both the
// direct and the transposed store are coalesced.
// RESID: the tile holds I - A B (identity on the first n diagonal entries) and the block
// folds max |.| over its n x n part into *rmax.
template <bool TRANS, bool RESID>
__global__ void __launch_bounds__(256) k_spmm(const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                                              const double* __restrict__ val, const double* __restrict__ B,
                                              int64_t ldb, double* __restrict__ out, int64_t ldo, int lower,
                                              int64_t n, double* rmax) {
  const int c0 = blockIdx.x * 64, r0 = blockIdx.y * 32;
  if (lower && c0 > r0 + 31) return;
  __shared__ double tile[32][65];
  __shared__ unsigned long long wmax[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int rr = warp; rr < 32; rr += 8) {
    const int64_t e0 = rowptr[r0 + rr], e1 = rowptr[r0 + rr + 1];
    double a0 = 0.0, a1 = 0.0;
    for (int64_t e = e0; e < e1; ++e) {
      const double* b = B + (int64_t)col[e] * ldb + c0;
      const double v = val[e];
      a0 = fma(v, b[lane], a0);
      a1 = fma(v, b[32 + lane], a1);
    }
    if (RESID) {
      // I - A B: off the diagonal a sign flip (no FP64 instruction), on it 1 + (-sum), the
      // same rounding as 1 - sum.  The addition sits behind a warp-uniform test (does row i's
      // diagonal fall in this tile?): a per-lane predicate alone would still issue the FP64
      // instruction for the whole warp on every row, ~13% more FP64 issue in this kernel.
      const int64_t i = r0 + rr;
      a0 = neg_f64(a0);
      a1 = neg_f64(a1);
      if (i < n && i >= c0 && i < c0 + 64) {
        if (i == c0 + lane) a0 += 1.0;
        if (i == c0 + 32 + lane) a1 += 1.0;
      }
    }
    tile[rr][lane] = a0;
    tile[rr][32 + lane] = a1;
  }
  __syncthreads();
  if (RESID) {
    // max |.| on the bit patterns with the sign cleared (integer order = order of |x|, and a
    // NaN ranks above every number, so it reaches *rmax instead of being skipped)
    unsigned long long mx = 0;
    for (int rr = warp; rr < 32; rr += 8) {
      if (r0 + rr >= n) break;
      if (c0 + lane < n) mx = umax64(mx, abs_bits(tile[rr][lane]));
      if (c0 + 32 + lane < n) mx = umax64(mx, abs_bits(tile[rr][32 + lane]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = umax64(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) wmax[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long m = 0;
      for (int w = 0; w < 8; ++w) m = umax64(m, wmax[w]);
      if (m != 0) atomicMax(reinterpret_cast<unsigned long long*>(rmax), m);
    }
  }
  if (!TRANS) {
    for (int e = threadIdx.x; e < 32 * 64; e += 256) {
      const int r = e >> 6, c = e & 63;
      out[(int64_t)(r0 + r) * ldo + c0 + c] = tile[r][c];
    }
  } else {
    for (int e = threadIdx.x; e < 32 * 64; e += 256) {
      const int c = e >> 5, r = e & 31;
      out[(int64_t)(c0 + c) * ldo + r0 + r] = tile[r][c];
    }
  }
}
}  // namespace

void csr_rowptr(const double* A, const double* Am, int64_t ld, int64_t n, int np, int* counts,
                int64_t* rowptr, cudaStream_t st) {
  k_row_counts<<<(np + kRowsPerBlock - 1) / kRowsPerBlock, 32 * kRowsPerBlock, 0, st>>>(A, Am, ld, n, np, counts);
  LAUNCH_CHECK();
  k_scan<<<1, 1024, 0, st>>>(counts, np, rowptr);
  LAUNCH_CHECK();
}

void csr_fill(const double* A, const double* Am, int64_t ld, int64_t n, int np, Csr& c, cudaStream_t st) {
  (void)np;
  k_csr_fill<<<(int)((n + kRowsPerBlock - 1) / kRowsPerBlock), 32 * kRowsPerBlock, 0, st>>>(A, Am, ld, n, c.rowptr,
                                                                                            c.col, c.val);
  LAUNCH_CHECK();
}

void spmm(const Csr& a, const double* B, int64_t ldb, double* out, int64_t ldo, int np, bool transpose,
          bool lower, cudaStream_t st) {
  if (np % 64) throw Error(GLASSO_ERR_ARG, "spmm: np must be a multiple of 64");
  dim3 grid(np / 64, np / 32);
  if (transpose)
    k_spmm<true, false><<<grid, 256, 0, st>>>(a.rowptr, a.col, a.val, B, ldb, out, ldo, lower ? 1 : 0, 0, nullptr);
  else
    k_spmm<false, false><<<grid, 256, 0, st>>>(a.rowptr, a.col, a.val, B, ldb, out, ldo, lower ? 1 : 0, 0, nullptr);
  LAUNCH_CHECK();
}

void spmm_residual(const Csr& a, const double* B, int64_t ldb, double* R, int64_t ldr, int64_t n, int np,
                   double* rmax, cudaStream_t st) {
  if (np % 64) throw Error(GLASSO_ERR_ARG, "spmm: np must be a multiple of 64");
  dim3 grid(np / 64, np / 32);
  k_spmm<false, true><<<grid, 256, 0, st>>>(a.rowptr, a.col, a.val, B, ldb, R, ldr, 0, n, rmax);
  LAUNCH_CHECK();
}

}  // namespace glasso
