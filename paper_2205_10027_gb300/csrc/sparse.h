// Sparsity-aware sandwich products: Y = Theta X Theta with Theta held in CSR form.
#pragma once
#include "common.cuh"

namespace glasso {

// CSR of the n x n block of a padded matrix (row-major, leading dimension ld): rowptr has
// np + 1 entries (rows n .. np - 1 are empty), col / val hold the nonzeros of each row in
// column order.  Capacity of col / val in entries.
struct Csr {
  int64_t* rowptr = nullptr;
  int* col = nullptr;
  double* val = nullptr;
  int64_t cap = 0;
};

// rowptr := exclusive prefix sum of the per-row nonzero counts of the n x n block of A, or of
// A - Am when Am is given (rowptr[np] = nnz).  counts: np ints of scratch.
void csr_rowptr(const double* A, const double* Am, int64_t ld, int64_t n, int np, int* counts,
                int64_t* rowptr, cudaStream_t st);
// col / val from rowptr (the caller has checked rowptr[np] <= cap); same A, Am.
void csr_fill(const double* A, const double* Am, int64_t ld, int64_t n, int np, Csr& c, cudaStream_t st);

// OUT = A B over np x np with A in CSR (rows of A beyond n are zero): out[i][j] or, with
// transpose, out[j][i] := sum_k A_ik B[k][j].  lower: only 32 x 64 tiles that meet the lower
// triangle are written (entries above the diagonal inside them are written too).  FP64
// arithmetic, terms summed in column order of A.
void spmm(const Csr& a, const double* B, int64_t ldb, double* out, int64_t ldo, int np, bool transpose,
          bool lower, cudaStream_t st);
// R = I - A B over np x np (the identity on the first n diagonal entries; rows of A beyond n
// are zero), and *rmax = max(*rmax, max |R_ij| over the n x n block).
void spmm_residual(const Csr& a, const double* B, int64_t ldb, double* R, int64_t ldr, int64_t n, int np,
                   double* rmax, cudaStream_t st);

}  // namespace glasso
