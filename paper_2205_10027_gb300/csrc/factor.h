// Cholesky factorisation and inverse from the factor (see factor.cu).
#pragma once
#include <algorithm>
#include <functional>
#include "gemm.h"

namespace glasso {

// Which product of the path a GEMM call is, so the dispatcher can pick the precision.
enum class GemmRole { Panel, Trailing, Inverse, Sandwich, Refine };
using GemmFn = std::function<void(const GemmArgs&, GemmRole, cudaStream_t)>;

// In-place lower Cholesky of the np x np matrix A (lower triangle read and overwritten;
// the upper triangle of the diagonal blocks is zeroed, the rest of the upper triangle is
// left as it was).  *pd must be 1 on entry and is cleared on a bad pivot, after which the
// remaining launches do nothing.  *logdet = 2 sum log L_ii (NaN when not PD).
// Dinv receives the inverses of the 64 x 64 diagonal blocks; ld_parts np/64 doubles.
void cholesky_f64(double* A, int64_t ld, int np, double* Dinv, double* ld_parts, int* pd,
                  double* logdet, const GemmFn& gemm, cudaStream_t st);

// W = (L L^T)^{-1} = X^T X with X = L^{-1} built from the factor's lower triangle and the
// diagonal-block inverses Dinv.  X and T are np x np scratch; W is written in full.
void inverse_from_factor(const double* L, const double* Dinv, int64_t ld, int np, double* X,
                         double* T, double* W, const GemmFn& gemm, cudaStream_t st);

void mirror_lower(double* M, int64_t ld, int np, cudaStream_t st);

}  // namespace glasso
