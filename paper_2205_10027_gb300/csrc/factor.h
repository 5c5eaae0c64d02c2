// Cholesky factorisation and inverse from the factor (see factor.cu).
#pragma once
#include <algorithm>
#include <functional>
#include <vector>
#include "gemm.h"

namespace glasso {

// Which product of the path a GEMM call is, so the dispatcher can pick the precision.
enum class GemmRole { Panel, Trailing, Inverse, Sandwich, Refine };
using GemmFn = std::function<void(const GemmArgs&, GemmRole, cudaStream_t)>;

// In-place lower Cholesky of the np x np matrix A (lower triangle read and overwritten; the
// upper triangle of the leaf blocks is zeroed, the rest of the upper triangle is left as it
// was).  panel <= 0: recursive halving over the whole matrix, and X = L^{-1} is written in full.
// panel > 0: right-looking over panels of that width (a multiple of the leaf), each diagonal
// block factored recursively; X then holds only the inverses of the diagonal panel blocks
// (inverse_merge completes it).  T is np x np scratch.  *pd must be 1 on entry and is
// cleared on a bad pivot, after which the remaining launches do nothing; *logdet =
// 2 sum log L_ii (NaN when not PD).  ld_parts: np/64 doubles.  split: the products run in a
// split-precision mode (the tensor-core panel products may then write their output in place).
// kind: the leaf kernel of the diagonal blocks.
enum class LeafKind {
  F64,      // 64 x 64, Cholesky and inverse in FP64 (the FP64 form)
  F64Chol,  // 64 x 64, Cholesky, pivots and log det in FP64, inverse of the factor in FP32
  F32       // 128 x 128, Cholesky and inverse in FP32 (an option of the split-precision forms)
};
// side: optional second stream (with fork / join events) on which the split-precision
// recursion runs the first inverse product of a node, X21 := L21 X11, beside the trailing
// update and the right half, which do not depend on it; the GEMM dispatcher must give
// products on that stream their own scratch.
struct SideStream {
  cudaStream_t st = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
void cholesky_inverse(double* A, double* X, int64_t ld, int np, double* T, double* ld_parts, int* pd,
                      double* logdet, const GemmFn& gemm, cudaStream_t st, bool split = false,
                      LeafKind kind = LeafKind::F64, int panel = 0, const SideStream* side = nullptr);

// The dense products the recursion issues for an np x np factorisation (shapes, structure
// and in-place flags; the pointers only encode which operands alias), for the autotuner.
void factorisation_products(int np, bool split, LeafKind kind, std::vector<GemmArgs>& out);

// Completes X = L^{-1} from the inverses of the diagonal panel blocks left by
// cholesky_inverse(..., panel).  T is np x np scratch.
void inverse_merge(const double* L, double* X, int64_t ld, int np, double* T, int panel, const GemmFn& gemm,
                   cudaStream_t st);

// W = X^T X = (L L^T)^{-1} from X = L^{-1} (lower): the lower triangle of W (mirror_lower
// completes it).
void inverse_from_inverse_factor(const double* X, int64_t ld, int np, double* W, const GemmFn& gemm,
                                 cudaStream_t st);

void mirror_lower(double* M, int64_t ld, int np, cudaStream_t st);

}  // namespace glasso
