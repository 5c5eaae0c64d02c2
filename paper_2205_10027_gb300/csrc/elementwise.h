// HBM-bound passes of the pISTA iteration (see elementwise.cu).
#pragma once
#include <algorithm>
#include "common.cuh"

namespace glasso {

constexpr int kRedBlocks = 1024;  // partial-sum slots per reduction (fixed: deterministic)
int red_blocks(int64_t work_rows);

// dst (np x np, ld) := the caller's n x n S (FP32 or FP64, device memory) with its lower
// triangle mirrored and zero padding; vmax[0] = max |S_ij - S_ji|, vmax[1] = max |S_ij|
// (both must be 0 on entry), *bad += number of non-finite entries and negative S_ii.
void load_symmetric(const void* src, bool f32, int64_t n, double* dst, int64_t ld, int np,
                    double* vmax, int* bad, cudaStream_t st);
// A[i][i] = 1/(S_ii + lam) for i < n, 1 on the padding (A zero elsewhere beforehand).
void init_diag(const double* S, int64_t ld, int64_t n, int np, double lam, double* A, cudaStream_t st);
void pad_identity(double* A, int64_t ld, int64_t n, int np, cudaStream_t st);
// K1: X, code and out5 = {||Z||_1, ||A||_1, ||Z||_F^2, nnz(A), |M|} (|M| the free-set entries
// of the n x n matrix); parts >= 5 * kRedBlocks.
void gradient(const double* S, const double* W, const double* A, int64_t ld, int64_t n, double lam,
              double* X, int8_t* code, int64_t ldc, double* parts, double* out5, cudaStream_t st);
// K3: At (full), Lt (lower) and out5 = {<S, At - A>, sum(|At| - |A|), tr(S At), ||At||_1, nnz(At)}.
void trial(const double* A, const double* Y, const int8_t* code, int64_t ldc, const double* S,
           int64_t ld, int64_t n, int np, double lam, double t, double* At, double* Lt,
           double* parts, double* out5, cudaStream_t st);
// S (n x n block) <- D^{-1/2} S D^{-1/2}, D = diag S, as (S_ij d_i) d_j with d_i = 1/sqrt(S_ii)
// (d: n doubles of scratch); *bad += the number of S_ii <= 0 (bad must be 0 on entry).
void standardize(double* S, int64_t ld, int64_t n, double* d, int* bad, cudaStream_t st);
// G-ISTA candidate (proximal gradient with H = I): At (full) = ST(A - t (S - W), t lam) on
// the n x n block (identity padding), Lt (lower) = At, and out5 = {tr(S At), ||At||_1,
// nnz(At), <S - W, At - A>, ||At - A||_F^2}.
void gista_trial(const double* A, const double* W, const double* S, int64_t ld, int64_t n, int np,
                 double lam, double t, double* At, double* Lt, double* parts, double* out5,
                 cudaStream_t st);
// out2 = {tr(S A), ||A||_1}.
void objective_terms(const double* S, const double* A, int64_t ld, int64_t n, double* parts,
                     double* out2, cudaStream_t st);
// Q = (At - A) W and out2 = {tr(Q), tr(Q^2)}: the first two terms of
// log det At - log det A = tr(E) - tr(E^2)/2 + ..., E similar to Q.
void logdet_difference_terms(const double* At, const double* A, const double* W, int64_t ld,
                             int64_t n, int np, double* Q, double* parts, double* out2,
                             cudaStream_t st);
// out2 = {tr(Q), tr(Q^2)} of a given Q (its n x n block).
void trace_terms(const double* Q, int64_t ld, int64_t n, int np, double* parts, double* out2,
                 cudaStream_t st);
// R = I - A W in FP64 over the padded size (padding of R zero), with the nonzeros of each
// row of A compacted first; *rmax = max |R_ij| over the n x n block.
void inverse_residual(const double* A, const double* W, int64_t ld, int64_t n, int np, double* R,
                      double* rmax, cudaStream_t st);
// lower(W) += lower(C), then W's upper triangle := its lower triangle transposed.
void add_lower_mirror(double* W, const double* C, int64_t ld, int np, cudaStream_t st);
void unpad(const double* src, int64_t ld, int64_t n, double* dst, cudaStream_t st);
void unpad_i8(const int8_t* src, int64_t ld, int64_t n, int8_t* dst, cudaStream_t st);
void pad_i8(const int8_t* src, int64_t n, int8_t* dst, int64_t ld, cudaStream_t st);

}  // namespace glasso
