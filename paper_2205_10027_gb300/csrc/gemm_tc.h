// Split-precision GEMM on the 5th-generation tensor cores (tcgen05 + TMEM + TMA).
#pragma once
#include "gemm.h"

namespace glasso {

class Engine;

enum class TcKind { TF32x3, BF16x3 };
// Output tile of the tensor-core kernel: 128 x 256 (Wide) or 128 x 128 (Square); Default
// takes Wide unless GLASSO_TC_TILE=128.
enum class TcTile { Default, Wide, Square };

// Device scratch the split operands of an np x np product need.
size_t tc_scratch_bytes_for(int np);
// Whether the tensor-core kernel covers this product's shape and options.
bool tc_gemm_supported(const GemmArgs& a);
// C = alpha op(A) op(B) + beta C with each FP64 operand split into hi + lo parts and the
// three products hi*hi + hi*lo + lo*hi accumulated in FP32 in TMEM; the epilogue adds
// alpha * acc to beta * C in FP64 and stores FP64.
void tc_gemm(const GemmArgs& a, TcKind kind, void* scratch, size_t scratch_bytes, cudaStream_t st,
             TcTile tile = TcTile::Default);
// Whether the driver exposes what the tensor-core path needs (TMA descriptor encoding).
bool tc_available();
// 1 if a tensor-core kernel timed out waiting on one of its barriers (synchronises st).
int tc_error_flag(cudaStream_t st);
// The device word the tensor-core kernels set on such a timeout (nullptr before the first
// tensor-core product), for callers that copy it back with other results.
const int* tc_error_word();
// Clear that word (after its timeout has been reported), in stream order on st.
void tc_clear_error(cudaStream_t st);

}  // namespace glasso
