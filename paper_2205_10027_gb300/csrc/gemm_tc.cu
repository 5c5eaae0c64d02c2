// Split-precision tensor-core GEMM (placeholder until the tcgen05 kernel lands).
#include "engine.h"
#include "gemm_tc.h"

namespace glasso {
size_t tc_scratch_bytes_for(int) { return 0; }
bool tc_gemm_supported(const GemmArgs&) { return false; }
void tc_gemm(const GemmArgs&, TcKind, void*, size_t, cudaStream_t) {
  throw Error(GLASSO_ERR_UNSUPPORTED, "tensor-core GEMM not available");
}
void refine_inverse(Engine&, const double*, cudaStream_t) {}
bool tc_available() { return false; }
}  // namespace glasso
