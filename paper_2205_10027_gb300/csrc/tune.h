// Autotuner of the split-precision dense products: for each product shape the factorisation
// and the step issue, which kernel and tile runs it (FP32 CUDA-core kernel, tensor-core
// 128 x 256 tiles, tensor-core 128 x 128 tiles), measured on the device and kept on disk.
#pragma once
#include <cstdint>
#include <string>
#include "gemm.h"

namespace glasso {

enum class GemmChoice : int { Default = 0, F32 = 1, TcWide = 2, TcSquare = 3 };

// What identifies a product for the tuner: its shape and structure, the precision mode and
// whether it writes in place (which excludes the CUDA-core kernel).
struct GemmShape {
  int M, N, K, krule, lower, transA, transB, inplace, precision;
  bool operator<(const GemmShape& o) const;
  static GemmShape of(const GemmArgs& a, int precision);
};

// Process-wide table per GPU model; read from / appended to the cache file named by
// GLASSO_TUNE_CACHE (default: $HOME/.cache/glasso_gemm_tune.txt; "off" keeps it in memory).
GemmChoice tuned_choice(const std::string& gpu, const GemmShape& s);
void record_choice(const std::string& gpu, const GemmShape& s, GemmChoice c, const double ms[4]);
bool tuned(const std::string& gpu, const GemmShape& s);

}  // namespace glasso
