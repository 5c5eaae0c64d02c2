// Shared definitions of the libglasso CUDA sources (device helpers, launch checks).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <cmath>

namespace glasso {

// Every dense n x n operand is stored padded to np = round_up(n, kPad) rows and columns
// with leading dimension np.  The padded block of Theta is the identity, so products,
// factorisations and log-dets of the padded matrices equal those of the n x n ones.
constexpr int kPad = 128;
// Width of the Cholesky panel / diagonal blocks whose inverses the factorisation keeps.
constexpr int kNb = 64;

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Scalars the line search and stop test read back, one struct per solve.  Each field is
// written by exactly one kernel.
struct Scalars {
  double z_l1, a_l1, z_fro2, nnz;      // gradient pass
  double m_free;                       // gradient pass: entries of the free set M (n x n)
  double lin_s, lin_l1;                // trial pass: <S, dA> and sum(|At| - |A|)
  double trsa_t, l1_t, nnz_t;          // trial pass: tr(S At), ||At||_1, nnz(At)
  double logdet_t;                     // Cholesky of the trial point
  int32_t pd_t;                        // 1 while the trial factorisation has met no bad pivot
  int32_t tc_err;                      // host mirror only: the tensor-core error word
  double tr_e, tr_e2;                  // second-order log-det difference (tier 2)
  double trsa, l1;                     // objective pieces of a given matrix
  double aux[8];
  double gista[5];                     // G-ISTA trial: tr(S At), ||At||_1, nnz(At), <g, D>, ||D||_F^2
};

// Deterministic block reduction: every block writes its partial sums; one block then
// adds them in index order.  kRedBlocks partials per quantity.
constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of v over the block (blockDim.x a multiple of 32, <= 1024); the result is valid in
// thread 0.  Fixed order: lanes by xor-butterfly, then warps in index order.
__device__ __forceinline__ double block_sum(double v, double* smem32) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) smem32[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) s += smem32[w];
  }
  return s;
}

// *addr = max(*addr, v) for non-negative doubles (which order like their bit patterns).
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// -x by the sign bit (an integer operation, no FP64 instruction)
__device__ __forceinline__ double neg_f64(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}
// |x| as its bit pattern: for two such patterns integer order is the order of |x|
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

__device__ __forceinline__ double sgn(double x) { return (x > 0.0) - (x < 0.0); }

// SoftThreshold(v, c) = sign(v) max(|v| - c, 0)  (App. A.1).
__device__ __forceinline__ double soft_threshold(double v, double c) {
  const double m = fabs(v) - c;
  return m > 0.0 ? copysign(m, v) : 0.0;
}

// Conversions between FP64 and FP32 by integer arithmetic (the FP64 pipe of this part is too
// narrow for bulk conversions).  Zero and subnormal inputs give zero; values beyond the FP32
// range are not expected by the callers (factor blocks of SPD matrices) and saturate to the
// largest finite magnitude; Inf and NaN become NaN, so a PD test downstream still fails.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFF;
  if (e == 0) return 0.0;
  const uint64_t s = (uint64_t)(u >> 31) << 63;
  const uint64_t m = (uint64_t)(u & 0x7FFFFF) << 29;
  const uint64_t e64 = (e == 0xFF) ? 0x7FF : (uint64_t)(e - 127 + 1023);
  return __longlong_as_double((long long)(s | (e64 << 52) | m));
}
__device__ __forceinline__ float f64_to_f32(double d) {  // round to nearest even
  const uint64_t b = (uint64_t)__double_as_longlong(d);
  const uint32_t s = (uint32_t)(b >> 63) << 31;
  if (((b >> 52) & 0x7FF) == 0x7FF) return __uint_as_float(0x7FC00000u);  // Inf / NaN -> NaN
  const int e = (int)((b >> 52) & 0x7FF) - 1023 + 127;
  if (e <= 0) return __uint_as_float(s);
  uint64_t m = b & ((1ull << 52) - 1);
  uint32_t m23 = (uint32_t)(m >> 29);
  const uint64_t rem = m & ((1ull << 29) - 1);
  uint32_t bits = ((uint32_t)e << 23) + m23;
  if (rem > (1ull << 28) || (rem == (1ull << 28) && (m23 & 1u))) ++bits;  // carries into e
  if (e >= 0xFF || bits >= 0x7F800000u) bits = 0x7F7FFFFFu;
  return __uint_as_float(s | bits);
}

template <typename T> __device__ __forceinline__ T from_f64(double d);
template <> __device__ __forceinline__ double from_f64<double>(double d) { return d; }
template <> __device__ __forceinline__ float from_f64<float>(double d) { return f64_to_f32(d); }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return f32_to_f64(v); }

}  // namespace glasso

#include <stdexcept>
#include <string>
#include <utility>
namespace glasso {
// Host code reports failures by throwing Error; the C ABI turns it into a status code.
struct Error : std::runtime_error {
  int status;
  Error(int st, const std::string& m) : std::runtime_error(m), status(st) {}
};
}  // namespace glasso

// GLASSO_ERR_CUDA = 7 in glasso.h
#define CUDA_CHECK(expr)                                                                 \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess)                                                               \
      throw ::glasso::Error(7, std::string(#expr) + ": " + cudaGetErrorString(_e) +      \
                                   " (" + __FILE__ + ":" + std::to_string(__LINE__) + ")"); \
  } while (0)
namespace glasso {
// per-thread count of kernel launches (incremented at every checked launch)
extern thread_local int64_t tl_launches;
}
#define LAUNCH_CHECK()                    \
  do {                                    \
    ++::glasso::tl_launches;              \
    CUDA_CHECK(cudaGetLastError());       \
  } while (0)

// ---- programmatic dependent launch ---------------------------------------------------------
// The factorisation and the products are long chains of dependent launches, many of them a few
// microseconds long.  A kernel launched through launch_dependent() may be scheduled while the
// kernel before it on the stream is still running: it calls dep_wait() before its first access
// to global memory (griddepcontrol.wait: returns once the previous kernel has completed and its
// writes are visible; a no-op for a kernel launched the ordinary way), then dep_release()
// (griddepcontrol.launch_dependents), which lets the next such kernel be scheduled in turn.  So
// the launch latency and the block scheduling of each kernel overlap the end of the one before.
// GLASSO_NO_PDL=1 launches them the ordinary way.
namespace glasso {
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void dep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
bool pdl_enabled();
template <typename... Params, typename... Args>
inline void launch_dependent(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                             Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  CUDA_CHECK(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
  ++tl_launches;
}
}  // namespace glasso
