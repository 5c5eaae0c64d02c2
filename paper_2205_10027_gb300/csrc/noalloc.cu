// Gradient / free-set / KKT pass for callers that cannot allocate device memory.
//
// Some hosts of this library run where cudaMalloc is not available to them: code inside a
// framework that owns every device allocation through its own pool, a stream-ordered
// runtime that forbids allocation on its hot path, or an embedding whose memory budget was
// fixed up front.  glasso_gradient_noalloc serves them: it works directly on the caller's
// dense n x n device arrays and keeps its only scratch -- one row of partial sums per matrix
// row -- in the file-scope device array below, which the library's module owns for the
// lifetime of the process on every GPU that loads it.
#include <mutex>
#include <unordered_map>
#include "../../include/glasso.h"
#include "common.cuh"

namespace glasso {
namespace {

constexpr int kSums = 4;  // ||Z||_1, ||A||_1, ||Z||_F^2, nnz(A)

// Per-row partial sums of the last call (GLASSO_NOALLOC_MAX_N * 4 doubles = 512 KB).
static __device__ __align__(256) double g_noalloc_scratch[GLASSO_NOALLOC_MAX_N * kSums];

// One block per row; scalar accesses, so any leading dimension and alignment works.
__global__ void k_gradient_rows(const double* __restrict__ S, const double* __restrict__ A,
                                const double* __restrict__ W, int64_t n, double lam,
                                double* __restrict__ X, int8_t* __restrict__ code,
                                double* __restrict__ part) {
  __shared__ double red[32];
  const int64_t i = blockIdx.x;
  double s_z = 0.0, s_a = 0.0, s_z2 = 0.0, s_nz = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const int64_t e = i * n + j;
    const double g = S[e] - W[e], a = A[e];
    const bool in_m = (a != 0.0) || (fabs(g) > lam);
    const double G = (a != 0.0) ? sgn(a) : -sgn(g);
    const double x = in_m ? g + lam * G : 0.0;
    X[e] = x;
    code[e] = in_m ? (int8_t)G : (int8_t)0;
    s_z += fabs(x);
    s_a += fabs(a);
    s_z2 += x * x;
    s_nz += (a != 0.0) ? 1.0 : 0.0;
  }
  const double t0 = block_sum(s_z, red);
  const double t1 = block_sum(s_a, red);
  const double t2 = block_sum(s_z2, red);
  const double t3 = block_sum(s_nz, red);
  if (threadIdx.x == 0) {
    part[i * kSums + 0] = t0;
    part[i * kSums + 1] = t1;
    part[i * kSums + 2] = t2;
    part[i * kSums + 3] = t3;
  }
}

// out[q] = sum over rows 0..n-1 of part[row][q], rows added in index order.
__global__ void k_sum_rows(const double* __restrict__ part, int64_t n, double* __restrict__ out) {
  __shared__ double red[32];
  for (int q = 0; q < kSums; ++q) {
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) s += part[r * kSums + q];
    const double tot = block_sum(s, red);
    if (threadIdx.x == 0) out[q] = tot;
    __syncthreads();
  }
}

// The device address of the scratch array belongs to the module instance of one CUDA
// context: after cudaDeviceReset, or under a driver-API context other than the device's
// primary one, the module is loaded again at another address.  The cached address is
// therefore keyed on the unique id of the calling thread's current context (cuCtxGetId),
// looked up through the runtime's driver entry points so that the library does not link
// libcuda directly.
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);

struct DriverFns {
  CtxGetCurrentFn get_current = nullptr;
  CtxGetIdFn get_id = nullptr;
};

const DriverFns& driver_fns() {
  static DriverFns fns;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fns.get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    else
      cudaGetLastError();
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fns.get_id = reinterpret_cast<CtxGetIdFn>(f);
    else
      cudaGetLastError();
  });
  return fns;
}

std::mutex g_setup_mu;
std::unordered_map<unsigned long long, double*> g_scratch_by_ctx;  // context id -> address

// Address of the scratch array in the calling thread's current context, looked up (once per
// context) with cudaGetSymbolAddress; nullptr on failure.
double* scratch_address() {
  const DriverFns& fns = driver_fns();
  if (!fns.get_current || !fns.get_id) return nullptr;
  // a thread with no current context gets its device's primary context (cudaSetDevice
  // initialises and binds it)
  void* ctx = nullptr;
  if (fns.get_current(&ctx) != 0 || !ctx) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    if (fns.get_current(&ctx) != 0 || !ctx) return nullptr;
  }
  unsigned long long id = 0;
  if (fns.get_id(ctx, &id) != 0) return nullptr;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  auto it = g_scratch_by_ctx.find(id);
  if (it != g_scratch_by_ctx.end()) return it->second;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return nullptr;
  }
  g_scratch_by_ctx.emplace(id, static_cast<double*>(p));
  return static_cast<double*>(p);
}

}  // namespace
}  // namespace glasso

extern "C" glasso_status glasso_gradient_noalloc(const double* S, const double* A, const double* W,
                                                 int64_t n, double lambda, double* X, int8_t* code,
                                                 double* sums, void* stream) {
  using namespace glasso;
  if (!S || !A || !W || !X || !code || !sums || n < 1 || !(lambda > 0.0)) return GLASSO_ERR_ARG;
  if (n > GLASSO_NOALLOC_MAX_N) return GLASSO_ERR_BUDGET;
  // set-up, once per context, with the caller's device current: the array's device address
  double* scratch = scratch_address();
  if (!scratch) return GLASSO_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_gradient_rows<<<(unsigned)n, 256, 0, st>>>(S, A, W, n, lambda, X, code, scratch);
  if (cudaGetLastError() != cudaSuccess) return GLASSO_ERR_CUDA;
  k_sum_rows<<<1, 256, 0, st>>>(scratch, n, sums);
  if (cudaGetLastError() != cudaSuccess) return GLASSO_ERR_CUDA;
  return GLASSO_OK;
}
