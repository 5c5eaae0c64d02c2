// pISTA outer loop (Algorithm 1) on the device kernels, with the line search of
// Sec. 4.3.2 and the Sec. 6 fallback step, and the single-step operations of the C ABI.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include "engine.h"
#include "gemm_tc.h"
#include "tune.h"

namespace glasso {

namespace {
constexpr double kUnitRoundoff = 1.1102230246251565e-16;  // 2^-53
constexpr double kDiffBand = 1000.0;                      // tier-2 band, in units of delta
constexpr double kFallbackFactor = 0.9;                   // Sec. 6: t <= (0.9 / cond A)^2

__global__ void k_set_int(int* p, int v) { *p = v; }

// lower triangle of src (ld) -> dense dst (n), zero upper
__global__ void k_unpad_lower(const double* __restrict__ src, int64_t ld, int64_t n, double* __restrict__ dst) {
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) dst[i * n + j] = (j <= i) ? src[i * ld + j] : 0.0;
}

// power iteration pieces: y = M x (one block per row), x = y / ||y||
__global__ void k_gemv_rows(const double* __restrict__ M, int64_t ld, int64_t n, const double* __restrict__ x,
                            double* __restrict__ y) {
  __shared__ double red[32];
  const int64_t i = blockIdx.x;
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s = fma(M[i * ld + j], x[j], s);
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) y[i] = t;
}
__global__ void k_normalize(double* __restrict__ y, int64_t n, double* __restrict__ x, double* nrm) {
  __shared__ double red[32];
  __shared__ double tot;
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s = fma(y[j], y[j], s);
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) { tot = sqrt(t); *nrm = tot; }
  __syncthreads();
  const double inv = tot > 0.0 ? 1.0 / tot : 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) x[j] = y[j] * inv;
}
__global__ void k_fill(double* x, int64_t n, double v) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) x[j] = v;
}

// ---- FP64 positive-definiteness certificate of a trial point (split-precision forms) ----
// M = X A X^T with X the trial's inverse Cholesky factor from the split-precision
// factorisation; A is PD iff M is (congruence), and M = I - X E X^T where E is the
// factorisation's backward error, so |M - I| is tiny for a PD trial and at least 1 for an
// indefinite one.  Three FP64 power steps on M - I estimate its spectral radius.

// part[b][j] = sum over rows i of block b (32 rows) of X[i][j] v[i], X lower triangular
__global__ void k_tmatvec_part(const double* __restrict__ X, int64_t ld, int64_t n, const double* __restrict__ v,
                               double* __restrict__ part) {
  const int64_t b = blockIdx.y;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int64_t r0 = b * 32, r1 = r0 + 32 < n ? r0 + 32 : n;
  double s = 0.0;
  for (int64_t i = (r0 > j ? r0 : j); i < r1; ++i) s = fma(X[i * ld + j], v[i], s);
  part[b * n + j] = s;
}
// y[j] = sum over row blocks b (from the one holding row j on) of part[b][j], in order
__global__ void k_sum_cols(const double* __restrict__ part, int64_t nb, int64_t n, double* __restrict__ y) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int64_t b = j / 32; b < nb; ++b) s += part[b * n + j];
  y[j] = s;
}
// y = X x for a lower-triangular X (one block per row, columns j <= i)
__global__ void k_gemv_lower(const double* __restrict__ X, int64_t ld, int64_t n, const double* __restrict__ x,
                             double* __restrict__ y) {
  __shared__ double red[32];
  const int64_t i = blockIdx.x;
  double s = 0.0;
  for (int64_t j = threadIdx.x; j <= i; j += blockDim.x) s = fma(X[i * ld + j], x[j], s);
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) y[i] = t;
}
// v <- (z - v) / |z - v|, *nrm = |z - v|
__global__ void k_diff_normalize(const double* __restrict__ z, int64_t n, double* __restrict__ v, double* nrm) {
  __shared__ double red[32];
  __shared__ double tot;
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double d = z[j] - v[j];
    s = fma(d, d, s);
  }
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) { tot = sqrt(t); *nrm = tot; }
  __syncthreads();
  const double inv = tot > 0.0 ? 1.0 / tot : 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) v[j] = (z[j] - v[j]) * inv;
}
// a fixed start vector with entries in [-1, 1] (a multiplicative hash of the index), scaled
// to unit length by the caller's first normalisation
__global__ void k_start_vector(double* x, int64_t n) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) {
    const uint32_t h = (uint32_t)(j + 1) * 2654435761u;
    x[j] = (double)h / 2147483648.0 - 1.0;
  }
}

// CSR capacity of the sparse sandwich: 256 nonzeros per row on average
int64_t csr_cap(int np) { return (int64_t)256 * np; }

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}
}  // namespace

// ------------------------------------------------------------------------------------------
// workspace
// ------------------------------------------------------------------------------------------
size_t Workspace::bytes_for(int np) {
  const size_t m = (size_t)np * np;
  const size_t csr = (size_t)(np + 1) * 8 + (size_t)np * 4 + (size_t)csr_cap(np) * 12;
  // 11 FP64 matrices, the int8 code, the tensor-core operand splits, the CSR, and the staging
  // buffer of a host input (up to np^2 FP64)
  return 12 * m * sizeof(double) + m + 2 * tc_scratch_bytes_for(np) + csr;
}

void Workspace::release() {
  dfree(S); dfree(A); dfree(At); dfree(W); dfree(L); dfree(Lt); dfree(X); dfree(Y); dfree(T);
  dfree(code); dfree(Li); dfree(Lti); dfree(ld_parts); dfree(parts); dfree(sc);
  dfree(pd); dfree(vmax); dfree(bad); dfree(vec);
  dfree(csr.rowptr); dfree(csr.col); dfree(csr.val); dfree(counts);
  csr.cap = 0;
  if (staging) cudaFree(staging);
  staging = nullptr;
  staging_bytes = 0;
  if (tc_scratch) cudaFree(tc_scratch);
  tc_scratch = nullptr;
  tc_scratch_bytes = 0;
  if (tc_scratch2) cudaFree(tc_scratch2);
  tc_scratch2 = nullptr;
  tc_scratch2_bytes = 0;
  if (hs) cudaFreeHost(hs);
  hs = nullptr;
  cap_np = 0;
}

void Workspace::ensure(int64_t n_new, size_t budget) {
  const int np_new = (int)round_up(n_new, kPad);
  if (np_new > cap_np) {
    const size_t need = bytes_for(np_new);
    if (budget && need > budget)
      throw Error(GLASSO_ERR_BUDGET, "problem needs " + std::to_string(need) +
                                         " bytes of device memory, budget is " +
                                         std::to_string(budget));
    release();
    const size_t m = (size_t)np_new * np_new;
    auto alloc = [&](auto*& p, size_t bytes) {
      void* q = nullptr;
      if (cudaMalloc(&q, bytes) != cudaSuccess) {
        cudaGetLastError();
        release();
        throw Error(GLASSO_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
      }
      p = reinterpret_cast<std::remove_reference_t<decltype(p)>>(q);
    };
    alloc(S, m * 8); alloc(A, m * 8); alloc(At, m * 8); alloc(W, m * 8); alloc(L, m * 8);
    alloc(Lt, m * 8); alloc(X, m * 8); alloc(Y, m * 8); alloc(T, m * 8); alloc(code, m);
    alloc(Li, m * 8); alloc(Lti, m * 8);
    alloc(ld_parts, (size_t)(np_new / kNb) * 8);
    alloc(parts, (size_t)8 * kRedBlocks * 8);
    alloc(sc, sizeof(Scalars));
    alloc(pd, sizeof(int));
    alloc(vmax, 2 * sizeof(double));
    alloc(bad, sizeof(int));
    alloc(vec, (size_t)3 * np_new * 8);
    alloc(csr.rowptr, (size_t)(np_new + 1) * 8);
    alloc(counts, (size_t)np_new * 4);
    csr.cap = csr_cap(np_new);
    alloc(csr.col, (size_t)csr.cap * 4);
    alloc(csr.val, (size_t)csr.cap * 8);
    tc_scratch_bytes = tc_scratch_bytes_for(np_new);
    if (tc_scratch_bytes) alloc(tc_scratch, tc_scratch_bytes);
    tc_scratch2_bytes = tc_scratch_bytes;
    if (tc_scratch2_bytes) alloc(tc_scratch2, tc_scratch2_bytes);
    if (cudaMallocHost((void**)&hs, sizeof(Scalars)) != cudaSuccess) {
      cudaGetLastError();
      hs = nullptr;
      release();
      throw Error(GLASSO_ERR_OOM, "cudaMallocHost failed");
    }
    cap_np = np_new;
    ++epoch;
  }
  n = n_new;
  np = (int)round_up(n_new, kPad);
  ld = np;
}

// ------------------------------------------------------------------------------------------
// launch counting and profiling
// ------------------------------------------------------------------------------------------
thread_local int64_t tl_launches = 0;
int64_t thread_launches() { return tl_launches; }

bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("GLASSO_NO_PDL");
    return !(e && e[0] == '1');
  }();
  return on;
}

cudaEvent_t Profiler::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  CUDA_CHECK(cudaEventCreate(&e));
  return e;
}
void Profiler::start() {
  for (auto& r : recs) { pool.push_back(r.a); pool.push_back(r.b); }
  recs.clear();
  on = true;
}
void Profiler::begin_rec(int cls, double work, cudaStream_t st, Rec& r) {
  r.cls = -1;
  if (!on) return;
  r.cls = cls;
  r.work = work;
  r.a = get();
  r.b = get();
  CUDA_CHECK(cudaEventRecord(r.a, st));
}
void Profiler::end_rec(Rec& r, cudaStream_t st) {
  if (r.cls < 0) return;
  CUDA_CHECK(cudaEventRecord(r.b, st));
  recs.push_back(r);
}
void Profiler::collect(glasso_profile* out) {
  std::memset(out, 0, sizeof(*out));
  for (auto& r : recs) {
    CUDA_CHECK(cudaEventSynchronize(r.b));
    float ms = 0.f;
    CUDA_CHECK(cudaEventElapsedTime(&ms, r.a, r.b));
    out->ms[r.cls] += ms;
    out->work[r.cls] += r.work;
    out->launches[r.cls] += 1;
  }
  for (auto& r : recs) { pool.push_back(r.a); pool.push_back(r.b); }
  recs.clear();
  on = false;
}
Profiler::~Profiler() {
  for (auto& r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : pool) cudaEventDestroy(e);
}

namespace {
// algorithmic FLOPs of one product with the structure the call declares; a dimension that
// spans the whole padded matrix (np) counts as the problem's n
double gemm_flops(const GemmArgs& a, int np, int64_t n) {
  auto alg = [&](int d) { return d == np ? (double)n : (double)d; };
  const double M = alg(a.M), N = alg(a.N), K = alg(a.K);
  switch (a.krule) {
    case KR_LO_COL: return M * N * (N + 1.0);                 // B lower triangular (K = N)
    case KR_HI_ROW: return N * M * (M + 1.0);                 // A lower triangular (K = M)
    case KR_LO_ROW: return K * K * K / 3.0 + K * K;           // X^T X, X lower, lower output
    case KR_HI_COL: return M * N * (N + 1.0);                 // op(B) upper triangular (K = N)
    default: return a.lower ? M * (M + 1.0) * K : 2.0 * M * N * K;
  }
}
int prof_class(GemmRole r) {
  switch (r) {
    case GemmRole::Sandwich: return GLASSO_PROF_SANDWICH;
    case GemmRole::Trailing: return GLASSO_PROF_TRAILING;
    case GemmRole::Panel: return GLASSO_PROF_PANEL;
    case GemmRole::Inverse: return GLASSO_PROF_INVERSE;
    default: return GLASSO_PROF_REFINE;
  }
}
}  // namespace

// ------------------------------------------------------------------------------------------
// engine
// ------------------------------------------------------------------------------------------
Engine::Engine(const glasso_config& cfg) : cfg_(cfg) {
  CUDA_CHECK(cudaSetDevice(cfg.device));
  {
    cudaDeviceProp prop;
    CUDA_CHECK(cudaGetDeviceProperties(&prop, cfg.device));
    gpu_name_ = prop.name;
  }
  // GLASSO_NO_GRAPHS=1 runs every factorisation launch by launch (for per-kernel profiling)
  const char* ng = std::getenv("GLASSO_NO_GRAPHS");
  use_graphs_ = !(ng && ng[0] == '1');
  // width of the right-looking panels of the factorisation (GLASSO_PANEL overrides; 0, the
  // default, = recursive halving over the whole matrix, which measured faster on GB300:
  // its trailing updates have K up to n/2 instead of the panel width)
  const char* pw = std::getenv("GLASSO_PANEL");
  panel_ = pw ? std::atoi(pw) : 0;
  if (panel_ < 0 || panel_ % kPad) panel_ = 0;
  ws.device = cfg.device;
  if (cfg.stream) {
    stream_ = (cudaStream_t)cfg.stream;
  } else {
    CUDA_CHECK(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
    own_stream_ = true;
  }
}

Engine::~Engine() {
  cudaSetDevice(cfg_.device);
  if (stream_) cudaStreamSynchronize(stream_);
  drop_graphs();
  if (cap_stream_) cudaStreamDestroy(cap_stream_);
  if (wait_ev_) cudaEventDestroy(wait_ev_);
  if (side_.st) cudaStreamDestroy(side_.st);
  if (side_.fork) cudaEventDestroy(side_.fork);
  if (side_.join) cudaEventDestroy(side_.join);
  if (t2_.st) {
    cudaStreamSynchronize(t2_.st);
    cudaStreamDestroy(t2_.st);
  }
  if (t2_.fork) cudaEventDestroy(t2_.fork);
  if (t2_.join) cudaEventDestroy(t2_.join);
  if (fac_.st) {
    cudaStreamSynchronize(fac_.st);
    cudaStreamDestroy(fac_.st);
  }
  if (fac_.join) cudaEventDestroy(fac_.join);
  ws.release();
  if (own_stream_ && stream_) cudaStreamDestroy(stream_);
}

void Engine::gemm(const GemmArgs& a, GemmRole role, cudaStream_t st) {
  Profiler::Rec rec;
  prof.begin_rec(prof_class(role), gemm_flops(a, ws.np, ws.n), st, rec);
  const bool mixed = cfg_.precision != GLASSO_FP64;
  const GemmChoice ch =
      mixed && cfg_.autotune ? tuned_choice(gpu_name_, GemmShape::of(a, cfg_.precision)) : GemmChoice::Default;
  if (mixed && gemm_f32_supported(a) && (ch == GemmChoice::Default || ch == GemmChoice::F32)) {
    gemm_f32(a, st);
  } else if (mixed && tc_gemm_supported(a)) {
    // products on the factorisation's side stream split their operands into a scratch of
    // their own (they run beside products on the main stream)
    const bool on_side = side_.st && st == side_.st;
    const TcTile tile = ch == GemmChoice::TcSquare ? TcTile::Square : ch == GemmChoice::TcWide ? TcTile::Wide
                                                                                               : TcTile::Default;
    tc_gemm(a, cfg_.precision == GLASSO_MIXED_BF16X3 ? TcKind::BF16x3 : TcKind::TF32x3,
            on_side ? ws.tc_scratch2 : ws.tc_scratch, on_side ? ws.tc_scratch2_bytes : ws.tc_scratch_bytes, st, tile);
  } else {
    // the FP64 kernel reads its operands tile by tile while writing C: no aliasing allowed
    if (a.C == a.A || a.C == a.B) throw Error(GLASSO_ERR_ARG, "in-place product on the FP64 kernel");
    gemm_f64(a, 1, st);
  }
  prof.end_rec(rec, st);
}

void Engine::autotune() {
  // every padded size this engine solves at is covered before its first solve, so that a
  // shape's kernel never changes between solves of a process (results stay reproducible)
  if (cfg_.precision == GLASSO_FP64 || !cfg_.autotune || tuned_np_ == ws.np) return;
  tuned_np_ = ws.np;
  const int np = ws.np;
  std::vector<GemmArgs> shapes;
  const LeafKind kind = cfg_.fp32_panels ? LeafKind::F32 : LeafKind::F64Chol;
  factorisation_products(np, true, kind, shapes);
  {
    // the step's own products: W = X^T X and the refinement W R (lower), the dense sandwich
    // (dummy pointers: only their equality, which marks shared or in-place operands, counts)
    const double* P = reinterpret_cast<const double*>(16);
    const double* Q = reinterpret_cast<const double*>(32);
    double* C = reinterpret_cast<double*>(48);
    GemmArgs w = gemm_args(P, np, 1, P, np, 0, C, np, np, np, np, 1.0, 0.0);
    w.lower = 1;
    w.krule = KR_LO_ROW;
    shapes.push_back(w);
    GemmArgs r = gemm_args(P, np, 0, Q, np, 0, C, np, np, np, np, 1.0, 0.0);
    r.lower = 1;
    shapes.push_back(r);
    GemmArgs d = gemm_args(P, np, 0, Q, np, 0, C, np, np, np, np, 1.0, 0.0);
    shapes.push_back(d);
  }
  cudaStream_t st = stream_;
  const size_t mat = sizeof(double) * ws.ld * ws.np;
  CUDA_CHECK(cudaMemsetAsync(ws.Y, 0, mat, st));
  CUDA_CHECK(cudaMemsetAsync(ws.T, 0, mat, st));
  CUDA_CHECK(cudaMemsetAsync(ws.X, 0, mat, st));
  cudaEvent_t e0, e1;
  CUDA_CHECK(cudaEventCreate(&e0));
  CUDA_CHECK(cudaEventCreate(&e1));
  const TcKind tk = cfg_.precision == GLASSO_MIXED_BF16X3 ? TcKind::BF16x3 : TcKind::TF32x3;
  std::vector<GemmShape> done;
  for (const GemmArgs& proto : shapes) {
    const GemmShape key = GemmShape::of(proto, cfg_.precision);
    if (tuned(gpu_name_, key)) continue;
    bool seen = false;
    for (const auto& d : done) seen = seen || (!(d < key) && !(key < d));
    if (seen) continue;
    done.push_back(key);
    // scratch operands with the prototype's aliasing: A in Y, B in T, C in X (or A / B)
    GemmArgs a = proto;
    a.A = ws.Y;
    a.B = (proto.B == proto.A) ? ws.Y : ws.T;
    a.C = (proto.C == proto.A) ? ws.Y : (proto.C == proto.B && proto.B != proto.A) ? ws.T : ws.X;
    a.lda = a.ldb = a.ldc = ws.ld;
    a.flag = nullptr;
    double ms[4] = {0, INFINITY, INFINITY, INFINITY};
    for (int cand = 1; cand <= 3; ++cand) {
      if (cand == 1 && !gemm_f32_supported(a)) continue;
      if (cand > 1 && !tc_gemm_supported(a)) continue;
      auto run = [&] {
        if (cand == 1) gemm_f32(a, st);
        else tc_gemm(a, tk, ws.tc_scratch, ws.tc_scratch_bytes, st, cand == 2 ? TcTile::Wide : TcTile::Square);
      };
      run();  // warm
      CUDA_CHECK(cudaEventRecord(e0, st));
      for (int r = 0; r < 3; ++r) run();
      CUDA_CHECK(cudaEventRecord(e1, st));
      CUDA_CHECK(cudaEventSynchronize(e1));
      float t = 0.f;
      CUDA_CHECK(cudaEventElapsedTime(&t, e0, e1));
      ms[cand] = t / 3.0;
    }
    int best = 0;
    for (int cand = 1; cand <= 3; ++cand)
      if (ms[cand] < INFINITY && (best == 0 || ms[cand] < ms[best])) best = cand;
    if (best) record_choice(gpu_name_, key, (GemmChoice)best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

GemmFn Engine::gemm_fn() {
  return [this](const GemmArgs& a, GemmRole r, cudaStream_t st) { gemm(a, r, st); };
}

// Wait for the work queued on st: cudaStreamSynchronize, or, for engines that share the host
// cores with many others (the slots of glasso_solve_batch and of the serving loop), a
// blocking-sync event, so that the waiting thread sleeps instead of spinning on a core.
cudaError_t Engine::wait_stream(cudaStream_t st) {
  if (!blocking_sync_) return cudaStreamSynchronize(st);
  if (!wait_ev_) {
    const cudaError_t e = cudaEventCreateWithFlags(&wait_ev_, cudaEventBlockingSync | cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  const cudaError_t e = cudaEventRecord(wait_ev_, st);
  if (e != cudaSuccess) return e;
  return cudaEventSynchronize(wait_ev_);
}

void Engine::sync_scalars() {
  CUDA_CHECK(cudaMemcpyAsync(ws.hs, ws.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, stream_));
  // the tensor-core error word rides on the same wait
  const int* err = cfg_.precision != GLASSO_FP64 ? tc_error_word() : nullptr;
  if (err) CUDA_CHECK(cudaMemcpyAsync(&ws.hs->tc_err, err, sizeof(int), cudaMemcpyDeviceToHost, stream_));
  CUDA_CHECK(wait_stream(stream_));
  if (err && ws.hs->tc_err) {
    tc_clear_error(stream_);  // reported once; the kernels that timed out left without writing
    CUDA_CHECK(wait_stream(stream_));
    throw Error(GLASSO_ERR_TIMEOUT, "a tensor-core GEMM timed out waiting on its pipeline");
  }
}

// Copy a caller matrix (n x n, leading dim n) into dst (padded), mirroring its lower
// triangle; with check_s the S checks of glasso_solve are applied.
void Engine::load_matrix(const void* src, bool f32, bool on_device, int64_t n, double* dst,
                         bool check_s) {
  const size_t elt = f32 ? 4 : 8;
  const size_t bytes = (size_t)n * n * elt;
  const void* dsrc = src;
  if (!on_device) {
    if (ws.staging_bytes < bytes) {
      if (ws.staging) cudaFree(ws.staging);
      ws.staging = nullptr;
      ws.staging_bytes = 0;
      if (cudaMalloc(&ws.staging, bytes) != cudaSuccess) {
        cudaGetLastError();
        throw Error(GLASSO_ERR_OOM, "staging allocation failed");
      }
      ws.staging_bytes = bytes;
    }
    CUDA_CHECK(cudaMemcpyAsync(ws.staging, src, bytes, cudaMemcpyHostToDevice, stream_));
    dsrc = ws.staging;
  }
  CUDA_CHECK(cudaMemsetAsync(ws.vmax, 0, 2 * sizeof(double), stream_));
  CUDA_CHECK(cudaMemsetAsync(ws.bad, 0, sizeof(int), stream_));
  load_symmetric(dsrc, f32, n, dst, ws.ld, ws.np, ws.vmax, ws.bad, stream_);
  if (check_s) {
    double vm[2];
    int bad = 0;
    CUDA_CHECK(cudaMemcpyAsync(vm, ws.vmax, sizeof(vm), cudaMemcpyDeviceToHost, stream_));
    CUDA_CHECK(cudaMemcpyAsync(&bad, ws.bad, sizeof(int), cudaMemcpyDeviceToHost, stream_));
    CUDA_CHECK(wait_stream(stream_));
    if (bad) throw Error(GLASSO_ERR_NONFINITE, "S holds non-finite entries or a negative diagonal");
    if (vm[0] > 1e-12 * vm[1])
      throw Error(GLASSO_ERR_NOT_SYMMETRIC, "S is not symmetric: max |S_ij - S_ji| = " +
                                                std::to_string(vm[0]));
  }
}

// Cholesky factor and its inverse of the matrix held in L (overwritten), PD flag and log det
// into the scalars.
void Engine::factor_direct(double* L, double* Li, cudaStream_t st) {
  k_set_int<<<1, 1, 0, st>>>(ws.pd, 1);
  LAUNCH_CHECK();
  const bool split = cfg_.precision != GLASSO_FP64;
  const LeafKind kind = !split ? LeafKind::F64 : cfg_.fp32_panels ? LeafKind::F32 : LeafKind::F64Chol;
  if (split && !side_.st) {
    CUDA_CHECK(cudaStreamCreateWithFlags(&side_.st, cudaStreamNonBlocking));
    CUDA_CHECK(cudaEventCreateWithFlags(&side_.fork, cudaEventDisableTiming));
    CUDA_CHECK(cudaEventCreateWithFlags(&side_.join, cudaEventDisableTiming));
  }
  // profiling keeps the products in stream order (their events are recorded on one stream)
  cholesky_inverse(L, Li, ws.ld, ws.np, ws.T, ws.ld_parts, ws.pd, &ws.sc->logdet_t, gemm_fn(), st, split, kind,
                   panel_, split && !prof.on ? &side_ : nullptr);
  CUDA_CHECK(cudaMemcpyAsync(&ws.sc->pd_t, ws.pd, sizeof(int), cudaMemcpyDeviceToDevice, st));
}

void Engine::drop_graphs() {
  for (auto& g : fgraphs_) cudaGraphExecDestroy(g.second.exec);
  fgraphs_.clear();
  fseen_.clear();
}

// The recursive factorisation is a fixed sequence of a few thousand launches for a given
// size and pair of buffers, so from its second use it is replayed as a captured CUDA graph
// (captured on a private stream, launched on the engine's stream).  Profiling runs it
// directly so that every product gets its own events.
void Engine::factor(double* L, double* Li, cudaStream_t st) {
  // profiling times a replayed graph as one FACTOR record (its launches cannot carry events);
  // before a graph exists the direct launches are recorded class by class
  Profiler::Rec rec;
  const double np3 = (double)ws.n * ws.n * ws.n;  // algorithmic: n^3 / 3 + n^3 / 3 on n
  if (graph_epoch_ != ws.epoch) {
    drop_graphs();
    graph_epoch_ = ws.epoch;
  }
  if (!use_graphs_) {
    prof.begin_rec(GLASSO_PROF_FACTOR, 2.0 * np3 / 3.0, st, rec);
    factor_direct(L, Li, st);
    prof.end_rec(rec, st);
    return;
  }
  const bool graphed = fgraphs_.count(GraphKey{L, Li, ws.np}) != 0;
  if (graphed) prof.begin_rec(GLASSO_PROF_FACTOR, 2.0 * np3 / 3.0, st, rec);
  factor_graphed(L, Li, st);
  if (graphed) prof.end_rec(rec, st);
}

void Engine::factor_graphed(double* L, double* Li, cudaStream_t st) {
  if (graph_epoch_ != ws.epoch) {
    drop_graphs();
    graph_epoch_ = ws.epoch;
  }
  const GraphKey key{L, Li, ws.np};
  auto it = fgraphs_.find(key);
  if (it == fgraphs_.end()) {
    if (++fseen_[key] < 2) {  // the first use runs directly (one-time set-up happens there)
      factor_direct(L, Li, st);
      return;
    }
    if (!cap_stream_) CUDA_CHECK(cudaStreamCreateWithFlags(&cap_stream_, cudaStreamNonBlocking));
    const int64_t l0 = tl_launches;
    const bool prof_on = prof.on;
    prof.on = false;  // no event records inside the capture
    CUDA_CHECK(cudaStreamBeginCapture(cap_stream_, cudaStreamCaptureModeThreadLocal));
    cudaGraph_t g = nullptr;
    try {
      factor_direct(L, Li, cap_stream_);
    } catch (...) {
      cudaStreamEndCapture(cap_stream_, &g);
      if (g) cudaGraphDestroy(g);
      tl_launches = l0;
      prof.on = prof_on;
      throw;
    }
    prof.on = prof_on;
    CUDA_CHECK(cudaStreamEndCapture(cap_stream_, &g));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    CUDA_CHECK(e);
    it = fgraphs_.emplace(key, FactorGraph{exec, tl_launches - l0}).first;
    tl_launches = l0;
  }
  CUDA_CHECK(cudaGraphLaunch(it->second.exec, st));
  tl_launches += it->second.launches;
}

// W = A^{-1} for the accepted factor (ws.L, Li): completes Li = L^{-1} from its diagonal panel
// blocks, then W = Li^T Li.
void Engine::compute_inverse(double* Li, cudaStream_t st) {
  if (panel_ > 0) inverse_merge(ws.L, Li, ws.ld, ws.np, ws.T, panel_, gemm_fn(), st);
  inverse_from_inverse_factor(Li, ws.ld, ws.np, ws.W, gemm_fn(), st);
  {
    Profiler::Rec rec;
    prof.begin_rec(GLASSO_PROF_AUX, 8.0 * (double)ws.n * (double)ws.n, st, rec);
    mirror_lower(ws.W, ws.ld, ws.np, st);
    prof.end_rec(rec, st);
  }
  if (cfg_.precision != GLASSO_FP64) refine_inverse(st);
}

// Mixed mode: Newton-Schulz sweeps W <- W + W R, R = I - A W formed exactly in FP64 from the
// sparse rows of A.  In exact arithmetic a sweep squares R; the correction product W R runs
// on the tensor cores and adds about c |R| (c = 3e-5 for BF16x3, 1e-6 for TF32x3 products).
// Sweeps stop once max |R| is measured below 1e-9, or is predicted below it after a sweep
// (|R|^2 + c |R|, with c an upper estimate of the correction product's relative error); at
// most three sweeps.  That keeps g = S - W, the stop test and the tier-2
// log-det difference at FP64-level accuracy for the decisions they feed.
void Engine::refine_inverse(cudaStream_t st) {
  const int np = ws.np;
  const int64_t ld = ws.ld;
  double* rmax = &ws.sc->aux[0];
  const double nn = (double)ws.n * (double)ws.n;  // algorithmic bytes count the n x n block
  const double c = cfg_.precision == GLASSO_MIXED_BF16X3 ? 3e-5 : 1e-6;
  for (int sweep = 0; sweep < 3; ++sweep) {
    {
      // the residual is a sparse-dense product: through the CSR of A when it fits
      const bool csr = ensure_csr_of_A(st);
      Profiler::Rec rec;
      // FP64-pipe bound: 2 nnz(A) FLOPs per column of W
      prof.begin_rec(GLASSO_PROF_RESIDUAL, 2.0 * (double)csr_nnz_ * (double)np, st, rec);
      if (csr) {
        CUDA_CHECK(cudaMemsetAsync(rmax, 0, sizeof(double), st));
        spmm_residual(ws.csr, ws.W, ld, ws.T, ld, ws.n, np, rmax, st);
      } else {
        inverse_residual(ws.A, ws.W, ld, ws.n, np, ws.T, rmax, st);
      }
      prof.end_rec(rec, st);
    }
    double h = 0.0;
    CUDA_CHECK(cudaMemcpyAsync(&h, rmax, sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(wait_stream(st));
    ws.hs->aux[1 + sweep] = h;
    if (h < 1e-9) break;
    GemmArgs g = gemm_args(ws.W, ld, 0, ws.T, ld, 0, ws.Y, ld, np, np, np, 1.0, 0.0);
    g.lower = 1;
    gemm(g, GemmRole::Refine, st);
    {
      Profiler::Rec rec;
      prof.begin_rec(GLASSO_PROF_AUX, 16.0 * nn, st, rec);
      add_lower_mirror(ws.W, ws.Y, ld, np, st);
      prof.end_rec(rec, st);
    }
    if (h * h + c * h < 1e-9) break;  // the sweep just made has brought it below 1e-9
  }
}

bool Engine::ensure_csr_of_A(cudaStream_t st) {
  if (csr_valid_) return true;
  csr_rowptr(ws.A, nullptr, ws.ld, ws.n, ws.np, ws.counts, ws.csr.rowptr, st);
  int64_t nnz = 0;
  CUDA_CHECK(cudaMemcpyAsync(&nnz, ws.csr.rowptr + ws.np, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CUDA_CHECK(wait_stream(st));
  csr_nnz_ = nnz;
  if (nnz > ws.csr.cap) return false;
  csr_fill(ws.A, nullptr, ws.ld, ws.n, ws.np, ws.csr, st);
  csr_valid_ = true;
  return true;
}

// log det At - log det A = log det(I + E) = tr E - tr E^2 / 2 + O(|E|^3), E similar to
// Q = (At - A) W; (At - A) is nonzero only where the step changed an entry, so Q is a sparse-
// dense product (through a CSR of the difference when at most nnz_bound entries fit).
void Engine::logdet_terms(double nnz_bound, cudaStream_t st, double* Q) {
  const int64_t n = st_.n;
  if (!Q) Q = ws.T;
  Profiler::Rec rec;
  prof.begin_rec(GLASSO_PROF_LOGDET2, 32.0 * (double)n * (double)n, st, rec);
  if (nnz_bound <= (double)ws.csr.cap) {
    csr_valid_ = false;  // the CSR buffers now hold the difference
    csr_rowptr(ws.At, ws.A, ws.ld, n, ws.np, ws.counts, ws.csr.rowptr, st);
    csr_fill(ws.At, ws.A, ws.ld, n, ws.np, ws.csr, st);
    spmm(ws.csr, ws.W, ws.ld, Q, ws.ld, ws.np, false, false, st);
    trace_terms(Q, ws.ld, n, ws.np, ws.parts, &ws.sc->tr_e, st);
  } else {
    logdet_difference_terms(ws.At, ws.A, ws.W, ws.ld, n, ws.np, Q, ws.parts, &ws.sc->tr_e, st);
  }
  prof.end_rec(rec, st);
}

bool Engine::sparse_sandwich(double nnz) const {
  if (cfg_.products == GLASSO_PRODUCTS_DENSE || nnz > (double)ws.csr.cap) return false;
  if (cfg_.products == GLASSO_PRODUCTS_SPARSE || cfg_.precision == GLASSO_FP64) return true;
  const double n = (double)ws.n;
  return nnz <= n * std::max(16.0, n / 256.0);
}

// Y = lower(A X A).  Sparse: T = (A X)^T = X A from the CSR of A, then Y = A T.  Dense:
// T = A X, then Y = T A on the lower triangle (Y is symmetric).
void Engine::sandwich(double nnz, cudaStream_t st) {
  const int np = ws.np;
  if (sparse_sandwich(nnz) && ensure_csr_of_A(st)) {
    Profiler::Rec rec;
    prof.begin_rec(GLASSO_PROF_SPMM, 3.0 * nnz * (double)np, st, rec);
    spmm(ws.csr, ws.X, ws.ld, ws.T, ws.ld, np, true, false, st);
    spmm(ws.csr, ws.T, ws.ld, ws.Y, ws.ld, np, false, true, st);
    prof.end_rec(rec, st);
    return;
  }
  GemmArgs a = gemm_args(ws.A, ws.ld, 0, ws.X, ws.ld, 0, ws.T, ws.ld, np, np, np, 1.0, 0.0);
  gemm(a, GemmRole::Sandwich, st);
  GemmArgs b = gemm_args(ws.T, ws.ld, 0, ws.A, ws.ld, 0, ws.Y, ws.ld, np, np, np, 1.0, 0.0);
  b.lower = 1;
  gemm(b, GemmRole::Sandwich, st);
}

double Engine::power_lambda_max(const double* M, cudaStream_t st, int iters) {
  const int64_t n = ws.n;
  double* x = ws.vec;
  double* y = ws.vec + ws.np;
  double* nrm = ws.vec + 2 * ws.np;
  k_fill<<<(int)((n + 255) / 256), 256, 0, st>>>(x, n, 1.0 / std::sqrt((double)n));
  LAUNCH_CHECK();
  for (int it = 0; it < iters; ++it) {
    k_gemv_rows<<<(int)n, 256, 0, st>>>(M, ws.ld, n, x, y);
    LAUNCH_CHECK();
    k_normalize<<<1, 1024, 0, st>>>(y, n, x, nrm);
    LAUNCH_CHECK();
  }
  double h = 0.0;
  CUDA_CHECK(cudaMemcpyAsync(&h, nrm, sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_CHECK(wait_stream(st));
  return h;
}

// Spectral radius estimate of M - I, M = X A X^T (X = the trial's inverse factor Lti, A the
// trial point At), from three FP64 power steps; see k_tmatvec_part.  Uses ws.T as scratch.
double Engine::congruence_radius(cudaStream_t st) {
  const int64_t n = ws.n, ld = ws.ld;
  const int64_t nb = (n + 31) / 32;
  double* v = ws.vec;
  double* u = ws.vec + ws.np;
  double* z = ws.vec + 2 * ws.np;
  double* nrm = &ws.sc->aux[4];
  const unsigned g = (unsigned)((n + 255) / 256);
  k_start_vector<<<g, 256, 0, st>>>(z, n);
  LAUNCH_CHECK();
  CUDA_CHECK(cudaMemsetAsync(v, 0, sizeof(double) * n, st));
  k_diff_normalize<<<1, 1024, 0, st>>>(z, n, v, nrm);  // v = z / |z|
  LAUNCH_CHECK();
  for (int it = 0; it < 3; ++it) {
    k_tmatvec_part<<<dim3(g, (unsigned)nb), 256, 0, st>>>(ws.Lti, ld, n, v, ws.T);   // X^T v
    LAUNCH_CHECK();
    k_sum_cols<<<g, 256, 0, st>>>(ws.T, nb, n, u);
    LAUNCH_CHECK();
    k_gemv_rows<<<(unsigned)n, 256, 0, st>>>(ws.At, ld, n, u, z);                     // A X^T v
    LAUNCH_CHECK();
    k_gemv_lower<<<(unsigned)n, 256, 0, st>>>(ws.Lti, ld, n, z, u);                   // X A X^T v
    LAUNCH_CHECK();
    k_diff_normalize<<<1, 1024, 0, st>>>(u, n, v, nrm);                               // (M - I) v
    LAUNCH_CHECK();
  }
  double h = 0.0;
  CUDA_CHECK(cudaMemcpyAsync(&h, nrm, sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_CHECK(wait_stream(st));
  return h;
}

void Engine::begin(const void* Sin, bool s_f32, bool s_on_device, int64_t n, double lam,
                   const double* theta0) {
  st_ = SolveState{};
  st_.t_begin = std::chrono::steady_clock::now();
  st_.launches_begin = tl_launches;
  CUDA_CHECK(cudaSetDevice(cfg_.device));
  ws.ensure(n, cfg_.hbm_budget_bytes);
  autotune();
  st_.launches_begin = tl_launches;
  csr_valid_ = false;
  w_valid_ = false;
  cudaStream_t st = stream_;
  const int np = ws.np;
  const int64_t ld = ws.ld;
  const size_t mat = sizeof(double) * ld * np;
  Scalars& h = *ws.hs;
  load_matrix(Sin, s_f32, s_on_device, n, ws.S, true);
  if (cfg_.standardize) {
    int bad = 0;
    CUDA_CHECK(cudaMemsetAsync(ws.bad, 0, sizeof(int), st));
    standardize(ws.S, ld, n, ws.vec, ws.bad, st);
    CUDA_CHECK(cudaMemcpyAsync(&bad, ws.bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(wait_stream(st));
    if (bad) throw Error(GLASSO_ERR_ARG, "standardize needs every S_ii > 0");
  }
  CUDA_CHECK(cudaMemsetAsync(ws.code, 0, (size_t)ld * np, st));
  CUDA_CHECK(cudaMemsetAsync(ws.X, 0, mat, st));
  if (theta0) {
    load_matrix(theta0, false, s_on_device, n, ws.A, false);
    pad_identity(ws.A, ld, n, np, st);
  } else {
    CUDA_CHECK(cudaMemsetAsync(ws.A, 0, mat, st));
    init_diag(ws.S, ld, n, np, lam, ws.A, st);
  }
  // factor the start point
  CUDA_CHECK(cudaMemcpyAsync(ws.Lt, ws.A, mat, cudaMemcpyDeviceToDevice, st));
  factor(ws.Lt, ws.Lti, st);
  objective_terms(ws.S, ws.A, ld, n, ws.parts, &ws.sc->trsa, st);
  sync_scalars();
  if (!h.pd_t) throw Error(GLASSO_ERR_NOT_PD, "the start point is not positive definite");
  std::swap(ws.L, ws.Lt);
  std::swap(ws.Li, ws.Lti);
  st_.active = true;
  st_.on_device = s_on_device;
  st_.n = n;
  st_.lam = lam;
  st_.ld_A = h.logdet_t;
  st_.trsa = h.trsa;
  st_.l1 = h.l1;
  st_.F = -st_.ld_A + st_.trsa + lam * st_.l1;
}

// One iteration of the plain proximal gradient method (glasso_method GISTA; Sec. 2.2, H = I):
// the gradient and stop test as in pISTA, then candidates ST(A - t g, t lam) from
// t = min(1, max(2 t_last, t_safe)), halved until the candidate is PD and
// f(At) <= f(A) + <g, D> + ||D||^2 / (2t) (f = -log det + tr(S .)), but not below
// t_safe = lambda_min(A)^2 / 2 = 1 / (2 lambda_max(W)^2); if no candidate above t_safe
// passes, the step is t_safe, halved further only while the candidate is not PD.
int Engine::gista_step(double tol, int max_iter, bool keep_trace) {
  cudaStream_t st = stream_;
  const int np = ws.np;
  const int64_t ld = ws.ld, n = st_.n;
  const double lam = st_.lam;
  Scalars& h = *ws.hs;
  SolveOut& out = st_.out;
  csr_valid_ = false;
  if (!w_valid_) compute_inverse(ws.Li, st);
  w_valid_ = true;
  {
    Profiler::Rec rec;
    prof.begin_rec(GLASSO_PROF_GRADIENT, 33.0 * (double)n * (double)n, st, rec);
    gradient(ws.S, ws.W, ws.A, ld, n, lam, ws.X, ws.code, ld, ws.parts, &ws.sc->z_l1, st);
    prof.end_rec(rec, st);
  }
  sync_scalars();
  out.r = h.z_l1 / h.a_l1;
  out.z_fro = std::sqrt(h.z_fro2);
  out.nnz = h.nnz;
  if (out.r <= tol) return GLASSO_OK;
  if (st_.k >= max_iter) return GLASSO_MAX_ITER;
  const double lmax_w = power_lambda_max(ws.W, st, 60);
  const double t_safe = 0.5 / (lmax_w * lmax_w);
  const double f = -st_.ld_A + st_.trsa;
  double t = std::min(1.0, std::max(2.0 * st_.t_last, t_safe));
  int trials = 0;
  bool accepted = false;
  auto candidate = [&](double tt) -> bool {  // PD
    {
      Profiler::Rec rec;
      prof.begin_rec(GLASSO_PROF_TRIAL, 32.0 * (double)n * (double)n, st, rec);
      gista_trial(ws.A, ws.W, ws.S, ld, n, np, lam, tt, ws.At, ws.Lt, ws.parts, ws.sc->gista, st);
      prof.end_rec(rec, st);
    }
    factor(ws.Lt, ws.Lti, st);
    sync_scalars();
    ++trials;
    return h.pd_t != 0;
  };
  while (t > t_safe) {
    if (candidate(t)) {
      const double fn = -h.logdet_t + h.gista[0];
      if (fn <= f + h.gista[3] + h.gista[4] / (2.0 * t)) { accepted = true; break; }
    }
    t *= 0.5;
  }
  if (!accepted) {
    t = t_safe;
    while (t > 1e-300) {
      if (candidate(t)) { accepted = true; break; }
      t *= 0.5;
    }
  }
  out.trials += trials;
  out.step_t = t;
  out.step_dF = 0.0;
  out.step_tier = 1;
  out.step_fallback = 0;
  if (keep_trace) out.trace.push_back(IterRecord{st_.k, trials, 1, st_.F, out.r, out.z_fro, out.nnz, t, 0.0});
  if (!accepted) return GLASSO_LINESEARCH_STALL;
  std::swap(ws.A, ws.At);
  std::swap(ws.L, ws.Lt);
  std::swap(ws.Li, ws.Lti);
  w_valid_ = false;
  st_.ld_A = h.logdet_t;
  st_.trsa = h.gista[0];
  st_.l1 = h.gista[1];
  st_.F = -st_.ld_A + st_.trsa + lam * st_.l1;
  st_.t_last = t;
  ++st_.k;
  return -1;
}

int Engine::step(double tol, int max_iter, bool keep_trace) {
  if (!st_.active) throw Error(GLASSO_ERR_ARG, "no solve in progress (call glasso_begin)");
  if (cfg_.method == GLASSO_METHOD_GISTA) return gista_step(tol, max_iter, keep_trace);
  cudaStream_t st = stream_;
  const int np = ws.np;
  const int64_t ld = ws.ld, n = st_.n;
  const double lam = st_.lam;
  Scalars& h = *ws.hs;
  SolveOut& out = st_.out;
  const double shrink = cfg_.shrink > 0 && cfg_.shrink < 1 ? cfg_.shrink : 0.5;
  const double t_min = cfg_.t_min > 0 ? cfg_.t_min : 1e-4;

  csr_valid_ = false;  // A changed since the last step (or the CSR holds a difference)
  if (!w_valid_) compute_inverse(ws.Li, st);
  w_valid_ = true;
  {
    Profiler::Rec rec;
    prof.begin_rec(GLASSO_PROF_GRADIENT, 33.0 * (double)n * (double)n, st, rec);
    gradient(ws.S, ws.W, ws.A, ld, n, lam, ws.X, ws.code, ld, ws.parts, &ws.sc->z_l1, st);
    prof.end_rec(rec, st);
  }
  sync_scalars();
  out.r = h.z_l1 / h.a_l1;
  out.z_fro = std::sqrt(h.z_fro2);
  out.nnz = h.nnz;
  if (out.r <= tol) return GLASSO_OK;
  if (st_.k >= max_iter) return GLASSO_MAX_ITER;
  sandwich(h.nnz, st);
  // rounding allowance of F: FP64 unit roundoff, or the split products' for the mixed modes
  // (whose Cholesky trailing updates carry about 2^-21 relative error)
  const double u = cfg_.precision == GLASSO_FP64 ? kUnitRoundoff : std::ldexp(1.0, -21);
  const double delta = 16.0 * u * (std::fabs(st_.ld_A) + std::fabs(st_.trsa) + lam * st_.l1);
  double t = 1.0, dF = INFINITY;
  int trials = 0, tier = 1;
  bool accepted = false;
  // Once a line search has needed the second-order difference (the split-precision forms near
  // convergence, where the decrease is below the rounding allowance), it is formed for every
  // trial on a second stream while the trial point is factored: it needs only At, A and W, and
  // the factorisation leaves most of the GPU idle.  Its product goes to X (free once the
  // sandwich has used it) instead of the factorisation's scratch T; supp(At - A) lies in the
  // free set M, so |M| bounds the difference's CSR.
  static const bool spec_off = [] {  // GLASSO_NO_SPEC_TIER2=1: form it only when needed, in line
    const char* e = std::getenv("GLASSO_NO_SPEC_TIER2");
    return e && e[0] == '1';
  }();
  const bool spec = !spec_off && cfg_.precision != GLASSO_FP64 && st_.band_hit && h.m_free <= (double)ws.csr.cap;
  if (spec && !t2_.st) {
    // the factorisation goes to a stream of the highest priority, so that its one-CTA leaves
    // and small products take the SMs they need first and the tier-2 kernels fill the rest
    int lo = 0, hi = 0;
    CUDA_CHECK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    CUDA_CHECK(cudaStreamCreateWithFlags(&t2_.st, cudaStreamNonBlocking));
    CUDA_CHECK(cudaEventCreateWithFlags(&t2_.fork, cudaEventDisableTiming));
    CUDA_CHECK(cudaEventCreateWithFlags(&t2_.join, cudaEventDisableTiming));
    CUDA_CHECK(cudaStreamCreateWithPriority(&fac_.st, cudaStreamNonBlocking, hi));
    CUDA_CHECK(cudaEventCreateWithFlags(&fac_.join, cudaEventDisableTiming));
  }
  bool band_hit = false;
  auto try_step = [&](double tt) -> double {
    {
      Profiler::Rec rec;
      prof.begin_rec(GLASSO_PROF_TRIAL, 24.5 * (double)n * (double)n, st, rec);
      trial(ws.A, ws.Y, ws.code, ld, ws.S, ld, n, np, lam, tt, ws.At, ws.Lt, ws.parts,
            &ws.sc->lin_s, st);
      prof.end_rec(rec, st);
    }
    if (spec) {
      CUDA_CHECK(cudaEventRecord(t2_.fork, st));
      CUDA_CHECK(cudaStreamWaitEvent(fac_.st, t2_.fork, 0));
      CUDA_CHECK(cudaStreamWaitEvent(t2_.st, t2_.fork, 0));
      factor(ws.Lt, ws.Lti, fac_.st);
      CUDA_CHECK(cudaEventRecord(fac_.join, fac_.st));
      logdet_terms(h.m_free, t2_.st, ws.X);
      CUDA_CHECK(cudaEventRecord(t2_.join, t2_.st));
      CUDA_CHECK(cudaStreamWaitEvent(st, fac_.join, 0));
      CUDA_CHECK(cudaStreamWaitEvent(st, t2_.join, 0));
    } else {
      factor(ws.Lt, ws.Lti, st);
    }
    sync_scalars();
    ++trials;
    tier = 1;
    if (!h.pd_t) return INFINITY;
    const double lin = h.lin_s + lam * h.lin_l1;
    double d = -(h.logdet_t - st_.ld_A) + lin;
    if (std::fabs(d) <= kDiffBand * delta) {
      band_hit = true;
      // log det At - log det A = log det(I + E) = tr E - tr E^2 / 2 + O(|E|^3)
      if (!spec) {
        logdet_terms(h.nnz + h.nnz_t, st);
        sync_scalars();
      }
      // the series is used while |E|_F <= 0.1, where its truncation (<= |E|_F^3 / 2.7) stays
      // far below the second-order term; otherwise the Cholesky difference stands
      if (h.tr_e2 <= 0.01) {
        d = -(h.tr_e - 0.5 * h.tr_e2) + lin;
        tier = 2;
      }
    }
    // Split-precision forms: the Cholesky pivots decide PD for the matrix the factorisation
    // saw, which differs from At by the split products' error.  A step about to be accepted
    // is therefore certified PD in FP64: by |E|_F <= 0.1 < 1 when tier 2 decided (At = A^{1/2}
    // (I + E) A^{1/2} with A PD), else by the congruence X At X^T = I + F with |F| < 1/2.
    if (d < 0.0 && tier == 1 && cfg_.precision != GLASSO_FP64) {
      ++out.pd_checks;
      if (!(congruence_radius(st) < 0.5)) {
        ++out.pd_refused;
        return INFINITY;
      }
    }
    return d;
  };
  while (t >= t_min) {
    dF = try_step(t);
    if (dF < 0.0) { accepted = true; break; }
    t *= shrink;
  }
  bool fallback = false;
  if (!accepted) {
    fallback = true;
    // cond_2 = lambda_max(A) lambda_max(W); power iteration underestimates both, and the
    // fallback step is an upper bound in Sec. 6, so it runs long enough (300 steps) to bring
    // the estimate within rounding on the spectra of the paper's workloads
    const double lmax_a = power_lambda_max(ws.A, st, 300);
    const double lmax_w = power_lambda_max(ws.W, st, 300);
    t = std::pow(kFallbackFactor / (lmax_a * lmax_w), 2.0);
    dF = try_step(t);
    accepted = dF < 0.0;
  }
  st_.band_hit = band_hit;
  out.trials += trials;
  out.step_t = t;
  out.step_dF = dF;
  out.step_tier = tier;
  out.step_fallback = fallback ? 1 : 0;
  if (keep_trace)
    out.trace.push_back(IterRecord{st_.k, trials, tier, st_.F, out.r, out.z_fro, out.nnz, t, dF});
  if (!accepted) return GLASSO_LINESEARCH_STALL;
  std::swap(ws.A, ws.At);
  std::swap(ws.L, ws.Lt);
  std::swap(ws.Li, ws.Lti);
  w_valid_ = false;
  st_.ld_A = h.logdet_t;
  st_.trsa = h.trsa_t;
  st_.l1 = h.l1_t;
  st_.F = -st_.ld_A + st_.trsa + lam * st_.l1;
  ++st_.k;
  return -1;
}

SolveOut Engine::finish(double* theta_out) {
  if (!st_.active) throw Error(GLASSO_ERR_ARG, "no solve in progress (call glasso_begin)");
  cudaStream_t st = stream_;
  const int64_t n = st_.n, ld = ws.ld;
  if (theta_out) {
    if (st_.on_device) {
      unpad(ws.A, ld, n, theta_out, st);
    } else {
      unpad(ws.A, ld, n, ws.T, st);
      CUDA_CHECK(cudaMemcpyAsync(theta_out, ws.T, sizeof(double) * n * n, cudaMemcpyDeviceToHost, st));
    }
  }
  CUDA_CHECK(wait_stream(st));
  SolveOut out = std::move(st_.out);
  out.iterations = st_.k;
  out.F = st_.F;
  out.logdet = st_.ld_A;
  out.launches = tl_launches - st_.launches_begin;
  out.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - st_.t_begin).count();
  st_.active = false;
  return out;
}

SolveOut Engine::solve(const void* Sin, bool s_f32, bool s_on_device, int64_t n, double lam,
                       double tol, const double* theta0, double* theta_out, bool keep_trace) {
  const int max_iter = cfg_.max_iter > 0 ? cfg_.max_iter : 500;
  begin(Sin, s_f32, s_on_device, n, lam, theta0);
  int status;
  while ((status = step(tol, max_iter, keep_trace)) < 0) {
  }
  SolveOut out = finish(theta_out);
  out.status = status;
  return out;
}

// ------------------------------------------------------------------------------------------
// device-resident states (serving: warm starts without the start point's factorisation)
// ------------------------------------------------------------------------------------------
void Engine::begin_resident(const void* Sin, bool s_f32, int64_t n, double lam, const Resident& r) {
  if (r.n != n || !r.theta || !r.li || !r.w) throw Error(GLASSO_ERR_ARG, "resident state of another size");
  st_ = SolveState{};
  st_.t_begin = std::chrono::steady_clock::now();
  st_.launches_begin = tl_launches;
  CUDA_CHECK(cudaSetDevice(cfg_.device));
  ws.ensure(n, cfg_.hbm_budget_bytes);
  autotune();
  st_.launches_begin = tl_launches;
  if (r.np != ws.np) throw Error(GLASSO_ERR_ARG, "resident state of another padded size");
  csr_valid_ = false;
  cudaStream_t st = stream_;
  const size_t mat = sizeof(double) * ws.ld * ws.np;
  load_matrix(Sin, s_f32, false, n, ws.S, true);
  if (cfg_.standardize) {
    int bad = 0;
    CUDA_CHECK(cudaMemsetAsync(ws.bad, 0, sizeof(int), st));
    standardize(ws.S, ws.ld, n, ws.vec, ws.bad, st);
    CUDA_CHECK(cudaMemcpyAsync(&bad, ws.bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(wait_stream(st));
    if (bad) throw Error(GLASSO_ERR_ARG, "standardize needs every S_ii > 0");
  }
  CUDA_CHECK(cudaMemsetAsync(ws.code, 0, (size_t)ws.ld * ws.np, st));
  CUDA_CHECK(cudaMemcpyAsync(ws.A, r.theta, mat, cudaMemcpyDeviceToDevice, st));
  CUDA_CHECK(cudaMemcpyAsync(ws.Li, r.li, mat, cudaMemcpyDeviceToDevice, st));
  CUDA_CHECK(cudaMemcpyAsync(ws.W, r.w, mat, cudaMemcpyDeviceToDevice, st));
  objective_terms(ws.S, ws.A, ws.ld, n, ws.parts, &ws.sc->trsa, st);
  sync_scalars();
  w_valid_ = true;
  st_.active = true;
  st_.on_device = false;
  st_.n = n;
  st_.lam = lam;
  st_.ld_A = r.logdet;
  st_.trsa = ws.hs->trsa;
  st_.l1 = ws.hs->l1;
  st_.F = -st_.ld_A + st_.trsa + lam * st_.l1;
}

double Engine::export_resident(double* theta, double* li, double* w) {
  if (!w_valid_) throw Error(GLASSO_ERR_ARG, "no current inverse to export");
  cudaStream_t st = stream_;
  const size_t mat = sizeof(double) * ws.ld * ws.np;
  CUDA_CHECK(cudaMemcpyAsync(theta, ws.A, mat, cudaMemcpyDeviceToDevice, st));
  CUDA_CHECK(cudaMemcpyAsync(li, ws.Li, mat, cudaMemcpyDeviceToDevice, st));
  CUDA_CHECK(cudaMemcpyAsync(w, ws.W, mat, cudaMemcpyDeviceToDevice, st));
  CUDA_CHECK(wait_stream(st));
  return st_.ld_A;
}

SolveOut Engine::solve_resident(const void* Sin, bool s_f32, int64_t n, double lam, double tol, const Resident& r,
                                double* theta_out) {
  const int max_iter = cfg_.max_iter > 0 ? cfg_.max_iter : 500;
  begin_resident(Sin, s_f32, n, lam, r);
  int status;
  while ((status = step(tol, max_iter, false)) < 0) {
  }
  SolveOut out = finish(theta_out);
  out.status = status;
  return out;
}

void Engine::release_workspace() {
  CUDA_CHECK(cudaSetDevice(cfg_.device));
  if (stream_) CUDA_CHECK(wait_stream(stream_));
  drop_graphs();
  ws.release();
  csr_valid_ = false;
  w_valid_ = false;
  st_.active = false;
}

// ------------------------------------------------------------------------------------------
// single steps
// ------------------------------------------------------------------------------------------
void Engine::op_cholesky(const double* A, int64_t n, double* L, int* pd, double* logdet) {
  CUDA_CHECK(cudaSetDevice(cfg_.device));
  ws.ensure(n, cfg_.hbm_budget_bytes);
  autotune();
  csr_valid_ = false;
  w_valid_ = false;
  cudaStream_t st = stream_;
  load_matrix(A, false, true, n, ws.Lt, false);
  pad_identity(ws.Lt, ws.ld, n, ws.np, st);
  factor(ws.Lt, ws.Lti, st);
  k_unpad_lower<<<red_blocks(n), 256, 0, st>>>(ws.Lt, ws.ld, n, L);
  LAUNCH_CHECK();
  sync_scalars();
  *pd = ws.hs->pd_t;
  *logdet = ws.hs->logdet_t;
}

int Engine::op_inverse(const double* A, int64_t n, double* W) {
  CUDA_CHECK(cudaSetDevice(cfg_.device));
  ws.ensure(n, cfg_.hbm_budget_bytes);
  autotune();
  csr_valid_ = false;
  w_valid_ = false;
  cudaStream_t st = stream_;
  load_matrix(A, false, true, n, ws.A, false);
  pad_identity(ws.A, ws.ld, n, ws.np, st);
  CUDA_CHECK(cudaMemcpyAsync(ws.L, ws.A, sizeof(double) * ws.ld * ws.np, cudaMemcpyDeviceToDevice, st));
  factor(ws.L, ws.Li, st);
  sync_scalars();
  if (!ws.hs->pd_t) return 0;
  compute_inverse(ws.Li, st);
  unpad(ws.W, ws.ld, n, W, st);
  CUDA_CHECK(wait_stream(st));
  return 1;
}

void Engine::op_gradient(const double* S, const double* A, const double* W, int64_t n, double lam,
                         double* X, int8_t* code, double sums[4]) {
  CUDA_CHECK(cudaSetDevice(cfg_.device));
  ws.ensure(n, cfg_.hbm_budget_bytes);
  autotune();
  csr_valid_ = false;
  w_valid_ = false;
  cudaStream_t st = stream_;
  load_matrix(S, false, true, n, ws.S, false);
  load_matrix(A, false, true, n, ws.A, false);
  load_matrix(W, false, true, n, ws.W, false);
  gradient(ws.S, ws.W, ws.A, ws.ld, n, lam, ws.X, ws.code, ws.ld, ws.parts, &ws.sc->z_l1, st);
  unpad(ws.X, ws.ld, n, X, st);
  unpad_i8(ws.code, ws.ld, n, code, st);
  sync_scalars();
  sums[0] = ws.hs->z_l1; sums[1] = ws.hs->a_l1; sums[2] = ws.hs->z_fro2; sums[3] = ws.hs->nnz;
}

void Engine::op_sandwich(const double* A, const double* X, int64_t n, double* Y) {
  CUDA_CHECK(cudaSetDevice(cfg_.device));
  ws.ensure(n, cfg_.hbm_budget_bytes);
  autotune();
  csr_valid_ = false;
  w_valid_ = false;
  cudaStream_t st = stream_;
  load_matrix(A, false, true, n, ws.A, false);
  load_matrix(X, false, true, n, ws.X, false);
  // nnz of A from its CSR row pointers
  csr_rowptr(ws.A, nullptr, ws.ld, n, ws.np, ws.counts, ws.csr.rowptr, st);
  int64_t nnz = 0;
  CUDA_CHECK(cudaMemcpyAsync(&nnz, ws.csr.rowptr + ws.np, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CUDA_CHECK(wait_stream(st));
  sandwich((double)nnz, st);
  mirror_lower(ws.Y, ws.ld, ws.np, st);
  unpad(ws.Y, ws.ld, n, Y, st);
  CUDA_CHECK(wait_stream(st));
}

void Engine::op_trial(const double* A, const double* Y, const int8_t* code, int64_t n, double lam,
                      double t, double* At) {
  CUDA_CHECK(cudaSetDevice(cfg_.device));
  ws.ensure(n, cfg_.hbm_budget_bytes);
  autotune();
  csr_valid_ = false;
  w_valid_ = false;
  cudaStream_t st = stream_;
  load_matrix(A, false, true, n, ws.A, false);
  load_matrix(Y, false, true, n, ws.Y, false);
  CUDA_CHECK(cudaMemsetAsync(ws.code, 0, (size_t)ws.ld * ws.np, st));
  pad_i8(code, n, ws.code, ws.ld, st);
  CUDA_CHECK(cudaMemsetAsync(ws.S, 0, sizeof(double) * ws.ld * ws.np, st));
  trial(ws.A, ws.Y, ws.code, ws.ld, ws.S, ws.ld, n, ws.np, lam, t, ws.At, ws.Lt, ws.parts,
        &ws.sc->lin_s, st);
  unpad(ws.At, ws.ld, n, At, st);
  CUDA_CHECK(wait_stream(st));
}

}  // namespace glasso
