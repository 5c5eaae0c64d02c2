// Host-side solver engine behind the C ABI: device workspaces, the pISTA outer loop with
// its line search (Algorithm 1), and the GEMM dispatch by precision mode.
#pragma once
#include <chrono>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>
#include "../../include/glasso.h"
#include "elementwise.h"
#include "factor.h"
#include "sparse.h"

namespace glasso {

// Device buffers of one problem of padded size np (all np x np FP64 unless noted).
struct Workspace {
  int device = 0;
  int64_t n = 0, ld = 0;
  int np = 0, cap_np = 0;
  double *S = nullptr, *A = nullptr, *At = nullptr, *W = nullptr, *L = nullptr, *Lt = nullptr;
  double *X = nullptr, *Y = nullptr, *T = nullptr;
  double *Li = nullptr, *Lti = nullptr;   // L^{-1} of the accepted / trial factor
  int8_t* code = nullptr;                 // np x np
  double* ld_parts = nullptr;             // np / 64
  double* parts = nullptr;                // 8 * kRedBlocks
  Scalars* sc = nullptr;                  // device scalars
  Scalars* hs = nullptr;                  // pinned host mirror
  int* pd = nullptr;                      // device PD flag
  double* vmax = nullptr;                 // [2]
  int* bad = nullptr;
  double* vec = nullptr;                  // 2 * np (power iteration)
  void* staging = nullptr;                // caller-sized staging for host inputs
  size_t staging_bytes = 0;
  void* tc_scratch = nullptr;             // split operands of the tensor-core GEMMs
  size_t tc_scratch_bytes = 0;
  void* tc_scratch2 = nullptr;            // the same for products on the side stream
  size_t tc_scratch2_bytes = 0;
  Csr csr;                                // Theta in CSR form for the sparse sandwich
  int* counts = nullptr;                  // np per-row nonzero counts
  uint64_t epoch = 0;                     // bumped at every reallocation

  static size_t bytes_for(int np);
  void ensure(int64_t n_new, size_t budget);  // (re)allocate for n_new; throws on failure
  void release();
  ~Workspace() { release(); }
};

struct IterRecord {
  int k, trials, tier;
  double F, r, z_fro, nnz, t, dF;
};

struct SolveOut {
  int status = 0;
  int iterations = 0, trials = 0;
  double r = 0, z_fro = 0, F = 0, logdet = 0, nnz = 0, seconds = 0;
  int64_t launches = 0;
  // the last line search: its final trial step, dF, tier and whether the fallback ran
  double step_t = 0, step_dF = 0;
  int step_tier = 0, step_fallback = 0;
  // split-precision forms: FP64 PD certificates run on trial points, and trials they refused
  int pd_checks = 0, pd_refused = 0;
  std::vector<IterRecord> trace;
};

// Iterate and objective pieces carried between outer iterations.
struct SolveState {
  bool active = false;
  bool on_device = false;
  int64_t n = 0;
  double lam = 0, ld_A = 0, trsa = 0, l1 = 0, F = 0;
  double t_last = 1.0;   // G-ISTA: the last accepted step
  int k = 0;
  bool band_hit = false;  // a trial of the last line search fell in the rounding band
  SolveOut out;
  std::chrono::steady_clock::time_point t_begin;
  int64_t launches_begin = 0;
};

// CUDA-event accounting of the kernel classes (glasso_profile_*).
struct Profiler {
  bool on = false;
  struct Rec { int cls; double work; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get();
  void start();
  void begin_rec(int cls, double work, cudaStream_t st, Rec& r);
  void end_rec(Rec& r, cudaStream_t st);
  void collect(glasso_profile* out);
  ~Profiler();
};

double probe_fp64_tflops(int device);

// Kernel launches made by the calling thread (each engine runs on one thread at a time).
int64_t thread_launches();

class Engine {
 public:
  explicit Engine(const glasso_config& cfg);
  ~Engine();
  const glasso_config& config() const { return cfg_; }
  cudaStream_t stream() const { return stream_; }

  // Full pISTA solve.  S is the caller's n x n matrix (host or device); theta0 may be null.
  SolveOut solve(const void* S, bool s_f32, bool s_on_device, int64_t n, double lam, double tol,
                 const double* theta0, double* theta_out, bool keep_trace = false);
  // The same solve one outer iteration at a time.
  void begin(const void* S, bool s_f32, bool s_on_device, int64_t n, double lam, const double* theta0);
  // Returns -1 after an accepted step, else the final status (OK, MAX_ITER, STALL).
  int step(double tol, int max_iter, bool keep_trace);
  SolveOut finish(double* theta_out);

  // Device-resident solver state: an iterate Theta, the inverse of its Cholesky factor and
  // W = Theta^{-1}, each np x np (leading dimension np, the workspace layout), and log det.
  struct Resident {
    int64_t n = 0;
    int np = 0;
    const double* theta = nullptr;
    const double* li = nullptr;
    const double* w = nullptr;
    double logdet = 0.0;
  };
  // Start a solve from a resident state of the same n (a warm start that skips the start
  // point's factorisation and the first inverse); S as for begin (host memory).
  void begin_resident(const void* S, bool s_f32, int64_t n, double lam, const Resident& r);
  // Copy the current iterate, its inverse factor and W into resident buffers (np x np each)
  // and return log det; valid after a solve ended (W is then the current iterate's inverse).
  double export_resident(double* theta, double* li, double* w);
  // A full solve started from a resident state (begin_resident + steps + finish).
  SolveOut solve_resident(const void* S, bool s_f32, int64_t n, double lam, double tol, const Resident& r,
                          double* theta_out);
  // Give the device workspace back (the next solve allocates it again).
  void release_workspace();
  const SolveState& state() const { return st_; }
  Profiler prof;

  // single steps on caller device arrays (leading dimension n)
  void op_cholesky(const double* A, int64_t n, double* L, int* pd, double* logdet);
  int op_inverse(const double* A, int64_t n, double* W);
  void op_gradient(const double* S, const double* A, const double* W, int64_t n, double lam,
                   double* X, int8_t* code, double sums[4]);
  void op_sandwich(const double* A, const double* X, int64_t n, double* Y);
  void op_trial(const double* A, const double* Y, const int8_t* code, int64_t n, double lam,
                double t, double* At);

  // the GEMM used for a given role in the configured precision mode
  void gemm(const GemmArgs& a, GemmRole role, cudaStream_t st);
  // Measure the kernel choices for every product shape an np x np solve issues (split-
  // precision forms; shapes already in the tuner's table are skipped).  Uses the workspace as
  // scratch, so it runs before a solve loads its inputs.
  void autotune();
  GemmFn gemm_fn();

  Workspace ws;

 private:
  void load_matrix(const void* src, bool f32, bool on_device, int64_t n, double* dst, bool check_s);
  // Y = lower(A X A): sparse products while nnz(A) (over the n x n block) permits, else dense
  void sandwich(double nnz, cudaStream_t st);
  bool sparse_sandwich(double nnz) const;
  // CSR of ws.A in ws.csr (built at most once per outer iteration); false when nnz(A)
  // exceeds the capacity
  bool ensure_csr_of_A(cudaStream_t st);
  bool csr_valid_ = false;
  bool w_valid_ = false;  // ws.W holds the inverse of ws.A (refined in the split-precision forms)
  // Q = (At - A) W and {tr Q, tr Q^2} into the scalars
  void logdet_terms(double nnz_bound, cudaStream_t st, double* Q = nullptr);
  int64_t csr_nnz_ = 0;  // nonzeros of A the last CSR pass counted
  void compute_inverse(double* Li, cudaStream_t st);
  void factor(double* L, double* Li, cudaStream_t st);
  void refine_inverse(cudaStream_t st);
  int gista_step(double tol, int max_iter, bool keep_trace);
  double power_lambda_max(const double* M, cudaStream_t st, int iters);
  double congruence_radius(cudaStream_t st);
  void sync_scalars();
  cudaError_t wait_stream(cudaStream_t st);
  cudaEvent_t wait_ev_ = nullptr;
  bool blocking_sync_ = false;

 public:
  // Waits sleep on a blocking-sync event instead of spinning (engines of many-slot pools).
  void set_blocking_sync(bool on) { blocking_sync_ = on; }

 private:

  // CUDA graphs of the factorisation, one per (factor buffer, inverse buffer) pair
  struct FactorGraph {
    cudaGraphExec_t exec;
    int64_t launches;
  };
  using GraphKey = std::tuple<const double*, const double*, int>;
  std::map<GraphKey, FactorGraph> fgraphs_;
  std::map<GraphKey, int> fseen_;
  uint64_t graph_epoch_ = 0;
  bool use_graphs_ = true;
  int panel_ = 0;
  cudaStream_t cap_stream_ = nullptr;
  SideStream side_;  // the factorisation's second stream (split-precision forms)
  SideStream t2_;    // the tier-2 terms formed alongside a trial's factorisation
  SideStream fac_;   // high-priority stream the trial is factored on meanwhile
  void drop_graphs();
  void factor_direct(double* L, double* Li, cudaStream_t st);
  void factor_graphed(double* L, double* Li, cudaStream_t st);

  glasso_config cfg_;
  std::string gpu_name_;
  int tuned_np_ = 0;  // padded size the autotuner last covered
  SolveState st_;
  cudaStream_t stream_ = nullptr;
  bool own_stream_ = false;
};

}  // namespace glasso
