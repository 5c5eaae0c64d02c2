/*
 * glasso.h -- C ABI of libglasso, a GB300 (sm_103a) solver for the graphical lasso
 *
 *     min_{Theta > 0}  F(Theta) = -log det Theta + tr(S Theta) + lambda * ||Theta||_1
 *
 * (Sec. 3.1 of Shalom, Treister & Yavneh, "pISTA: preconditioned Iterative Soft
 * Thresholding Algorithm for Graphical Lasso", eq. sparse_obj; ||.||_1 sums all n*n
 * entries, the diagonal included) by pISTA (Sec. 4, Algorithm 1).
 *
 * Conventions shared by every entry point
 *   - Matrices are dense, row-major, n x n with leading dimension n.  S and Theta are
 *     symmetric; the library reads the LOWER triangle of S and mirrors it.
 *   - Ownership: the caller owns every pointer it passes and every output buffer; the
 *     library owns the handle and all device state behind it.  Nothing passed in is
 *     retained after a call returns (glasso_submit copies S before it returns).
 *   - Errors: every call returns a glasso_status; nothing throws across the ABI.  On an
 *     error the outputs are unspecified and glasso_last_error(h) describes the cause.
 *   - Threading: one handle serves one host thread at a time, except that glasso_submit
 *     and glasso_poll may be called from any thread while the serving loop runs.
 *   - GLASSO_ERR_CUDA means a CUDA call failed; the handle should then be destroyed.
 *   - All work runs on the handle's stream; calls return after that work has finished.
 */
#ifndef GLASSO_H
#define GLASSO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GLASSO_OK = 0,
  GLASSO_ERR_ARG = 1,            /* invalid argument (n < 1, lambda <= 0, tol < 0, NULL ...) */
  GLASSO_ERR_NOT_SYMMETRIC = 2,  /* |S_ij - S_ji| > 1e-12 * max|S| */
  GLASSO_ERR_NONFINITE = 3,      /* S holds NaN or Inf, or some S_ii < 0 */
  GLASSO_ERR_NOT_PD = 4,         /* the start point Theta0 (or the op input) is not PD */
  GLASSO_ERR_OOM = 5,            /* a device or pinned-host allocation failed */
  GLASSO_ERR_BUDGET = 6,         /* the problem cannot fit the configured HBM budget */
  GLASSO_ERR_CUDA = 7,           /* a CUDA runtime / driver call failed */
  GLASSO_ERR_TIMEOUT = 8,        /* a bounded wait ran out */
  GLASSO_MAX_ITER = 9,           /* stopped at max_iter; the result is the last PD iterate */
  GLASSO_LINESEARCH_STALL = 10,  /* no step passed the line search; the result is the last
                                    PD iterate (Sec. 4.3.2, Sec. 6 fallback step) */
  GLASSO_PENDING = 11,           /* glasso_poll: the request has not finished yet */
  GLASSO_ERR_UNSUPPORTED = 12    /* the device is not an sm_103 GPU, or the mode is absent */
} glasso_status;

typedef enum {
  GLASSO_FP64 = 0,          /* every step in FP64 */
  GLASSO_MIXED_TF32X3 = 1,  /* dense products wider than 256 on the tensor cores with
                               3-term TF32 splits, smaller ones in FP32 arithmetic, all added
                               to FP64 storage in FP64; Cholesky panels in FP64 (see
                               glasso_config.fp32_panels); W refined to FP64 accuracy; every
                               accepted trial certified PD in FP64; FP64 line-search and stop
                               decisions */
  GLASSO_MIXED_BF16X3 = 2   /* as GLASSO_MIXED_TF32X3 with 3-term BF16 splits */
} glasso_precision;

typedef enum { GLASSO_F64 = 0, GLASSO_F32 = 1 } glasso_dtype;
typedef enum { GLASSO_HOST = 0, GLASSO_DEVICE = 1 } glasso_memory;

/* How Theta X Theta (eq. b) is formed.  DENSE: two dense products (tensor cores in the
 * split-precision modes, FP64 CUDA cores otherwise).  SPARSE: two FP64 products with Theta in
 * CSR form, O(nnz(Theta) n) work, exact to FP64 rounding; used while nnz(Theta) <= 256 n.
 * AUTO (default): SPARSE in the FP64 form, and in the split-precision forms while
 * nnz(Theta) <= n max(16, n / 256), where it also costs less than the dense products. */
typedef enum { GLASSO_PRODUCTS_AUTO = 0, GLASSO_PRODUCTS_DENSE = 1, GLASSO_PRODUCTS_SPARSE = 2 } glasso_products;

/* The outer method.  PISTA: Algorithm 1 (the default).  GISTA: the plain proximal gradient
 * method, eq. proximal_gen with H = I (Sec. 2.2): Theta <- ST(Theta - t g, t lambda), t
 * chosen by halving from twice the last step until the candidate is PD and satisfies the
 * sufficient-decrease bound f(Theta_t) <= f(Theta) + <g, D> + ||D||_F^2 / (2t), never below
 * t_safe = lambda_min(Theta)^2 / 2 (at which the gradient is Lipschitz with constant at
 * most 1/lambda_min^2 near Theta, the bound behind Lemma 5.2); the same stop rule. */
typedef enum { GLASSO_METHOD_PISTA = 0, GLASSO_METHOD_GISTA = 1 } glasso_method;

typedef struct glasso_handle glasso_handle;

typedef struct {
  int device;               /* CUDA ordinal */
  void* stream;             /* cudaStream_t to run on; NULL: the library creates its own */
  glasso_precision precision;
  int max_iter;             /* default 500 */
  double shrink;            /* line-search factor; default 0.5 (Sec. 4.3.2 leaves it open) */
  double t_min;             /* halving stops below this t; default 1e-4 (Sec. 6) */
  size_t hbm_budget_bytes;  /* device memory the handle may hold; 0 = no limit */
  int serve_slots;          /* requests the serving loop runs at once; default 8 */
  int products;             /* glasso_products: how the sandwich products of eq. b are formed */
  int method;               /* glasso_method; default GLASSO_METHOD_PISTA */
  int standardize;          /* 1: every solve replaces S by its correlation matrix
                               D^{-1/2} S D^{-1/2}, D = diag S (entry (i, j) computed as
                               (S_ij d_i) d_j, d_i = 1 / sqrt(S_ii)), the preprocessing the
                               paper applies to its gene-expression data (Sec. 6.2); the
                               result is the estimate for the standardised problem.  S_ii
                               must then be > 0 (else GLASSO_ERR_ARG).  Default 0. */
  int fp32_panels;          /* split-precision modes only.  0 (default): the Cholesky panels
                               (64 x 64 diagonal blocks) are factored in FP64, so the pivots,
                               the PD test and the log det are FP64 arithmetic on the FP64
                               Schur complement; the inverse of each block's factor, which
                               only feeds split-precision products, is formed in FP32.
                               1: 128 x 128 panels factored and inverted in FP32 (faster,
                               FP32-grade pivots). */
  int autotune;             /* split-precision modes.  1 (default): the first solve of a size
                               measures, for each dense product shape it will issue, the FP32
                               CUDA-core kernel and the tensor-core kernel with 128 x 256 and
                               128 x 128 tiles, and runs each shape on the fastest from then
                               on; results are kept per GPU model in the file named by the
                               environment variable GLASSO_TUNE_CACHE (default
                               $HOME/.cache/glasso_gemm_tune.txt; "off": in memory only).
                               0: the built-in rule (FP32 CUDA cores up to 256, else 128 x 256
                               tensor-core tiles). */
} glasso_config;

typedef struct {
  int32_t status;           /* glasso_status of this solve */
  int32_t iterations;       /* accepted pISTA iterations */
  int32_t trials;           /* line-search trials (Cholesky factorisations of trial points) */
  int32_t nnz;              /* nonzeros of Theta over all n*n entries */
  double rel_kkt_l1;        /* ||Z||_1 / ||Theta||_1, Z the minimum-norm sub-gradient (Sec. 6) */
  double min_subgrad_fro;   /* ||Z||_F */
  double objective;         /* F(Theta), eq. sparse_obj */
  double logdet;            /* log det Theta */
  double seconds;           /* wall time of the solve inside the library */
  double t_submit, t_start, t_done;  /* serving timestamps (s, monotonic clock), else 0 */
  int64_t kernel_launches;  /* CUDA kernels this solve (or step) launched */
  /* The last line search (glasso_step: this call's, all 0 when the call formed no
   * direction; glasso_solve: the solve's last one, accepted or refused): */
  double step_t;            /* step size of the last trial (Sec. 4.3.2 halving or the Sec. 6
                               fallback t = (0.9 / cond Theta)^2) */
  double step_dF;           /* F(Theta_t) - F(Theta) the accept test saw (eq. t_cond_min) */
  int32_t step_tier;        /* 1: dF from the two Cholesky log-dets; 2: the log-det
                               difference re-evaluated from Theta^{-1} near the decision */
  int32_t step_fallback;    /* 1 if halving went below t_min and the fallback step was tried */
} glasso_result;

/* ---- handle ------------------------------------------------------------------------------ */

/* Fill *cfg with the defaults listed above (device 0, own stream, FP64). */
glasso_status glasso_config_default(glasso_config* cfg);

/* Create a handle for cfg->device (NULL cfg: defaults).  GLASSO_ERR_UNSUPPORTED when the
 * device is not compute capability 10.3.  *out is set to the handle, or NULL on error. */
glasso_status glasso_create(const glasso_config* cfg, glasso_handle** out);

/* Stop the serving loop (unfinished requests are dropped), free all device memory and
 * the handle.  NULL is accepted. */
glasso_status glasso_destroy(glasso_handle* h);

/* Text of the last error on this handle ("" if none); valid until the next call. */
const char* glasso_last_error(const glasso_handle* h);

/* Name of a status code. */
const char* glasso_status_string(glasso_status s);

/* ---- solve (Algorithm 1) ------------------------------------------------------------------ */

/* One pISTA solve of the graphical lasso for (S, lambda), stopped when
 * ||Z||_1 <= tol * ||Theta||_1 (Sec. 6 stop rule, checked before each direction).
 *   S        n x n, dtype s_dtype (FP32 is promoted exactly to FP64), in host or device
 *            memory as `where` says.
 *   theta0   optional start point (FP64, same memory kind as S); NULL: the start point of
 *            Sec. 6, diag(1/(S_ii + lambda)).  Must be symmetric positive definite.
 *   theta_out  n x n FP64 output (same memory kind as S), may be NULL.
 *   res      optional summary.
 * Returns GLASSO_OK on convergence, GLASSO_MAX_ITER / GLASSO_LINESEARCH_STALL with the last
 * (positive-definite) iterate in theta_out, or an error. */
glasso_status glasso_solve(glasso_handle* h, const void* S, glasso_dtype s_dtype,
                           glasso_memory where, int64_t n, double lambda, double tol,
                           const double* theta0, double* theta_out, glasso_result* res);

/* ---- step-wise solve: the same iteration as glasso_solve, one outer iteration per call ---- */

/* Load S and the start point as glasso_solve does and factor the start point.  The handle
 * then holds the iterate until glasso_end (or the next glasso_begin / glasso_solve). */
glasso_status glasso_begin(glasso_handle* h, const void* S, glasso_dtype s_dtype,
                           glasso_memory where, int64_t n, double lambda, const double* theta0);

/* One outer iteration of Algorithm 1: W = Theta^{-1}, gradient and stop test; if
 * ||Z||_1 > tol ||Theta||_1, the direction and the line search.  Returns GLASSO_PENDING
 * when a step was accepted, GLASSO_OK when the stop test held (no step taken),
 * GLASSO_LINESEARCH_STALL when no trial passed.  res (optional) describes the iterate the
 * stop test saw and counts this call's trials and kernel launches. */
glasso_status glasso_step(glasso_handle* h, double tol, glasso_result* res);

/* Copy the current iterate to theta_out (n x n FP64, the memory kind given to
 * glasso_begin; may be NULL) and end the step-wise solve. */
glasso_status glasso_end(glasso_handle* h, double* theta_out, glasso_result* res);

/* ---- device-time accounting of the kernel classes (CUDA events around each launch) --------- */

enum {
  GLASSO_PROF_SANDWICH = 0,   /* the two products of eq. b: FLOPs */
  GLASSO_PROF_TRAILING = 1,   /* Cholesky trailing updates: FLOPs */
  GLASSO_PROF_PANEL = 2,      /* Cholesky panel solves: FLOPs */
  GLASSO_PROF_INVERSE = 3,    /* triangular inverse and W = X^T X: FLOPs */
  GLASSO_PROF_REFINE = 4,     /* mixed mode: refinement products of W: FLOPs */
  GLASSO_PROF_GRADIENT = 5,   /* gradient / free-set / KKT pass: bytes moved */
  GLASSO_PROF_TRIAL = 6,      /* trial-point pass: bytes moved */
  GLASSO_PROF_FACTOR = 7,     /* whole Cholesky-with-inverse calls (their products included):
                                 FLOPs n^3/3 + n^3/3 */
  GLASSO_PROF_RESIDUAL = 8,   /* mixed mode: FP64 residual I - Theta W from the sparse rows of
                                 Theta: FP64 FLOPs, 2 nnz(Theta) per column of W */
  GLASSO_PROF_LOGDET2 = 9,    /* second-order log-det difference near the decision boundary:
                                 bytes of the dTheta W and trace passes */
  GLASSO_PROF_AUX = 10,       /* symmetrising copies of W and the refinement update: bytes */
  GLASSO_PROF_SPMM = 11,      /* sparse sandwich products with their CSR build: FP64 FLOPs
                                 2 nnz(Theta) n + nnz(Theta) n (the second product lower only) */
  GLASSO_PROF_CLASSES = 12
};

typedef struct {
  double ms[GLASSO_PROF_CLASSES];      /* summed device time of the class's launches */
  double work[GLASSO_PROF_CLASSES];    /* algorithmic FLOPs or bytes of those launches */
  int64_t launches[GLASSO_PROF_CLASSES];
} glasso_profile;

/* Start recording (clears earlier records).  Adds two event records per launch. */
glasso_status glasso_profile_start(glasso_handle* h);
/* Wait for the recorded work, fill *out and stop recording. */
glasso_status glasso_profile_stop(glasso_handle* h, glasso_profile* out);

/* Peak FP64 FMA throughput of a device in TFLOP/s, measured by a register-resident FMA
 * kernel (the roofline denominator of the FP64 form; it allocates a small buffer). */
glasso_status glasso_probe_fp64_peak(int device, double* tflops);

/* Device memory one solve of size n holds on a handle (its workspace: the n x n iterates,
 * factors, products and scratch, padded to a multiple of 128), the figure the HBM budget of
 * glasso_config and the serving loop's admission count per slot.  GLASSO_ERR_ARG for n < 1. */
glasso_status glasso_workspace_bytes(int64_t n, size_t* bytes);

/* ---- batched regularisation paths -------------------------------------------------------- */

typedef struct {
  int64_t n;
  const void* S;            /* host memory, n x n, dtype below */
  glasso_dtype dtype;
  int32_t n_lambda;
  const double* lambdas;    /* n_lambda values, solved in DESCENDING order, each warm-started
                               from the previous solution of the same problem */
  double tol;
  double* theta_out;        /* host, n_lambda * n * n FP64 (in the order given), or NULL */
} glasso_problem;

/* Solve `count` independent problems, each along its lambda path.  Problems run
 * concurrently on the device.  results: count * n_lambda entries, problem-major, in the
 * order the lambdas were given.  Returns the first error met, else GLASSO_OK (per-solve
 * convergence is in results[].status). */
glasso_status glasso_solve_batch(glasso_handle* h, const glasso_problem* probs, int32_t count,
                                 glasso_result* results);

/* ---- serving (continuous batching) ------------------------------------------------------- */

typedef struct {
  int64_t n;
  const void* S;            /* host memory, copied before glasso_submit returns */
  glasso_dtype dtype;
  double lambda;
  double tol;
  int64_t dataset_id;       /* requests with the same id share S; the solution of the nearest
                               earlier lambda for the id warm-starts the solve; -1: none */
} glasso_request;

/* Queue a request; returns at once with *ticket.  Requests are admitted while their device
 * memory fits hbm_budget_bytes and a slot is free, and run concurrently with the requests
 * already on the device.  GLASSO_ERR_BUDGET if the request can never fit. */
glasso_status glasso_submit(glasso_handle* h, const glasso_request* req, uint64_t* ticket);

/* GLASSO_PENDING while the request runs; otherwise its final status, with *res filled and,
 * if theta_out is not NULL, the n x n FP64 solution copied to host memory.  A finished
 * ticket can be polled once; GLASSO_ERR_ARG for an unknown ticket. */
glasso_status glasso_poll(glasso_handle* h, uint64_t ticket, glasso_result* res,
                          double* theta_out);

/* ---- single steps on device memory (one pISTA step each, for testing and composition) ---- */
/* All pointers are device pointers to n x n row-major FP64 arrays (code: int8) with leading
 * dimension n; the step runs in the handle's precision mode and returns when done. */

/* Cholesky factor A = L L^T (lower L, upper triangle of L set to 0), *pd = 1 if A is
 * positive definite (every pivot finite and > 0), log det A = 2 sum log L_ii (Sec. 4.3.2,
 * eq. t_cond_pd and the objective of eq. sparse_obj). */
glasso_status glasso_op_cholesky(glasso_handle* h, const double* A, int64_t n, double* L,
                                 int32_t* pd, double* logdet);

/* W = A^{-1} (eq. grad_hessian needs it) for a symmetric positive-definite A, from the
 * Cholesky factor: W = L^{-T} L^{-1}.  In the split-precision modes W is refined until
 * max |I - A W| <= 1e-9 (measured or predicted).  GLASSO_ERR_NOT_PD if A is not PD. */
glasso_status glasso_op_inverse(glasso_handle* h, const double* A, int64_t n, double* W);

/* From (S, A, W = A^{-1}): g = S - W (eq. grad_hessian), free set M (eqs. free_set, M),
 * sign guess G (eq. G+), X = (g + lambda G) . M, which is the minimum-norm sub-gradient Z,
 * and code = G . M in {-1, 0, 1}.  sums[0..3] = ||Z||_1, ||A||_1, ||Z||_F^2, nnz(A). */
glasso_status glasso_op_gradient(glasso_handle* h, const double* S, const double* A,
                                 const double* W, int64_t n, double lambda, double* X,
                                 int8_t* code, double sums[4]);

/* Y = A X A for symmetric A, X (the two products of eq. b), formed as the handle's
 * glasso_config.products says: from the CSR of A in FP64, or by two dense products. */
glasso_status glasso_op_sandwich(glasso_handle* h, const double* A, const double* X, int64_t n,
                                 double* Y);

/* Trial point A_t = A + M . D with D = -A + ST(A - tB, tC) (eq. d_sol), where
 * B = Y - C . code (eq. b), C from eq. c, and M = (code != 0). */
glasso_status glasso_op_trial(glasso_handle* h, const double* A, const double* Y,
                              const int8_t* code, int64_t n, double lambda, double t,
                              double* At);

/* ---- allocation-free variant of the gradient step ------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory themselves -- code running under a framework that owns every device
 * allocation, a stream-ordered runtime that forbids cudaMalloc on its hot path, or an
 * embedding with a memory budget fixed in advance.  It computes what glasso_op_gradient
 * computes, with no handle and no allocation: no cudaMalloc, cudaFree or allocating library
 * call.  Its only scratch is a file-scope device array of GLASSO_NOALLOC_MAX_N * 4 doubles
 * (512 KB) inside the library, which every GPU that loads the library holds until the
 * process exits.
 *   S, A, W   device pointers, n x n FP64 row-major, leading dimension n (no padding).
 *   X, code   device outputs, n x n (FP64 and int8): X = (g + lambda G).M, code = G.M.
 *   sums      device output of 4 doubles: ||Z||_1, ||A||_1, ||Z||_F^2, nnz(A).
 *   stream    cudaStream_t to run on (NULL: the legacy default stream).
 * Runs on the device that is current for the calling thread and returns once the work is
 * queued on `stream` (the outputs are ready when the stream reaches it).  The first call in
 * a CUDA context looks up the device address of the scratch array there (cudaGetSymbolAddress)
 * and caches it under the context's unique id, so a new context -- after cudaDeviceReset, or
 * a driver-API context other than the device's primary one -- gets its own address; make the
 * first call in each context before any stream capture.  Every call on a device
 * shares the one scratch array and overwrites its first n rows, so nothing in it has to
 * start at zero; calls whose work overlaps on the GPU (different streams, or graphs replayed
 * concurrently) race on it and must be serialised by the caller.
 * Returns GLASSO_ERR_BUDGET when n > GLASSO_NOALLOC_MAX_N, GLASSO_ERR_ARG for NULL
 * pointers, n < 1 or lambda <= 0, GLASSO_ERR_CUDA when a CUDA call fails. */
#define GLASSO_NOALLOC_MAX_N 16384
glasso_status glasso_gradient_noalloc(const double* S, const double* A, const double* W,
                                      int64_t n, double lambda, double* X, int8_t* code,
                                      double* sums, void* stream);

#ifdef __cplusplus
}
#endif
#endif
