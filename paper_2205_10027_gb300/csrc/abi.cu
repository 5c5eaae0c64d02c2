// extern "C" entry points of libglasso (declared in include/glasso.h): argument checks,
// exception-to-status translation, and the handle that owns the engine.
#include <cstring>
#include <memory>
#include <new>
#include "engine.h"
#include "serve.h"

struct glasso_handle {
  glasso_config cfg;
  std::unique_ptr<glasso::Engine> engine;
  std::unique_ptr<glasso::Server> server;
  std::mutex mu;  // one caller at a time on the engine
  std::string last_error;
};

namespace {

glasso_status fail(glasso_handle* h, int st, const std::string& msg) {
  if (h) h->last_error = msg;
  return (glasso_status)st;
}

template <typename F>
glasso_status guarded(glasso_handle* h, F&& f) {
  try {
    return f();
  } catch (const glasso::Error& e) {
    return fail(h, e.status, e.what());
  } catch (const std::bad_alloc&) {
    return fail(h, GLASSO_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(h, GLASSO_ERR_CUDA, e.what());
  }
}

void fill_result(glasso_result* res, const glasso::SolveOut& o) {
  if (!res) return;
  std::memset(res, 0, sizeof(*res));
  res->status = o.status;
  res->iterations = o.iterations;
  res->trials = o.trials;
  res->nnz = (int32_t)o.nnz;
  res->rel_kkt_l1 = o.r;
  res->min_subgrad_fro = o.z_fro;
  res->objective = o.F;
  res->logdet = o.logdet;
  res->seconds = o.seconds;
  res->kernel_launches = o.launches;
  res->step_t = o.step_t;
  res->step_dF = o.step_dF;
  res->step_tier = o.step_tier;
  res->step_fallback = o.step_fallback;
}

bool valid_problem(int64_t n, double lambda, double tol) {
  return n >= 1 && n <= (int64_t)1 << 20 && std::isfinite(lambda) && lambda > 0.0 &&
         std::isfinite(tol) && tol >= 0.0;
}

}  // namespace

extern "C" {

glasso_status glasso_config_default(glasso_config* cfg) {
  if (!cfg) return GLASSO_ERR_ARG;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->device = 0;
  cfg->stream = nullptr;
  cfg->precision = GLASSO_FP64;
  cfg->max_iter = 500;
  cfg->shrink = 0.5;
  cfg->t_min = 1e-4;
  cfg->hbm_budget_bytes = 0;
  cfg->serve_slots = 8;
  cfg->products = GLASSO_PRODUCTS_AUTO;
  cfg->method = GLASSO_METHOD_PISTA;
  cfg->standardize = 0;
  cfg->fp32_panels = 0;
  cfg->autotune = 1;
  return GLASSO_OK;
}

glasso_status glasso_create(const glasso_config* cfg_in, glasso_handle** out) {
  if (!out) return GLASSO_ERR_ARG;
  *out = nullptr;
  glasso_config cfg;
  if (cfg_in) cfg = *cfg_in; else glasso_config_default(&cfg);
  if (cfg.precision < GLASSO_FP64 || cfg.precision > GLASSO_MIXED_BF16X3) return GLASSO_ERR_ARG;
  if (cfg.serve_slots <= 0) cfg.serve_slots = 8;
  if (cfg.products < GLASSO_PRODUCTS_AUTO || cfg.products > GLASSO_PRODUCTS_SPARSE) return GLASSO_ERR_ARG;
  if (cfg.method != GLASSO_METHOD_PISTA && cfg.method != GLASSO_METHOD_GISTA) return GLASSO_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg.device < 0 || cfg.device >= ndev) {
    cudaGetLastError();
    return GLASSO_ERR_UNSUPPORTED;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, cfg.device) != cudaSuccess) return GLASSO_ERR_CUDA;
  if (prop.major != 10 || prop.minor != 3) return GLASSO_ERR_UNSUPPORTED;
  if (cfg.precision != GLASSO_FP64 && !glasso::tc_available()) return GLASSO_ERR_UNSUPPORTED;
  auto* h = new (std::nothrow) glasso_handle;
  if (!h) return GLASSO_ERR_OOM;
  h->cfg = cfg;
  const glasso_status st = guarded(h, [&] {
    h->engine = std::make_unique<glasso::Engine>(cfg);
    return GLASSO_OK;
  });
  if (st != GLASSO_OK) {
    delete h;
    return st;
  }
  *out = h;
  return GLASSO_OK;
}

glasso_status glasso_destroy(glasso_handle* h) {
  if (!h) return GLASSO_OK;
  h->server.reset();
  h->engine.reset();
  delete h;
  return GLASSO_OK;
}

const char* glasso_last_error(const glasso_handle* h) { return h ? h->last_error.c_str() : ""; }

const char* glasso_status_string(glasso_status s) {
  switch (s) {
    case GLASSO_OK: return "GLASSO_OK";
    case GLASSO_ERR_ARG: return "GLASSO_ERR_ARG";
    case GLASSO_ERR_NOT_SYMMETRIC: return "GLASSO_ERR_NOT_SYMMETRIC";
    case GLASSO_ERR_NONFINITE: return "GLASSO_ERR_NONFINITE";
    case GLASSO_ERR_NOT_PD: return "GLASSO_ERR_NOT_PD";
    case GLASSO_ERR_OOM: return "GLASSO_ERR_OOM";
    case GLASSO_ERR_BUDGET: return "GLASSO_ERR_BUDGET";
    case GLASSO_ERR_CUDA: return "GLASSO_ERR_CUDA";
    case GLASSO_ERR_TIMEOUT: return "GLASSO_ERR_TIMEOUT";
    case GLASSO_MAX_ITER: return "GLASSO_MAX_ITER";
    case GLASSO_LINESEARCH_STALL: return "GLASSO_LINESEARCH_STALL";
    case GLASSO_PENDING: return "GLASSO_PENDING";
    case GLASSO_ERR_UNSUPPORTED: return "GLASSO_ERR_UNSUPPORTED";
  }
  return "unknown status";
}

glasso_status glasso_solve(glasso_handle* h, const void* S, glasso_dtype s_dtype,
                           glasso_memory where, int64_t n, double lambda, double tol,
                           const double* theta0, double* theta_out, glasso_result* res) {
  if (!h || !S) return GLASSO_ERR_ARG;
  if (!valid_problem(n, lambda, tol) || (s_dtype != GLASSO_F64 && s_dtype != GLASSO_F32) ||
      (where != GLASSO_HOST && where != GLASSO_DEVICE))
    return fail(h, GLASSO_ERR_ARG, "invalid n, lambda, tol, dtype or memory kind");
  std::lock_guard<std::mutex> lock(h->mu);
  return guarded(h, [&] {
    glasso::SolveOut o = h->engine->solve(S, s_dtype == GLASSO_F32, where == GLASSO_DEVICE, n,
                                          lambda, tol, theta0, theta_out);
    fill_result(res, o);
    return (glasso_status)o.status;
  });
}

glasso_status glasso_begin(glasso_handle* h, const void* S, glasso_dtype s_dtype,
                           glasso_memory where, int64_t n, double lambda, const double* theta0) {
  if (!h || !S) return GLASSO_ERR_ARG;
  if (!valid_problem(n, lambda, 0.0) || (s_dtype != GLASSO_F64 && s_dtype != GLASSO_F32) ||
      (where != GLASSO_HOST && where != GLASSO_DEVICE))
    return fail(h, GLASSO_ERR_ARG, "invalid n, lambda, dtype or memory kind");
  std::lock_guard<std::mutex> lock(h->mu);
  return guarded(h, [&] {
    h->engine->begin(S, s_dtype == GLASSO_F32, where == GLASSO_DEVICE, n, lambda, theta0);
    return GLASSO_OK;
  });
}

glasso_status glasso_step(glasso_handle* h, double tol, glasso_result* res) {
  if (!h || !(tol >= 0.0)) return GLASSO_ERR_ARG;
  std::lock_guard<std::mutex> lock(h->mu);
  return guarded(h, [&] {
    const int64_t l0 = glasso::thread_launches();
    const int t0 = h->engine->state().out.trials;
    const int st = h->engine->step(tol, INT32_MAX, false);
    if (res) {
      const glasso::SolveState& s = h->engine->state();
      glasso::SolveOut o;
      o.status = st < 0 ? GLASSO_PENDING : st;
      o.iterations = s.k;
      o.trials = s.out.trials - t0;
      o.r = s.out.r;
      o.z_fro = s.out.z_fro;
      o.nnz = s.out.nnz;
      o.F = s.F;
      o.logdet = s.ld_A;
      o.launches = glasso::thread_launches() - l0;
      if (o.trials > 0) {  // this call formed a direction and ran a line search
        o.step_t = s.out.step_t;
        o.step_dF = s.out.step_dF;
        o.step_tier = s.out.step_tier;
        o.step_fallback = s.out.step_fallback;
      }
      fill_result(res, o);
    }
    return st < 0 ? GLASSO_PENDING : (glasso_status)st;
  });
}

glasso_status glasso_end(glasso_handle* h, double* theta_out, glasso_result* res) {
  if (!h) return GLASSO_ERR_ARG;
  std::lock_guard<std::mutex> lock(h->mu);
  return guarded(h, [&] {
    glasso::SolveOut o = h->engine->finish(theta_out);
    o.status = GLASSO_OK;
    fill_result(res, o);
    return GLASSO_OK;
  });
}

glasso_status glasso_profile_start(glasso_handle* h) {
  if (!h) return GLASSO_ERR_ARG;
  std::lock_guard<std::mutex> lock(h->mu);
  return guarded(h, [&] {
    h->engine->prof.start();
    return GLASSO_OK;
  });
}

glasso_status glasso_profile_stop(glasso_handle* h, glasso_profile* out) {
  if (!h || !out) return GLASSO_ERR_ARG;
  std::lock_guard<std::mutex> lock(h->mu);
  return guarded(h, [&] {
    h->engine->prof.collect(out);
    return GLASSO_OK;
  });
}

glasso_status glasso_probe_fp64_peak(int device, double* tflops) {
  if (!tflops) return GLASSO_ERR_ARG;
  return guarded(nullptr, [&] {
    *tflops = glasso::probe_fp64_tflops(device);
    return GLASSO_OK;
  });
}

glasso_status glasso_workspace_bytes(int64_t n, size_t* bytes) {
  if (!bytes || n < 1 || n > ((int64_t)1 << 20)) return GLASSO_ERR_ARG;
  *bytes = glasso::Workspace::bytes_for((int)glasso::round_up(n, glasso::kPad));
  return GLASSO_OK;
}

glasso_status glasso_solve_batch(glasso_handle* h, const glasso_problem* probs, int32_t count,
                                 glasso_result* results) {
  if (!h || (count > 0 && (!probs || !results)) || count < 0) return GLASSO_ERR_ARG;
  for (int32_t i = 0; i < count; ++i) {
    const glasso_problem& p = probs[i];
    if (!p.S || p.n_lambda < 1 || !p.lambdas || (p.dtype != GLASSO_F64 && p.dtype != GLASSO_F32))
      return fail(h, GLASSO_ERR_ARG, "invalid problem " + std::to_string(i));
    for (int32_t j = 0; j < p.n_lambda; ++j)
      if (!valid_problem(p.n, p.lambdas[j], p.tol))
        return fail(h, GLASSO_ERR_ARG, "invalid n, lambda or tol in problem " + std::to_string(i));
  }
  std::lock_guard<std::mutex> lock(h->mu);
  return guarded(h, [&] { return (glasso_status)glasso::solve_batch(*h->engine, probs, count, results); });
}

glasso_status glasso_submit(glasso_handle* h, const glasso_request* req, uint64_t* ticket) {
  if (!h || !req || !ticket || !req->S) return GLASSO_ERR_ARG;
  if (!valid_problem(req->n, req->lambda, req->tol) ||
      (req->dtype != GLASSO_F64 && req->dtype != GLASSO_F32))
    return fail(h, GLASSO_ERR_ARG, "invalid request");
  return guarded(h, [&] {
    {
      std::lock_guard<std::mutex> lock(h->mu);
      if (!h->server) h->server = std::make_unique<glasso::Server>(h->cfg);
    }
    return (glasso_status)h->server->submit(*req, ticket);
  });
}

glasso_status glasso_poll(glasso_handle* h, uint64_t ticket, glasso_result* res, double* theta_out) {
  if (!h) return GLASSO_ERR_ARG;
  if (!h->server) return fail(h, GLASSO_ERR_ARG, "no request was submitted");
  return guarded(h, [&] { return (glasso_status)h->server->poll(ticket, res, theta_out); });
}

glasso_status glasso_op_cholesky(glasso_handle* h, const double* A, int64_t n, double* L,
                                 int32_t* pd, double* logdet) {
  if (!h || !A || !L || !pd || !logdet || n < 1) return GLASSO_ERR_ARG;
  std::lock_guard<std::mutex> lock(h->mu);
  return guarded(h, [&] {
    int p = 0;
    h->engine->op_cholesky(A, n, L, &p, logdet);
    *pd = p;
    return GLASSO_OK;
  });
}

glasso_status glasso_op_inverse(glasso_handle* h, const double* A, int64_t n, double* W) {
  if (!h || !A || !W || n < 1) return GLASSO_ERR_ARG;
  std::lock_guard<std::mutex> lock(h->mu);
  return guarded(h, [&] {
    return h->engine->op_inverse(A, n, W) ? GLASSO_OK
                                          : fail(h, GLASSO_ERR_NOT_PD, "A is not positive definite");
  });
}

glasso_status glasso_op_gradient(glasso_handle* h, const double* S, const double* A,
                                 const double* W, int64_t n, double lambda, double* X,
                                 int8_t* code, double sums[4]) {
  if (!h || !S || !A || !W || !X || !code || !sums || n < 1 || !(lambda > 0.0)) return GLASSO_ERR_ARG;
  std::lock_guard<std::mutex> lock(h->mu);
  return guarded(h, [&] {
    h->engine->op_gradient(S, A, W, n, lambda, X, code, sums);
    return GLASSO_OK;
  });
}

glasso_status glasso_op_sandwich(glasso_handle* h, const double* A, const double* X, int64_t n,
                                 double* Y) {
  if (!h || !A || !X || !Y || n < 1) return GLASSO_ERR_ARG;
  std::lock_guard<std::mutex> lock(h->mu);
  return guarded(h, [&] {
    h->engine->op_sandwich(A, X, n, Y);
    return GLASSO_OK;
  });
}

glasso_status glasso_op_trial(glasso_handle* h, const double* A, const double* Y,
                              const int8_t* code, int64_t n, double lambda, double t, double* At) {
  if (!h || !A || !Y || !code || !At || n < 1 || !(lambda > 0.0) || !(t > 0.0)) return GLASSO_ERR_ARG;
  std::lock_guard<std::mutex> lock(h->mu);
  return guarded(h, [&] {
    h->engine->op_trial(A, Y, code, n, lambda, t, At);
    return GLASSO_OK;
  });
}

}  // extern "C"
