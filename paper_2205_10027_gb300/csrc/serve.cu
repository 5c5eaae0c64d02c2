// Batched lambda paths and the request server.  Concurrency comes from several engines,
// each with its own stream and workspace on the same GPU: kernels of different problems
// overlap on the device while each problem's iteration stays in order.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>
#include "gemm_tc.h"
#include "serve.h"

namespace glasso {

double monotonic_seconds() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

namespace {
void to_result(glasso_result* r, const SolveOut& o) {
  std::memset(r, 0, sizeof(*r));
  r->status = o.status;
  r->iterations = o.iterations;
  r->trials = o.trials;
  r->nnz = (int32_t)o.nnz;
  r->rel_kkt_l1 = o.r;
  r->min_subgrad_fro = o.z_fro;
  r->objective = o.F;
  r->logdet = o.logdet;
  r->seconds = o.seconds;
  r->kernel_launches = o.launches;
}
}  // namespace

int solve_batch(Engine& main, const glasso_problem* probs, int32_t count, glasso_result* results) {
  if (count == 0) return GLASSO_OK;
  const glasso_config cfg = main.config();
  const int slots = std::max(1, std::min<int>(cfg.serve_slots, count));
  // larger problems first so the tail of the batch is short
  std::vector<int32_t> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return probs[a].n > probs[b].n; });
  std::atomic<int32_t> next{0};
  std::atomic<int> first_error{GLASSO_OK};
  std::mutex err_mu;
  auto run = [&](Engine& eng) {
    for (;;) {
      const int32_t q = next.fetch_add(1);
      if (q >= count || first_error.load() != GLASSO_OK) return;
      const int32_t i = order[q];
      const glasso_problem& p = probs[i];
      std::vector<int32_t> lo(p.n_lambda);
      std::iota(lo.begin(), lo.end(), 0);
      std::stable_sort(lo.begin(), lo.end(), [&](int32_t a, int32_t b) { return p.lambdas[a] > p.lambdas[b]; });
      std::vector<double> theta((size_t)p.n * p.n);
      bool have = false;
      for (int32_t j : lo) {
        try {
          SolveOut o = eng.solve(p.S, p.dtype == GLASSO_F32, false, p.n, p.lambdas[j], p.tol,
                                 have ? theta.data() : nullptr, theta.data());
          have = true;
          to_result(&results[(size_t)i * p.n_lambda + j], o);
          if (p.theta_out)
            std::memcpy(p.theta_out + (size_t)j * p.n * p.n, theta.data(), sizeof(double) * p.n * p.n);
        } catch (const Error& e) {
          int expected = GLASSO_OK;
          first_error.compare_exchange_strong(expected, e.status);
          return;
        }
      }
    }
  };
  std::vector<std::unique_ptr<Engine>> extra;
  std::vector<std::thread> th;
  for (int s = 1; s < slots; ++s) {
    glasso_config c = cfg;
    c.stream = nullptr;
    extra.push_back(std::make_unique<Engine>(c));
  }
  for (int s = 1; s < slots; ++s) th.emplace_back([&, s] { cudaSetDevice(cfg.device); run(*extra[s - 1]); });
  run(main);
  for (auto& t : th) t.join();
  return first_error.load();
}

// ------------------------------------------------------------------------------------------
Server::Server(const glasso_config& cfg) : cfg_(cfg) {
  const int slots = std::max(1, cfg.serve_slots);
  slot_bytes_.assign(slots, 0);
  for (int s = 0; s < slots; ++s) threads_.emplace_back([this, s] { worker(s); });
}

Server::~Server() {
  {
    std::lock_guard<std::mutex> lk(mu_);
    stop_ = true;
  }
  cv_.notify_all();
  for (auto& t : threads_) t.join();
}

int Server::submit(const glasso_request& req, uint64_t* ticket) {
  const int np = (int)round_up(req.n, kPad);
  if (cfg_.hbm_budget_bytes && Workspace::bytes_for(np) > cfg_.hbm_budget_bytes)
    throw Error(GLASSO_ERR_BUDGET, "request can never fit the HBM budget");
  Request r;
  r.n = req.n;
  r.S.resize((size_t)req.n * req.n);
  if (req.dtype == GLASSO_F32) {
    const float* s = (const float*)req.S;
    for (size_t e = 0; e < r.S.size(); ++e) r.S[e] = (double)s[e];
  } else {
    std::memcpy(r.S.data(), req.S, sizeof(double) * r.S.size());
  }
  r.lam = req.lambda;
  r.tol = req.tol;
  r.dataset = req.dataset_id;
  r.t_submit = monotonic_seconds();
  {
    std::lock_guard<std::mutex> lk(mu_);
    r.id = next_id_++;
    *ticket = r.id;
    queue_.push_back(std::move(r));
  }
  cv_.notify_all();
  return GLASSO_OK;
}

int Server::poll(uint64_t ticket, glasso_result* res, double* theta_out) {
  std::lock_guard<std::mutex> lk(mu_);
  auto it = done_.find(ticket);
  if (it == done_.end()) {
    if (running_.count(ticket)) return GLASSO_PENDING;
    for (const auto& q : queue_)
      if (q.id == ticket) return GLASSO_PENDING;
    throw Error(GLASSO_ERR_ARG, "unknown ticket");
  }
  if (res) *res = it->second.res;
  if (theta_out) std::memcpy(theta_out, it->second.theta.data(), sizeof(double) * it->second.theta.size());
  const int st = it->second.res.status;
  done_.erase(it);
  return st;
}

void Server::worker(int slot) {
  cudaSetDevice(cfg_.device);
  glasso_config c = cfg_;
  c.stream = nullptr;
  std::unique_ptr<Engine> eng;
  try {
    eng = std::make_unique<Engine>(c);
  } catch (...) {
    return;
  }
  for (;;) {
    Request r;
    std::shared_ptr<const std::vector<double>> warm;
    {
      std::unique_lock<std::mutex> lk(mu_);
      cv_.wait(lk, [&] {
        if (stop_) return true;
        if (queue_.empty()) return false;
        const size_t need = Workspace::bytes_for((int)round_up(queue_.front().n, kPad));
        const size_t mine = std::max(need, slot_bytes_[slot]);
        return !cfg_.hbm_budget_bytes || in_use_ - slot_bytes_[slot] + mine <= cfg_.hbm_budget_bytes;
      });
      if (stop_) return;
      r = std::move(queue_.front());
      queue_.pop_front();
      const size_t need = Workspace::bytes_for((int)round_up(r.n, kPad));
      if (need > slot_bytes_[slot]) {
        in_use_ += need - slot_bytes_[slot];
        slot_bytes_[slot] = need;
      }
      running_[r.id] = slot;
      if (r.dataset >= 0) {
        auto ci = cache_.find(r.dataset);
        if (ci != cache_.end() && !ci->second.empty()) {
          auto hi = ci->second.lower_bound(r.lam);
          auto best = ci->second.end();
          double bd = INFINITY;
          for (auto cand : {hi, hi == ci->second.begin() ? ci->second.end() : std::prev(hi)}) {
            if (cand == ci->second.end()) continue;
            const double d = std::fabs(cand->first - r.lam);
            if (d < bd) { bd = d; best = cand; }
          }
          if (best != ci->second.end() && best->second->size() == r.S.size()) warm = best->second;
        }
      }
    }
    Finished f;
    std::memset(&f.res, 0, sizeof(f.res));
    const double t_start = monotonic_seconds();
    f.theta.resize(r.S.size());
    try {
      SolveOut o = eng->solve(r.S.data(), false, false, r.n, r.lam, r.tol,
                              warm ? warm->data() : nullptr, f.theta.data());
      to_result(&f.res, o);
    } catch (const Error& e) {
      f.res.status = e.status;
    }
    f.res.t_submit = r.t_submit;
    f.res.t_start = t_start;
    f.res.t_done = monotonic_seconds();
    {
      std::lock_guard<std::mutex> lk(mu_);
      running_.erase(r.id);
      if (r.dataset >= 0 && (f.res.status == GLASSO_OK))
        cache_[r.dataset][r.lam] = std::make_shared<const std::vector<double>>(f.theta);
      done_[r.id] = std::move(f);
    }
    cv_.notify_all();
  }
}

}  // namespace glasso
