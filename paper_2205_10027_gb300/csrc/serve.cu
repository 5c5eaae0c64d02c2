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
    extra.back()->set_blocking_sync(slots > 1);
  }
  main.set_blocking_sync(slots > 1);
  for (int s = 1; s < slots; ++s) th.emplace_back([&, s] { cudaSetDevice(cfg.device); run(*extra[s - 1]); });
  run(main);
  for (auto& t : th) t.join();
  main.set_blocking_sync(false);
  return first_error.load();
}

// ------------------------------------------------------------------------------------------
namespace {
// How many admissions may go past a queue head that does not fit, per slot, before the slots
// stop admitting anything else and give their workspaces back until it fits.
constexpr int kSkipsPerSlot = 4;
}  // namespace

Server::Server(const glasso_config& cfg) : cfg_(cfg) {
  const int slots = std::max(1, cfg.serve_slots);
  budget_ = cfg.hbm_budget_bytes;
  if (!budget_) {
    // no budget: residents may hold a quarter of the memory free at start
    size_t fr = 0, tot = 0;
    CUDA_CHECK(cudaSetDevice(cfg.device));
    CUDA_CHECK(cudaMemGetInfo(&fr, &tot));
    resident_cap_ = fr / 4;
  }
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
  cudaSetDevice(cfg_.device);
  cudaDeviceSynchronize();
  for (auto& d : cache_)
    for (auto& e : d.second) cudaFree(e.second.mem);
  for (double* p : to_free_) cudaFree(p);
}

int Server::submit(const glasso_request& req, uint64_t* ticket) {
  const int np = (int)round_up(req.n, kPad);
  if (budget_ && Workspace::bytes_for(np) > budget_)
    throw Error(GLASSO_ERR_BUDGET, "request can never fit the HBM budget");
  {
    std::lock_guard<std::mutex> lk(mu_);
    if (started_ == (int)slot_bytes_.size() && alive_ == 0)
      throw Error(dead_status_ ? dead_status_ : GLASSO_ERR_CUDA, "no serving slot is running: " + dead_msg_);
  }
  Request r;
  r.n = req.n;
  if (req.dataset_id >= 0) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = datasets_.find(req.dataset_id);
    if (it != datasets_.end() && it->second->size() == (size_t)req.n * req.n) r.S = it->second;
  }
  if (!r.S) {
    auto v = std::make_shared<std::vector<double>>((size_t)req.n * req.n);
    if (req.dtype == GLASSO_F32) {
      const float* s = (const float*)req.S;
      for (size_t e = 0; e < v->size(); ++e) (*v)[e] = (double)s[e];
    } else {
      std::memcpy(v->data(), req.S, sizeof(double) * v->size());
    }
    r.S = v;
    if (req.dataset_id >= 0) {
      std::lock_guard<std::mutex> lk(mu_);
      datasets_[req.dataset_id] = r.S;
    }
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
    if (started_ == (int)slot_bytes_.size() && alive_ == 0) fail_all_queued(dead_status_, dead_msg_);
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
  if (theta_out && !it->second.theta.empty())
    std::memcpy(theta_out, it->second.theta.data(), sizeof(double) * it->second.theta.size());
  const int st = it->second.res.status;
  done_.erase(it);
  return st;
}

void Server::fail_all_queued(int status, const std::string& msg) {
  (void)msg;
  for (auto& q : queue_) {
    Finished f;
    std::memset(&f.res, 0, sizeof(f.res));
    f.res.status = status ? status : GLASSO_ERR_CUDA;
    f.res.t_submit = q.t_submit;
    done_[q.id] = std::move(f);
  }
  queue_.clear();
}

bool Server::evict_for(size_t need) {
  // residents fit when workspaces + residents + need stay within the budget (or, with no
  // budget, residents + need within the resident cap)
  auto over = [&]() {
    return budget_ ? in_use_ + resident_bytes_ + need > budget_ : resident_bytes_ + need > resident_cap_;
  };
  while (over()) {
    std::map<double, Resident>* best_map = nullptr;
    std::map<double, Resident>::iterator best;
    uint64_t oldest = UINT64_MAX;
    for (auto& d : cache_)
      for (auto it = d.second.begin(); it != d.second.end(); ++it)
        if (it->second.readers == 0 && it->second.last_use < oldest) {
          oldest = it->second.last_use;
          best_map = &d.second;
          best = it;
        }
    if (!best_map) return false;
    resident_bytes_ -= best->second.bytes();
    to_free_.push_back(best->second.mem);  // freed once the lock is released
    best_map->erase(best);
  }
  return true;
}

// Stream-ordered frees of evicted residents (no stream uses them: a reader synchronises its
// stream before it lets go of an entry), outside the lock so no slot waits on them.
void Server::free_evicted(std::vector<double*>& victims, cudaStream_t st) {
  for (double* p : victims) cudaFreeAsync(p, st);
  victims.clear();
}

bool Server::admit(int slot, Request& out, bool& shrink) {
  if (queue_.empty()) return false;
  const size_t mine = slot_bytes_[slot];
  const size_t others = in_use_ - mine;
  size_t evictable = 0;
  for (auto& d : cache_)
    for (auto& e : d.second)
      if (e.second.readers == 0) evictable += e.second.bytes();
  // 1: fits keeping this slot's workspace, 2: fits once the slot shrinks it to the request's
  auto fit = [&](size_t need) -> int {
    if (!budget_) return 1;
    const size_t floor = resident_bytes_ - evictable;  // residents that cannot be evicted now
    if (others + std::max(need, mine) + floor <= budget_) return 1;
    if (others + need + floor <= budget_) return 2;
    return 0;
  };
  auto take = [&](std::deque<Request>::iterator it, int how) {
    const size_t need = Workspace::bytes_for((int)round_up(it->n, kPad));
    const size_t ws = how == 1 ? std::max(need, mine) : need;
    in_use_ = others + ws;
    slot_bytes_[slot] = ws;
    shrink = how == 2 && mine > 0;
    evict_for(0);  // residents give way to the admitted workspace
    out = std::move(*it);
    queue_.erase(it);
  };
  auto head = queue_.begin();
  const int h = fit(Workspace::bytes_for((int)round_up(head->n, kPad)));
  if (h) {
    take(head, h);
    return true;
  }
  // the head does not fit now: later requests may go first a bounded number of times
  if (head->skipped >= kSkipsPerSlot * (int)slot_bytes_.size()) return false;
  for (auto it = std::next(head); it != queue_.end(); ++it) {
    const int f = fit(Workspace::bytes_for((int)round_up(it->n, kPad)));
    if (f) {
      ++head->skipped;
      take(it, f);
      return true;
    }
  }
  return false;
}

void Server::worker(int slot) {
  cudaSetDevice(cfg_.device);
  glasso_config c = cfg_;
  c.stream = nullptr;
  std::unique_ptr<Engine> eng;
  int fail_status = 0;
  std::string fail_msg;
  try {
    // GLASSO_TEST_FAIL_SLOTS=k: the first k slots report an allocation failure instead of
    // building their engine (host-side failure injection for the tests of this path)
    const char* tf = std::getenv("GLASSO_TEST_FAIL_SLOTS");
    if (tf && slot < std::atoi(tf)) throw Error(GLASSO_ERR_OOM, "slot engine allocation failed (injected)");
    eng = std::make_unique<Engine>(c);
    eng->set_blocking_sync(slot_bytes_.size() > 1);
  } catch (const Error& e) {
    fail_status = e.status;
    fail_msg = e.what();
  } catch (const std::exception& e) {
    fail_status = GLASSO_ERR_CUDA;
    fail_msg = e.what();
  }
  {
    std::lock_guard<std::mutex> lk(mu_);
    ++started_;
    if (eng) {
      ++alive_;
    } else if (!dead_status_) {
      dead_status_ = fail_status;
      dead_msg_ = fail_msg;
    }
    if (started_ == (int)slot_bytes_.size() && alive_ == 0) fail_all_queued(dead_status_, dead_msg_);
  }
  cv_.notify_all();
  if (!eng) return;
  std::vector<double*> victims;
  for (;;) {
    Request r;
    bool shrink = false;
    Resident* warm = nullptr;
    Engine::Resident wr;
    {
      std::unique_lock<std::mutex> lk(mu_);
      for (;;) {
        if (stop_) return;
        if (admit(slot, r, shrink)) {
          victims.swap(to_free_);
          break;
        }
        if (!queue_.empty() && slot_bytes_[slot] > 0) {
          // a queued request waits and this slot is idle: give its workspace back
          in_use_ -= slot_bytes_[slot];
          slot_bytes_[slot] = 0;
          lk.unlock();
          eng->release_workspace();
          lk.lock();
          cv_.notify_all();
          continue;
        }
        cv_.wait(lk);
      }
      running_[r.id] = slot;
      if (r.dataset >= 0) {
        // warm start: the resident solution of the same dataset with the nearest lambda
        auto ci = cache_.find(r.dataset);
        if (ci != cache_.end() && !ci->second.empty()) {
          auto hi = ci->second.lower_bound(r.lam);
          double bd = INFINITY;
          for (auto cand : {hi, hi == ci->second.begin() ? ci->second.end() : std::prev(hi)}) {
            if (cand == ci->second.end() || cand->second.n != r.n) continue;
            const double d = std::fabs(cand->first - r.lam);
            if (d < bd) {
              bd = d;
              warm = &cand->second;
            }
          }
          if (warm) {
            ++warm->readers;
            warm->last_use = ++clock_;
            const size_t m = (size_t)warm->np * warm->np;
            wr.n = warm->n;
            wr.np = warm->np;
            wr.theta = warm->mem;
            wr.li = warm->mem + m;
            wr.w = warm->mem + 2 * m;
            wr.logdet = warm->logdet;
          }
        }
      }
    }
    free_evicted(victims, eng->stream());
    if (shrink) eng->release_workspace();
    Finished f;
    std::memset(&f.res, 0, sizeof(f.res));
    const double t_start = monotonic_seconds();
    f.theta.resize(r.S->size());
    bool solved = false;
    try {
      SolveOut o = warm ? eng->solve_resident(r.S->data(), false, r.n, r.lam, r.tol, wr, f.theta.data())
                        : eng->solve(r.S->data(), false, false, r.n, r.lam, r.tol, nullptr, f.theta.data());
      to_result(&f.res, o);
      solved = true;
    } catch (const Error& e) {
      f.res.status = e.status;
    }
    f.res.t_submit = r.t_submit;
    f.res.t_start = t_start;
    f.res.t_done = monotonic_seconds();
    // keep the solution resident for later warm starts (same dataset id)
    double* mem = nullptr;
    const int np = (int)round_up(r.n, kPad);
    const size_t rbytes = (size_t)3 * np * np * sizeof(double);
    if (solved && f.res.status == GLASSO_OK && r.dataset >= 0) {
      bool room;
      {
        std::lock_guard<std::mutex> lk(mu_);
        if (warm) --warm->readers;
        warm = nullptr;
        room = evict_for(rbytes);
        if (room) resident_bytes_ += rbytes;  // reserved
        victims.swap(to_free_);
      }
      free_evicted(victims, eng->stream());
      if (room) {
        double logdet = 0.0;
        bool ok = cudaMallocAsync((void**)&mem, rbytes, eng->stream()) == cudaSuccess;
        if (!ok) cudaGetLastError();
        if (ok) {
          try {
            const size_t m = (size_t)np * np;
            logdet = eng->export_resident(mem, mem + m, mem + 2 * m);
          } catch (const Error&) {
            ok = false;
          }
        }
        std::lock_guard<std::mutex> lk(mu_);
        auto& slotmap = cache_[r.dataset];
        auto old = slotmap.find(r.lam);
        if (ok && (old == slotmap.end() || old->second.readers == 0)) {
          if (old != slotmap.end()) {
            resident_bytes_ -= old->second.bytes();
            to_free_.push_back(old->second.mem);
            slotmap.erase(old);
          }
          Resident e;
          e.n = r.n;
          e.np = np;
          e.mem = mem;
          e.logdet = logdet;
          e.last_use = ++clock_;
          slotmap.emplace(r.lam, e);
        } else {
          resident_bytes_ -= rbytes;
          if (mem) to_free_.push_back(mem);
        }
        victims.swap(to_free_);
      }
      free_evicted(victims, eng->stream());
    }
    {
      std::lock_guard<std::mutex> lk(mu_);
      if (warm) --warm->readers;
      running_.erase(r.id);
      done_[r.id] = std::move(f);
    }
    cv_.notify_all();
  }
}

}  // namespace glasso
