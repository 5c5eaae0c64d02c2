// Batched regularisation paths and the continuous-batching request server.
#pragma once
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>
#include "engine.h"

namespace glasso {

bool tc_available();

// Problems run concurrently, one worker (engine + stream) per slot; each problem's lambda
// path runs in descending order on one worker, every solve warm-started from the previous.
int solve_batch(Engine& main, const glasso_problem* probs, int32_t count, glasso_result* results);

// Continuous batching: requests are admitted onto slots (one engine and stream each) while
// their device memory fits the HBM budget; the solves of different slots overlap on the GPU.
// Solutions are kept on the device for warm starts (Theta, its inverse Cholesky factor and
// W = Theta^{-1}), under the same budget, evicted least recently used.
class Server {
 public:
  explicit Server(const glasso_config& cfg);
  ~Server();
  int submit(const glasso_request& req, uint64_t* ticket);
  int poll(uint64_t ticket, glasso_result* res, double* theta_out);

 private:
  struct Request {
    uint64_t id;
    int64_t n;
    std::shared_ptr<const std::vector<double>> S;  // promoted to FP64; shared per dataset id
    double lam, tol;
    int64_t dataset;
    double t_submit;
    int skipped = 0;        // admissions that went past this request while it waited at the head
  };
  struct Finished {
    glasso_result res;
    std::vector<double> theta;
  };
  // One resident solution: Theta, its inverse factor and W, padded np x np, in one allocation.
  struct Resident {
    int64_t n = 0;
    int np = 0;
    double* mem = nullptr;  // 3 np^2 doubles: theta | li | w
    double logdet = 0.0;
    uint64_t last_use = 0;
    int readers = 0;        // slots copying from it right now (not evictable)
    size_t bytes() const { return (size_t)3 * np * np * sizeof(double); }
  };
  void worker(int slot);
  // Under mu_: pick the request this idle slot runs next (queue order, past a head that does
  // not fit for a bounded number of admissions), making room by evicting resident solutions
  // and, when the slot's own workspace is what blocks it, by shrinking that workspace.
  bool admit(int slot, Request& out, bool& shrink);
  bool evict_for(size_t need);  // under mu_: evict LRU residents until need bytes fit
  static void free_evicted(std::vector<double*>& victims, cudaStream_t st);
  std::vector<double*> to_free_;  // evicted residents not yet freed (under mu_)
  void fail_all_queued(int status, const std::string& msg);  // under mu_

  glasso_config cfg_;
  size_t budget_ = 0;             // bytes for workspaces and residents (0: no limit)
  size_t resident_cap_ = 0;       // bytes residents may take when there is no budget
  std::mutex mu_;
  std::condition_variable cv_;
  std::deque<Request> queue_;
  std::unordered_map<uint64_t, Finished> done_;
  std::unordered_map<uint64_t, int> running_;
  std::vector<size_t> slot_bytes_;
  size_t in_use_ = 0;             // workspace bytes of all slots
  size_t resident_bytes_ = 0;
  uint64_t next_id_ = 1, clock_ = 0;
  bool stop_ = false;
  int alive_ = 0, started_ = 0;   // slots whose engine was built / slots that finished starting
  int dead_status_ = 0;
  std::string dead_msg_;
  // dataset id -> lambda -> resident solution
  std::unordered_map<int64_t, std::map<double, Resident>> cache_;
  // dataset id -> its S (host, FP64): requests of one id share S (glasso_request), so a
  // stream of many requests over few datasets holds one copy per dataset
  std::unordered_map<int64_t, std::shared_ptr<const std::vector<double>>> datasets_;
  std::vector<std::thread> threads_;
};

double monotonic_seconds();

}  // namespace glasso
