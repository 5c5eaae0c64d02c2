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
    std::vector<double> S;  // promoted to FP64
    double lam, tol;
    int64_t dataset;
    double t_submit;
  };
  struct Finished {
    glasso_result res;
    std::vector<double> theta;
  };
  void worker(int slot);

  glasso_config cfg_;
  std::mutex mu_;
  std::condition_variable cv_;
  std::deque<Request> queue_;
  std::unordered_map<uint64_t, Finished> done_;
  std::unordered_map<uint64_t, int> running_;
  std::vector<size_t> slot_bytes_;
  size_t in_use_ = 0;
  uint64_t next_id_ = 1;
  bool stop_ = false;
  // warm-start cache: dataset id -> lambda -> solution
  std::unordered_map<int64_t, std::map<double, std::shared_ptr<const std::vector<double>>>> cache_;
  std::vector<std::thread> threads_;
};

double monotonic_seconds();

}  // namespace glasso
