// Concurrent execution of independent st-HOSVD plans (Alg. 2 on several
// tensors at once).
//
// One tensor's st-HOSVD is a chain: each mode's Gram needs the previous
// mode's TTM, and the eigensolver between them runs on one or a few CTAs
// while the other SMs idle.  Plans of independent tensors on their own
// streams fill those SMs: one tensor's eigensolver overlaps another's Gram.
// The eigensolver reads a convergence summary on the host between its
// launch groups, so each plan's host code runs on its own thread; the
// threads come from a persistent pool (they keep their capture streams and
// graph-cache entries between calls).
#include <cuda_runtime.h>

#include <condition_variable>
#include <deque>
#include <functional>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "atk_internal.cuh"

namespace atk {
namespace {

// Persistent worker threads.  run(count, f) calls f(0) on the calling thread
// and f(1) .. f(count-1) on workers, and returns when every call has returned.
class HostPool {
 public:
  void run(int count, const std::function<void(int)>& f) {
    if (count <= 0) return;
    std::unique_lock<std::mutex> lk(mu_);
    while ((int)workers_ < count - 1) {
      std::thread(&HostPool::loop, this).detach();  // the pool lives until exit
      ++workers_;
    }
    int pending = count - 1;
    std::condition_variable done;
    for (int i = 1; i < count; ++i)
      queue_.push_back([&, i] {
        f(i);
        std::lock_guard<std::mutex> g(mu_);
        if (--pending == 0) done.notify_all();
      });
    cv_.notify_all();
    lk.unlock();
    f(0);
    lk.lock();
    done.wait(lk, [&] { return pending == 0; });
  }

 private:
  void loop() {
    std::unique_lock<std::mutex> lk(mu_);
    for (;;) {
      cv_.wait(lk, [&] { return !queue_.empty(); });
      std::function<void()> task = std::move(queue_.front());
      queue_.pop_front();
      lk.unlock();
      task();
      lk.lock();
    }
  }
  std::mutex mu_;
  std::condition_variable cv_;
  std::deque<std::function<void()>> queue_;
  size_t workers_ = 0;
};

HostPool& pool() {
  static HostPool* p = new HostPool();  // never destroyed: workers are detached
  return *p;
}

// Run body(i) for every plan, plan i on a thread whose current device is the
// caller's.  Returns the first failing status in plan order, with its message.
int run_plans(int count, const atucker_plan_t* plans, const std::function<int(int)>& body) {
  if (count <= 0 || !plans) { set_error("run_many: need count >= 1 and a plan array"); return ATK_EINVAL; }
  for (int i = 0; i < count; ++i) {
    if (!plans[i]) { set_error("run_many: null plan"); return ATK_EINVAL; }
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) { set_error("run_many: a plan appears twice"); return ATK_EINVAL; }
  }
  int dev = 0;
  ATK_CUDA(cudaGetDevice(&dev));
  std::vector<int> status(count, ATK_OK);
  std::vector<std::string> msg(count);
  pool().run(count, [&](int i) {
    if (i > 0 && cudaSetDevice(dev) != cudaSuccess) {
      status[i] = ATK_ECUDA;
      msg[i] = "run_many: cudaSetDevice failed on a worker thread";
      return;
    }
    status[i] = body(i);
    if (status[i] != ATK_OK) msg[i] = atucker_last_error();
  });
  for (int i = 0; i < count; ++i)
    if (status[i] != ATK_OK) {
      set_error("plan " + std::to_string(i) + ": " + msg[i]);
      return status[i];
    }
  return ATK_OK;
}

}  // namespace
}  // namespace atk

using namespace atk;

extern "C" {

int atucker_sthosvd_many(int count, const atucker_plan_t* plans, const float* const* xs, float* const* cores,
                         float* const* factors, double* const* discarded) {
  if (!xs || !cores || !factors) { set_error("run_many: null array"); return ATK_EINVAL; }
  return run_plans(count, plans, [&](int i) {
    return atucker_sthosvd(plans[i], xs[i], cores[i], factors[i], discarded ? discarded[i] : nullptr);
  });
}

int atucker_sthosvd_host_many(int count, const atucker_plan_t* plans, const float* const* xs_host,
                              float* const* cores_host, float* const* factors_host,
                              double* const* discarded_host) {
  if (!xs_host || !cores_host || !factors_host) { set_error("run_many: null array"); return ATK_EINVAL; }
  return run_plans(count, plans, [&](int i) {
    return atucker_sthosvd_host(plans[i], xs_host[i], cores_host[i], factors_host[i],
                                discarded_host ? discarded_host[i] : nullptr);
  });
}

}  // extern "C"
