// trace.cuh -- per-context launch accounting: a count of every kernel the
// library launches, and (when switched on) CUDA events recorded on the
// launching stream around each launch, read back as per-kernel device times.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

namespace drc {

class Tracer {
 public:
  ~Tracer() {
    for (auto &r : pending_) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : pool_) cudaEventDestroy(e);
  }

  // Call immediately before a kernel launch on `st`.
  void begin(const char *name, cudaStream_t st) {
    ++launches_;
    open_ = false;
    if (!timing_) return;
    Rec r;
    r.name = name_index(name);
    r.a = take();
    r.b = take();
    if (!r.a || !r.b) {  // no event: leave this launch untimed
      give(r.a);
      give(r.b);
      ++untimed_;
      return;
    }
    cudaEventRecord(r.a, st);
    pending_.push_back(r);
    open_ = true;
  }
  // Call immediately after the launch (same stream).
  void end(cudaStream_t st) {
    if (open_) cudaEventRecord(pending_.back().b, st);
    open_ = false;
  }

  unsigned long long launches() const { return launches_; }
  // Kernels launched inside a graph (counted, not timed one by one).
  void add_launches(unsigned long long n) { launches_ += n; }
  void set_timing(bool on) { timing_ = on; }

  struct Total {
    std::string name;
    long long launches = 0;
    double ms = 0.0;
  };
  // Synchronise on the recorded events and fold them into the per-name
  // totals, which are returned and cleared.
  std::vector<Total> drain() {
    for (auto &r : pending_) {
      float ms = 0.f;
      if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
        totals_[r.name].launches += 1;
        totals_[r.name].ms += ms;
      }
      cudaGetLastError();
      give(r.a);
      give(r.b);
    }
    pending_.clear();
    std::vector<Total> out;
    for (auto &t : totals_)
      if (t.launches) out.push_back(t);
    for (auto &t : totals_) {
      t.launches = 0;
      t.ms = 0.0;
    }
    return out;
  }

 private:
  struct Rec {
    int name;
    cudaEvent_t a, b;
  };
  int name_index(const char *name) {
    for (size_t i = 0; i < totals_.size(); ++i)
      if (totals_[i].name == name) return (int)i;
    totals_.push_back(Total{name, 0, 0.0});
    return (int)totals_.size() - 1;
  }
  cudaEvent_t take() {
    if (!pool_.empty()) {
      cudaEvent_t e = pool_.back();
      pool_.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }
  void give(cudaEvent_t e) {
    if (e) pool_.push_back(e);
  }

  unsigned long long launches_ = 0, untimed_ = 0;
  bool timing_ = false, open_ = false;
  std::vector<Rec> pending_;
  std::vector<cudaEvent_t> pool_;
  std::vector<Total> totals_;
};

// Bracket one launch statement with a (nullable) tracer.
#define DRC_TRACED(tr, name, st, launch_stmt) \
  do {                                        \
    if (tr) (tr)->begin((name), (st));        \
    launch_stmt;                              \
    if (tr) (tr)->end((st));                  \
  } while (0)

}  // namespace drc
