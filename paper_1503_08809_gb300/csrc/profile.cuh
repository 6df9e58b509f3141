// profile.cuh -- opt-in CUDA-event timing of the library's own launches.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

namespace modal {

struct Profiler {
  bool on = false;
  struct Rec {
    const char *name;
    cudaEvent_t a, b;
    int kernels;  // kernel launches inside the scope
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void begin(const char *name, cudaStream_t st, int kernels) {
    if (!on) return;
    Rec r{name, get(), get(), kernels};
    cudaEventRecord(r.a, st);
    recs.push_back(r);
  }
  void end(cudaStream_t st) {
    if (!on || recs.empty()) return;
    cudaEventRecord(recs.back().b, st);
  }
  // name -> (kernel launches, ms)
  std::map<std::string, std::pair<long long, double>> drain() {
    std::map<std::string, std::pair<long long, double>> out;
    for (auto &r : recs) {
      cudaEventSynchronize(r.b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, r.a, r.b);
      auto &e = out[r.name];
      e.first += r.kernels;
      e.second += ms;
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    recs.clear();
    return out;
  }
  ~Profiler() {
    for (auto &r : recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// RAII scope around `kernels` launches (timed together)
struct ProfScope {
  Profiler *p;
  cudaStream_t st;
  ProfScope(Profiler *p_, const char *name, cudaStream_t s, int kernels = 1) : p(p_), st(s) {
    if (p) p->begin(name, st, kernels);
  }
  ~ProfScope() {
    if (p) p->end(st);
  }
};

}  // namespace modal
