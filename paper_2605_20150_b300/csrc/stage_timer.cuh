// Per-stage CUDA-event timing on the stream that launches each stage (the
// tracing facility of the step; off unless enabled).
#pragma once
#include <utility>
#include <vector>

#include "common.cuh"

namespace tgs {

struct StageTimer {
  enum { PRE = 0, SORT, FWD, LOSS, BWD, PBWD, ADAM, BOUNDS, NSTAGE };
  bool on = false;
  double ms[NSTAGE] = {0};
  uint64_t count[NSTAGE] = {0};
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::vector<cudaEvent_t> free_ev;
  cudaEvent_t open_ev[NSTAGE] = {nullptr};

  cudaEvent_t get() {
    cudaEvent_t e;
    if (!free_ev.empty()) {
      e = free_ev.back();
      free_ev.pop_back();
    } else {
      TGS_CUDA(cudaEventCreate(&e));
    }
    return e;
  }
  void begin(int st, cudaStream_t s) {
    if (!on) return;
    open_ev[st] = get();
    TGS_CUDA(cudaEventRecord(open_ev[st], s));
  }
  void end(int st, cudaStream_t s) {
    if (!on || !open_ev[st]) return;
    cudaEvent_t e = get();
    TGS_CUDA(cudaEventRecord(e, s));
    pending.push_back({st, {open_ev[st], e}});
    open_ev[st] = nullptr;
  }
  void collect() {
    for (auto& p : pending) {
      TGS_CUDA(cudaEventSynchronize(p.second.second));
      float t = 0.f;
      TGS_CUDA(cudaEventElapsedTime(&t, p.second.first, p.second.second));
      ms[p.first] += t;
      count[p.first] += 1;
      free_ev.push_back(p.second.first);
      free_ev.push_back(p.second.second);
    }
    pending.clear();
  }
  void reset() {
    collect();
    for (int i = 0; i < NSTAGE; ++i) {
      ms[i] = 0;
      count[i] = 0;
    }
  }
  ~StageTimer() {
    for (auto& p : pending) {
      cudaEventDestroy(p.second.first);
      cudaEventDestroy(p.second.second);
    }
    for (auto e : free_ev) cudaEventDestroy(e);
  }
};

}  // namespace tgs
