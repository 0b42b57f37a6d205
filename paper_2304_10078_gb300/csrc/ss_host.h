// Host-only declarations shared by the C-ABI translation unit and the
// per-key-type instantiation units.
#pragma once
#include <cuda_runtime.h>

#include "ss_plan.h"

namespace ss {

// Per-kernel CUDA-event timing of one call (SS_FLAG_PHASE_TIMING).
struct PhaseTimer {
  static constexpr int kMax = 64;
  cudaEvent_t ev[kMax + 1];
  const char* name[kMax];
  int count = 0;
  bool on = false;
  cudaStream_t st = nullptr;
  void start(cudaStream_t s) {
    st = s;
    count = 0;
    if (on) cudaEventRecord(ev[0], st);
  }
  void mark(const char* n) {
    if (!on || count >= kMax) return;
    name[count] = n;
    cudaEventRecord(ev[count + 1], st);
    ++count;
  }
};

struct LaunchCfg {
  int num_sms;
  PhaseTimer* timer;
  int* launches;  // incremented once per kernel enqueued
};

// One entry per key type; op is an Op, vt the value type code (0 u32, 1 u64).
cudaError_t run_u32(int op, int vt, const Plan& P, const Work& w, cudaStream_t st, const LaunchCfg& c);
cudaError_t run_u64(int op, int vt, const Plan& P, const Work& w, cudaStream_t st, const LaunchCfg& c);
cudaError_t run_u128(int op, int vt, const Plan& P, const Work& w, cudaStream_t st, const LaunchCfg& c);

}  // namespace ss
