// Pipeline instantiations for 32-bit keys.
#include "ss_launch.cuh"

namespace ss {

cudaError_t run_u32(int op, int vt, const Plan& P, const Work& w, cudaStream_t st, const LaunchCfg& c) {
  switch (op) {
    case kOpEqual:
      return vt == 0   ? launch_pipeline<uint32_t, uint32_t, kOpEqual>(P, w, st, c)
             : vt == 1 ? launch_pipeline<uint32_t, uint64_t, kOpEqual>(P, w, st, c)
                       : launch_pipeline<uint32_t, void, kOpEqual>(P, w, st, c);
    case kOpLess:
      return vt == 0   ? launch_pipeline<uint32_t, uint32_t, kOpLess>(P, w, st, c)
             : vt == 1 ? launch_pipeline<uint32_t, uint64_t, kOpLess>(P, w, st, c)
                       : launch_pipeline<uint32_t, void, kOpLess>(P, w, st, c);
    case kOpReduce:
      return launch_pipeline<uint32_t, uint64_t, kOpReduce>(P, w, st, c);
    case kOpHist:
      return launch_pipeline<uint32_t, void, kOpHist>(P, w, st, c);
    default:
      return cudaErrorNotSupported;
  }
}

}  // namespace ss
