// Host-side launcher of the semisort pipeline (templated; instantiated once per
// key/value/operation combination in the ss_inst_*.cu translation units).
#pragma once
#include <cuda_runtime.h>

#include "ss_host.h"
#include "ss_kernels.cuh"

namespace ss {

template <class F>
static cudaError_t set_smem(F* f, size_t bytes) {
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Buffer roles.  semisort: level 0 reads the input and writes T; level 1
// reads T and writes the output; and so on (the swap of Sec. 3.4, so records
// move twice in the common two-level case).  Heavy records go straight to the
// output array whenever that array is not being read at the same level.
// collect-reduce / histogram alternate between T and T2 and never move heavy
// records.
template <int OP>
static LevelBufs level_bufs(const Work& w, int level) {
  LevelBufs b;
  b.level = level;
  b.salt = level_salt(w.seed, level);
  auto k_of = [&](uint32_t id) -> void* {
    return id == kBufIn ? const_cast<void*>(w.in_k) : id == kBufT ? w.t_k : id == kBufOut ? w.out_k : w.t2_k;
  };
  auto v_of = [&](uint32_t id) -> void* {
    return id == kBufIn ? const_cast<void*>(w.in_v) : id == kBufT ? w.t_v : id == kBufOut ? w.out_v : w.t2_v;
  };
  uint32_t src_id, dst_id, hdst_id;
  if (OP == kOpEqual || OP == kOpLess) {
    dst_id = (level % 2 == 0) ? kBufT : kBufOut;
    src_id = level == 0 ? kBufIn : ((level - 1) % 2 == 0 ? kBufT : kBufOut);
    const bool src_is_out = src_id == kBufOut || (src_id == kBufIn && w.in_k == w.out_k);
    hdst_id = src_is_out ? dst_id : kBufOut;
  } else {
    dst_id = (level % 2 == 0) ? kBufT : kBufT2;
    src_id = level == 0 ? kBufIn : ((level - 1) % 2 == 0 ? kBufT : kBufT2);
    hdst_id = dst_id;
  }
  b.src_k = k_of(src_id);
  b.src_v = v_of(src_id);
  b.dst_k = k_of(dst_id);
  b.dst_v = v_of(dst_id);
  b.hdst_k = k_of(hdst_id);
  b.hdst_v = v_of(hdst_id);
  b.dst_id = dst_id;
  b.hdst_id = hdst_id;
  return b;
}

template <class K, class V, int OP>
cudaError_t launch_pipeline(const Plan& P, const Work& w, cudaStream_t st, const LaunchCfg& cfg) {
  PhaseTimer* tm = cfg.timer;
  const int nsm = cfg.num_sms;
  const size_t dist_smem = sizeof(DistSmem<K>);
  const size_t ref_smem = sizeof(RefSmem<K>);
  cudaError_t e;
  if ((e = set_smem(k_distribute<K, V, OP>, dist_smem)) != cudaSuccess) return e;
  if ((e = set_smem(k_finish_equal<K, V>, ref_smem)) != cudaSuccess) return e;
  const uint32_t s_cap_max = P.s1 > P.s2 ? P.s1 : P.s2;
  if ((e = set_smem(k_sample<K>, (size_t)s_cap_max * sizeof(K))) != cudaSuccess) return e;

  int& nl = *cfg.launches;
  k_init<<<1, 32, 0, st>>>(w);
  ++nl;
  if (tm) tm->mark("init");
  if (P.n > P.alpha) {
    for (int level = 0; level < kMaxLevels; ++level) {
      const LevelBufs lb = level_bufs<OP>(w, level);
      const uint32_t segs = P.seg_cap[level];
      const uint32_t tiles = P.tile_cap[level];
      auto cap = [](uint32_t want, uint32_t lim) { return want < lim ? (want ? want : 1) : lim; };
      k_plan<<<1, 1024, 0, st>>>(w, level);
      if (tm) tm->mark(level == 0 ? "plan.L0" : "plan.L1+");
      const uint32_t s_cap = level == 0 ? P.s1 : P.s2;
      k_sample<K><<<cap(segs, nsm * 2), 1024, (size_t)s_cap * sizeof(K), st>>>(w, lb, s_cap);
      if (tm) tm->mark(level == 0 ? "sample.L0" : "sample.L1+");
      k_count<K, OP><<<cap(tiles, nsm * 4), 512, 0, st>>>(w, lb);
      if (tm) tm->mark(level == 0 ? "count.L0" : "count.L1+");
      k_scan<OP><<<cap(segs, nsm * 2), 1024, 0, st>>>(w, lb);
      if (tm) tm->mark(level == 0 ? "scan.L0" : "scan.L1+");
      k_distribute<K, V, OP><<<cap(tiles, nsm * 2), kDistThreads, dist_smem, st>>>(w, lb);
      if (tm) tm->mark(level == 0 ? "distribute.L0" : "distribute.L1+");
      k_scan_items<<<1, 1024, 0, st>>>(w, level);
      k_emit<OP><<<cap(segs, nsm * 2), 1024, 0, st>>>(w, lb);
      nl += 7;
      if (tm) tm->mark(level == 0 ? "emit.L0" : "emit.L1+");
    }
  }
  if (OP == kOpEqual) {
    k_finish_equal<K, V><<<nsm * 2, kRefThreads, ref_smem, st>>>(w);
    ++nl;
    if (tm) tm->mark("refine");
  }
  return cudaGetLastError();
}

}  // namespace ss
