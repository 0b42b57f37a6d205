// Host-side launcher of the semisort pipeline (templated; instantiated once per
// key/value/operation combination in the ss_inst_*.cu translation units).
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <utility>
#include <vector>

#include "ss_host.h"
#include "ss_kernels.cuh"

namespace ss {

// Raise a kernel's dynamic shared-memory limit once per (kernel, device); the
// attribute persists, so later calls -- including ones being captured into a
// CUDA graph -- make no runtime call for it.
template <class F>
static cudaError_t set_smem(F* f, size_t bytes) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const void* key = reinterpret_cast<const void*>(f);
  std::lock_guard<std::mutex> g(mu);
  for (const auto& d : done)
    if (d.first == key && d.second == dev) return cudaSuccess;
  e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done.emplace_back(key, dev);
  return e;
}

// Buffer roles.  Level 0 reads the caller's input (structure of arrays) and
// writes light records to the temporary T (array of structures); level
// l >= 1 reads T or T2 and writes the other one, so records move once per
// level.  With SS_FLAG_SWAP_OUTPUT (semisort_= and semisort_< only) T2 is not
// used: odd levels read T and write the caller's output arrays (structure of
// arrays), even levels >= 2 read the output and write T -- the swap of A and
// T of Sec. 3.4.  Heavy records go straight to the output whenever the output
// is not being read at that level; otherwise (in-place level 0, even levels
// >= 2 of the swap) they stay in T and a copy item moves them later.
// collect-reduce / histogram never move heavy records.
template <int OP>
static LevelBufs level_bufs(const Work& w, int level) {
  constexpr bool kSemi = OP == kOpEqual || OP == kOpLess;
  LevelBufs b;
  b.level = level;
  uint32_t src_id, dst_id;
  if (kSemi && w.swap) {
    src_id = level == 0 ? (uint32_t)kBufIn : (level % 2 == 1 ? (uint32_t)kBufT : (uint32_t)kBufOut);
    dst_id = level % 2 == 0 ? (uint32_t)kBufT : (uint32_t)kBufOut;
  } else {
    src_id = level == 0 ? (uint32_t)kBufIn : (level % 2 == 1 ? (uint32_t)kBufT : (uint32_t)kBufT2);
    dst_id = level % 2 == 0 ? (uint32_t)kBufT : (uint32_t)kBufT2;
  }
  auto ptr = [&](uint32_t id) -> void* {
    return id == kBufIn ? const_cast<void*>(w.in_k) : id == kBufT ? w.t_k : id == kBufOut ? w.out_k : w.t2_k;
  };
  const bool soa_src = src_id == kBufIn || src_id == kBufOut;
  b.src_k = ptr(src_id);
  b.src_v = src_id == kBufIn ? w.in_v : src_id == kBufOut ? w.out_v : nullptr;
  b.src_aos = soa_src ? 0u : 1u;
  b.dst = ptr(dst_id);
  b.dst_v = dst_id == kBufOut ? w.out_v : nullptr;
  b.dst_aos = dst_id == kBufOut ? 0u : 1u;
  b.dst_id = dst_id;
  const bool out_is_read = src_id == kBufOut || (src_id == kBufIn && w.in_k == w.out_k);
  if (kSemi && !out_is_read) {
    b.hdst_k = w.out_k;
    b.hdst_v = w.out_v;
    b.hdst_aos = 0;
    b.hdst_id = kBufOut;
  } else {
    // heavy records into the level's AoS destination: T for semisort (the
    // output is being read), the level's temporary for collect-reduce
    const uint32_t hid = kSemi ? (uint32_t)kBufT : dst_id;
    b.hdst_k = ptr(hid);
    b.hdst_v = nullptr;
    b.hdst_aos = 1;
    b.hdst_id = hid;
  }
  return b;
}

template <class K, class V, int OP>
cudaError_t launch_pipeline(const Plan& P, const Work& w, cudaStream_t st, const LaunchCfg& cfg) {
  PhaseTimer* tm = cfg.timer;
  const int nsm = cfg.num_sms;
  constexpr bool kWide = TopWide<K, OP>::value;  // semisort_< top level in the wide bucket space
  constexpr size_t kSmemMax = 232448;              // opt-in shared memory per block (sm_103a)
  static_assert(sizeof(DistSmem<K, V, false, OP>) <= kSmemMax && sizeof(DistSmem<K, V, kWide, OP>) <= kSmemMax, "smem");
  static_assert(sizeof(CountSmem<K, OP, kWide>) <= kSmemMax && sizeof(RefSmem<K, V>) <= kSmemMax, "smem");
  static_assert(sizeof(LessSmem<K, V>) <= kSmemMax && sizeof(RedSmem<K>) <= kSmemMax, "smem");
  const size_t dist_smem = sizeof(DistSmem<K, V, false, OP>);
  const size_t dist_smem_top = sizeof(DistSmem<K, V, kWide, OP>);
  const size_t count_smem = sizeof(CountSmem<K, OP, false>);
  const size_t count_smem_top = sizeof(CountSmem<K, OP, kWide>);
  size_t ref_smem = 0;
  cudaError_t e;
  if ((e = set_smem(k_distribute<K, V, OP, false>, dist_smem)) != cudaSuccess) return e;
  if ((e = set_smem(k_distribute<K, V, OP, kWide>, dist_smem_top)) != cudaSuccess) return e;
  if ((e = set_smem(k_count<K, V, OP, false, 4>, count_smem)) != cudaSuccess) return e;
  if ((e = set_smem(k_count<K, V, OP, false, 16>, count_smem)) != cudaSuccess) return e;
  if ((e = set_smem(k_count<K, V, OP, kWide, 16>, count_smem_top)) != cudaSuccess) return e;
  const size_t bigs_smem = (size_t)BigRun<K>::len * sizeof(K);
  const size_t split_smem = less_split_smem<K>();
  if constexpr (kWide) {
    if ((e = set_smem(k_learn_train, sizeof(TrainSmem))) != cudaSuccess) return e;
    if ((e = set_smem(k_bigsample_sort<K>, bigs_smem)) != cudaSuccess) return e;
    if ((e = set_smem(k_less_split<K>, split_smem)) != cudaSuccess) return e;
  }
  if constexpr (OP == kOpEqual) {
    ref_smem = sizeof(RefSmem<K, V>);
    if ((e = set_smem(k_finish_equal<K, V>, ref_smem)) != cudaSuccess) return e;
    if ((e = set_smem(k_finish_less<K, V>, sizeof(LessSmem<K, V>))) != cudaSuccess) return e;
  } else if constexpr (OP == kOpLess) {
    ref_smem = sizeof(LessSmem<K, V>);
    if ((e = set_smem(k_finish_less<K, V>, ref_smem)) != cudaSuccess) return e;
  } else {
    ref_smem = sizeof(RedSmem<K>);
    if ((e = set_smem(k_finish_reduce<K, V, OP>, ref_smem)) != cudaSuccess) return e;
  }
  const uint32_t s_cap_max = P.s1 > P.s2 ? P.s1 : P.s2;
  if ((e = set_smem(k_sample<K, V, OP>, (size_t)s_cap_max * sizeof(K))) != cudaSuccess) return e;

  int& nl = *cfg.launches;
  k_init<<<1, 1024, 0, st>>>(w);
  ++nl;
  if (tm) tm->mark("init");
  if (P.n > P.alpha) {
    for (int level = 0; level < kMaxLevels; ++level) {
      const LevelBufs lb = level_bufs<OP>(w, level);
      const uint32_t segs = P.seg_cap[level];
      const uint32_t tiles = P.tile_cap[level];
      auto cap = [](uint32_t want, uint32_t lim) { return want < lim ? (want ? want : 1) : lim; };
      const bool top_wide = kWide && level == 0 && w.num_inst <= 1;
      k_plan<OP><<<1, 1024, 0, st>>>(w, level);
      if (tm) tm->mark(level == 0 ? "plan.L0" : "plan.L1+");
      if (top_wide) {
        if constexpr (kWide) {
        k_bigsample_sort<K><<<BigRun<K>::runs, 1024, bigs_smem, st>>>(w);
        k_bigsample_merge<K><<<kBigSample / 256, 256, 0, st>>>(w);
        nl += 2;
        LearnState* ls = nullptr;
        if (w.splitter_mode == 1) {
          // learned splitters: fit the CDF model to the sorted sample, invert it
          ls = reinterpret_cast<LearnState*>(w.learn);
          k_learn_prep<K><<<1, 1024, 0, st>>>(reinterpret_cast<const K*>(w.bigs), ls, w.seed, w.segs[0],
                                              reinterpret_cast<K*>(w.bigs_tmp), 0u);
          // every Adam step in one launch of one thread-block cluster
          k_learn_train<<<kTrainCTAs, kTrainThreads, sizeof(TrainSmem), st>>>(ls, kLearnSteps, kLearnLr, 1);
          k_learn_invert<K><<<((1u << kLessTopLog2) + 255) / 256, 256, 0, st>>>(ls, w.segs[0], 0);
          nl += 3;
          if (tm) tm->mark("learn.L0");
        }
        k_less_split<K><<<1, 1024, split_smem, st>>>(w, ls);
        ++nl;
        }
      } else {
        if constexpr (kWide) {
          if (level == 0 && w.num_inst > 1 && w.splitter_mode == 1) {
            // batched learned mode: one model from a sample of the whole batch,
            // inverted at 2^8 ranges; k_sample judges it per instance
            LearnState* ls = reinterpret_cast<LearnState*>(w.learn);
            k_bigsample_sort<K><<<BigRun<K>::runs, 1024, bigs_smem, st>>>(w);
            k_bigsample_merge<K><<<kBigSample / 256, 256, 0, st>>>(w);
            k_learn_prep<K><<<1, 1024, 0, st>>>(reinterpret_cast<const K*>(w.bigs), ls, w.seed, nullptr,
                                                reinterpret_cast<K*>(w.bigs_tmp), (uint32_t)kBatchLearnLog2);
            k_learn_train<<<kTrainCTAs, kTrainThreads, sizeof(TrainSmem), st>>>(ls, kLearnSteps, kLearnLr, 1);
            k_learn_invert<K><<<((1u << kBatchLearnLog2) + 255) / 256, 256, 0, st>>>(ls, nullptr, kBatchLearnLog2);
            nl += 5;
            if (tm) tm->mark("learn.L0");
          }
        }
        const uint32_t s_cap = level == 0 ? P.s1 : P.s2;
        k_sample<K, V, OP><<<cap(segs, nsm * 2), 1024, (size_t)s_cap * sizeof(K), st>>>(w, lb, s_cap);
        ++nl;
      }
      if (tm) tm->mark(level == 0 ? "sample.L0" : "sample.L1+");
      if (top_wide)
        k_count<K, V, OP, kWide, 16><<<cap(tiles, nsm * 4), kCountThreads, count_smem_top, st>>>(w, lb);
      else if (lb.src_aos)
        k_count<K, V, OP, false, 4><<<cap(tiles, nsm * 4), kCountThreads, count_smem, st>>>(w, lb);
      else
        k_count<K, V, OP, false, 16><<<cap(tiles, nsm * 4), kCountThreads, count_smem, st>>>(w, lb);
      if (tm) tm->mark(level == 0 ? "count.L0" : "count.L1+");
      k_scan<OP><<<cap(segs, nsm * 2), 1024, 0, st>>>(w, lb);
      if (tm) tm->mark(level == 0 ? "scan.L0" : "scan.L1+");
      if (top_wide)
        k_distribute<K, V, OP, kWide><<<cap(tiles, nsm * 2), kDT, dist_smem_top, st>>>(w, lb);
      else
        k_distribute<K, V, OP, false><<<cap(tiles, nsm * 2), kDT, dist_smem, st>>>(w, lb);
      if (tm) tm->mark(level == 0 ? "distribute.L0" : "distribute.L1+");
      k_scan_items<<<1, 1024, 0, st>>>(w, level);
      k_emit<OP><<<cap(segs, nsm * 2), 1024, 0, st>>>(w, lb);
      nl += 6;
      if (tm) tm->mark(level == 0 ? "emit.L0" : "emit.L1+");
    }
  }
  if constexpr (OP == kOpEqual) {
    if (w.less_base)  // hash buckets with a sorting base case: the paper's semisort_<
      k_finish_less<K, V><<<nsm * 2, kRT, sizeof(LessSmem<K, V>), st>>>(w);
    else
      k_finish_equal<K, V><<<nsm * 2, kRT, ref_smem, st>>>(w);
    ++nl;
    if (tm) tm->mark("refine");
  } else if constexpr (OP == kOpLess) {
    k_finish_less<K, V><<<nsm * 2, kRT, ref_smem, st>>>(w);
    ++nl;
    if (tm) tm->mark("refine");
  } else {
    k_finish_reduce<K, V, OP><<<nsm * 2, kRT, ref_smem, st>>>(w);
    if (tm) tm->mark("refine");
    const uint32_t nch = (P.item_cap + kScanChunk - 1) / kScanChunk;
    k_iscan_a<<<nch, 1024, 0, st>>>(w);
    k_iscan_b<<<1, 1024, 0, st>>>(w);
    k_iscan_c<<<nch, 1024, 0, st>>>(w);
    if (w.offsets) {  // batched: make each instance's outputs contiguous
      const uint32_t g = (kItemClasses * w.num_inst + 255) / 256;
      k_inst_reset<<<g < 1024 ? g : 1024, 256, 0, st>>>(w);
      k_inst_accum<<<nsm * 4, 256, 0, st>>>(w);
      k_inst_scan<<<1, 1024, 0, st>>>(w);
      nl += 3;
    }
    if (tm) tm->mark("scan_out");
    k_pack<K, V, OP><<<nsm * 8, 256, 0, st>>>(w);
    if (tm) tm->mark("pack");
    nl += 5;
  }
  return cudaGetLastError();
}

}  // namespace ss
