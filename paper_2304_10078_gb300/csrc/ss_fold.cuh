// Ordered segmented fold: collect-reduce with any monoid (op, identity)
// over records that a stable semisort_= has already grouped (Sec. 3.5: with
// a stable grouping the records of a key are in input order, so the monoid
// need not be commutative).  Each run of equal adjacent keys becomes one
// output (key, v_1 op v_2 op ... op v_m) with the values in run order.
//
// Three passes over tiles of kFoldTile records:
//   k_fold_count   run starts per tile;
//   k_fold_scan    exclusive scan of the tile counts (output index of each
//                  tile's first run) and the number of runs;
//   k_fold_tiles   per tile, a block-wide segmented scan gives every run's
//                  fold inside the tile; runs that end in their own tile are
//                  written out, and the tile keeps a "head" (fold of its
//                  leading records that continue a run from an earlier tile)
//                  and a "tail" (fold of its last run, when that run goes on);
//   k_fold_join    a run that crosses tiles is its tail op the heads of the
//                  following tiles, taken in tile order.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ss_common.cuh"

namespace ss {

constexpr int kFoldThreads = 256;
constexpr int kFoldPer = 16;
constexpr int kFoldTile = kFoldThreads * kFoldPer;

// Tile flags.
enum : uint32_t { kFoldHasStart = 1u, kFoldTailOpen = 2u };

template <class K>
__device__ __forceinline__ bool fold_run_start(const K* k, uint64_t i) {
  return i == 0 || !KeyT<K>::eq(k[i], k[i - 1]);
}

template <class K>
__global__ void __launch_bounds__(kFoldThreads) k_fold_count(const K* k, uint64_t n, uint32_t* tile_starts) {
  __shared__ uint32_t tmp[33];
  const uint64_t t0 = (uint64_t)blockIdx.x * kFoldTile;
  uint32_t c = 0;
  for (uint32_t j = threadIdx.x; j < (uint32_t)kFoldTile; j += kFoldThreads) {
    const uint64_t i = t0 + j;
    if (i < n && fold_run_start<K>(k, i)) ++c;
  }
  const uint32_t tot = block_reduce_sum(c, tmp);
  if (threadIdx.x == 0) tile_starts[blockIdx.x] = tot;
}

// One CTA: tile_base[t] = runs starting before tile t; *num_runs = all runs.
static __global__ void __launch_bounds__(1024) k_fold_scan(const uint32_t* tile_starts, uint32_t ntiles,
                                                           uint64_t* tile_base, uint64_t* num_runs) {
  __shared__ uint64_t tmp[33];
  uint64_t carry = 0;
  for (uint32_t b = 0; b < ntiles; b += blockDim.x) {
    const uint32_t t = b + threadIdx.x;
    const uint64_t v = t < ntiles ? tile_starts[t] : 0;
    uint64_t tot;
    const uint64_t ex = block_exclusive_scan64(v, tmp, &tot);
    if (t < ntiles) tile_base[t] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *num_runs = carry;
}

template <class V>
struct FoldSmem {
  V agg[kFoldThreads];
  uint32_t flag[kFoldThreads];
  V agg2[kFoldThreads];
  uint32_t flag2[kFoldThreads];
  uint32_t scan_tmp[33];
};

template <class K, class V, class Op>
__global__ void __launch_bounds__(kFoldThreads) k_fold_tiles(const K* k, const V* v, uint64_t n,
                                                             const uint64_t* tile_base, K* ukeys, V* sums,
                                                             uint64_t capacity, V* head, V* tail,
                                                             uint32_t* tflags, Op op, V identity) {
  __shared__ FoldSmem<V> sm;
  const int tid = threadIdx.x;
  const uint64_t t0 = (uint64_t)blockIdx.x * kFoldTile;
  const uint64_t i0 = t0 + (uint64_t)tid * kFoldPer;
  // this thread's summary: (a run starts here, fold since its last start)
  uint32_t nst = 0, f = 0;
  V a = identity;
  for (int r = 0; r < kFoldPer; ++r) {
    const uint64_t i = i0 + r;
    if (i >= n) break;
    if (fold_run_start<K>(k, i)) {
      f = 1;
      ++nst;
      a = v[i];
    } else {
      a = op(a, v[i]);
    }
  }
  // exclusive segmented scan over threads: (f1, a1) then (f2, a2) combine to
  // (f1 | f2, f2 ? a2 : a1 op a2), an associative operator
  sm.agg[tid] = a;
  sm.flag[tid] = f;
  __syncthreads();
  V* src_a = sm.agg;
  uint32_t* src_f = sm.flag;
  V* dst_a = sm.agg2;
  uint32_t* dst_f = sm.flag2;
  for (int d = 1; d < kFoldThreads; d <<= 1) {
    if (tid >= d) {
      const uint32_t f2 = src_f[tid];
      dst_a[tid] = f2 ? src_a[tid] : op(src_a[tid - d], src_a[tid]);
      dst_f[tid] = src_f[tid - d] | f2;
    } else {
      dst_a[tid] = src_a[tid];
      dst_f[tid] = src_f[tid];
    }
    __syncthreads();
    V* ta = src_a;
    src_a = dst_a;
    dst_a = ta;
    uint32_t* tf = src_f;
    src_f = dst_f;
    dst_f = tf;
  }
  // inclusive result in src; the exclusive prefix of thread tid is src[tid - 1]
  const bool pre_f = tid > 0 ? src_f[tid - 1] != 0 : false;
  V acc = tid > 0 ? src_a[tid - 1] : identity;
  bool cont = tid > 0 ? true : false;  // acc holds a fold of the current run's earlier records
  uint32_t tot;
  uint32_t idx = block_exclusive_scan(nst, sm.scan_tmp, &tot);
  const uint64_t base = tile_base[blockIdx.x];
  const uint64_t tile_end = t0 + kFoldTile < n ? t0 + kFoldTile : n;
  bool started = pre_f;  // the current run started inside this tile
  for (int r = 0; r < kFoldPer; ++r) {
    const uint64_t i = i0 + r;
    if (i >= n) break;
    if (fold_run_start<K>(k, i)) {
      acc = v[i];
      started = true;
      const uint64_t o = base + idx;
      if (o < capacity) ukeys[o] = k[i];
      ++idx;
    } else {
      acc = cont ? op(acc, v[i]) : v[i];
    }
    cont = true;
    const bool last_of_run = i + 1 == n || fold_run_start<K>(k, i + 1);
    if (i + 1 == tile_end && !last_of_run) {
      // the tile ends inside a run
      if (started) {
        tail[blockIdx.x] = acc;
      } else {
        head[blockIdx.x] = acc;  // the whole tile continues an earlier run
      }
    } else if (last_of_run) {
      if (started) {
        const uint64_t o = base + idx - 1;
        if (o < capacity) sums[o] = acc;
      } else {
        head[blockIdx.x] = acc;  // the leading records end an earlier tile's run
      }
    }
  }
  if (tid == 0) {
    const bool open = tile_end < n && !fold_run_start<K>(k, tile_end);
    tflags[blockIdx.x] = (tot ? kFoldHasStart : 0u) | (open && tot ? kFoldTailOpen : 0u);
  }
}

// One thread per tile whose last run goes on: that run's fold is the tile's
// tail op the heads of the next tiles, up to the first tile with a run start.
template <class V, class Op>
__global__ void k_fold_join(uint32_t ntiles, const uint64_t* tile_base, const uint32_t* tile_starts,
                            const uint32_t* tflags, const V* head, const V* tail, V* sums, uint64_t capacity,
                            Op op) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles || !(tflags[t] & kFoldTailOpen)) return;
  V acc = tail[t];
  for (uint32_t u = t + 1; u < ntiles; ++u) {
    acc = op(acc, head[u]);
    if (tflags[u] & kFoldHasStart) break;
  }
  const uint64_t o = tile_base[t] + tile_starts[t] - 1;
  if (o < capacity) sums[o] = acc;
}

}  // namespace ss
