// Device-side building blocks shared by the semisort kernels (sm_103a).
//
// Contents: the fixed key hash, key-type traits, block-wide scans, the stable
// block-wide digit rank (the in-tile ordering step of Blocked Distributing,
// Sec. 3.2, and of the base cases, Sec. 3.3), and the descriptors of the
// device-resident work lists that drive the recursion (Algorithm 1).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ss_plan.h"

namespace ss {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint32_t kFull = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// Hash: the output mixer of SplitMix64 (Steele, Lea, Flood 2014).  It is a
// bijection of 64-bit words, so for 32- and 64-bit keys equal hashes imply
// equal keys.  Each recursion level uses a different salt, which gives the
// family of hash functions Sec. 2.1 asks the user to supply.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

struct alignas(16) k128 {
  uint64_t lo, hi;
};

template <class K>
struct KeyT;

template <>
struct KeyT<uint32_t> {
  static constexpr int kCode = 0;
  __device__ __forceinline__ static uint64_t hash(uint32_t k, uint64_t salt, bool ident) {
    return ident ? (uint64_t)k << 32 : mix64((uint64_t)k ^ salt);
  }
  __device__ __forceinline__ static bool eq(uint32_t a, uint32_t b) { return a == b; }
  __device__ __forceinline__ static bool lt(uint32_t a, uint32_t b) { return a < b; }
};

template <>
struct KeyT<uint64_t> {
  static constexpr int kCode = 1;
  __device__ __forceinline__ static uint64_t hash(uint64_t k, uint64_t salt, bool ident) {
    return ident ? k : mix64(k ^ salt);
  }
  __device__ __forceinline__ static bool eq(uint64_t a, uint64_t b) { return a == b; }
  __device__ __forceinline__ static bool lt(uint64_t a, uint64_t b) { return a < b; }
};

template <>
struct KeyT<k128> {
  static constexpr int kCode = 2;
  __device__ __forceinline__ static uint64_t hash(k128 k, uint64_t salt, bool ident) {
    return ident ? k.hi : mix64(k.lo ^ mix64(k.hi ^ salt));
  }
  __device__ __forceinline__ static bool eq(k128 a, k128 b) { return a.lo == b.lo && a.hi == b.hi; }
  __device__ __forceinline__ static bool lt(k128 a, k128 b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
  }
};

// Light-bucket id: the top `bits` bits of the level hash (bits >= 1).
__device__ __forceinline__ uint32_t light_bucket(uint64_t h, uint32_t bits) {
  return (uint32_t)(h >> (64 - bits));
}

// ---------------------------------------------------------------------------
// Warp / block scans.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

__device__ __forceinline__ uint64_t warp_inclusive_scan64(uint64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t t = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan of one value per thread over the whole block; `tmp` holds
// at least 33 words of shared memory.  Returns the exclusive prefix and
// writes the block total to *total.  Contains __syncthreads.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* tmp, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  uint32_t inc = warp_inclusive_scan(v);
  if (lane == 31) tmp[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t x = lane < nw ? tmp[lane] : 0;
    uint32_t xi = warp_inclusive_scan(x);
    if (lane < nw) tmp[lane] = xi - x;
    if (lane == 31) tmp[32] = xi;
  }
  __syncthreads();
  uint32_t r = tmp[w] + inc - v;
  *total = tmp[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ uint64_t block_exclusive_scan64(uint64_t v, uint64_t* tmp, uint64_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  uint64_t inc = warp_inclusive_scan64(v);
  if (lane == 31) tmp[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint64_t x = lane < nw ? tmp[lane] : 0;
    uint64_t xi = warp_inclusive_scan64(x);
    if (lane < nw) tmp[lane] = xi - x;
    if (lane == 31) tmp[32] = xi;
  }
  __syncthreads();
  uint64_t r = tmp[w] + inc - v;
  *total = tmp[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ uint32_t block_reduce_sum(uint32_t v, uint32_t* tmp) {
  uint32_t t;
  block_exclusive_scan(v, tmp, &t);
  return t;
}

// ---------------------------------------------------------------------------
// Stable block-wide rank by an 8-bit digit.
//
// Items are held R per thread in warp-striped order: item r of lane `lane` in
// warp w has order index w*32*R + r*32 + lane.  On return rank[r] is the
// item's position in the stable order by digit (ties keep order index).
// Within a warp, equal digits are found with __match_any_sync and ordered by
// lane; across rounds the per-warp counters advance in order; across warps a
// prefix over warps is added.  Atomics never decide a position, so the result
// is deterministic.  hist: NW*256 uint16 in shared memory; dsum: 256+33 words.
// ---------------------------------------------------------------------------
template <int NW, int R>
__device__ __forceinline__ void block_rank8(const uint32_t (&digit)[R], uint32_t (&rank)[R],
                                            uint16_t* hist, uint32_t* dsum) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint16_t* my = hist + w * 256;
  for (int d = lane; d < 256; d += 32) my[d] = 0;
  __syncwarp();
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t d = digit[r];
    const uint32_t peers = __match_any_sync(kFull, d);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader) {
      base = my[d];
      my[d] = (uint16_t)(base + __popc(peers));
    }
    base = __shfl_sync(kFull, base, leader);
    rank[r] = base + __popc(peers & lt);
    __syncwarp();
  }
  __syncthreads();
  // Per digit: exclusive prefix over warps (in place) and the digit total.
  for (int d = threadIdx.x; d < 256; d += blockDim.x) {
    uint32_t s = 0;
#pragma unroll
    for (int ww = 0; ww < NW; ++ww) {
      uint32_t c = hist[ww * 256 + d];
      hist[ww * 256 + d] = (uint16_t)s;
      s += c;
    }
    dsum[d] = s;
  }
  __syncthreads();
  // Exclusive scan of the 256 digit totals (first 256 threads).
  {
    uint32_t v = threadIdx.x < 256 ? dsum[threadIdx.x] : 0;
    uint32_t tot;
    uint32_t ex = block_exclusive_scan(v, dsum + 256, &tot);
    if (threadIdx.x < 256) dsum[threadIdx.x] = ex;
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < R; ++r) rank[r] += dsum[digit[r]] + my[digit[r]];
  __syncthreads();
}

}  // namespace ss
