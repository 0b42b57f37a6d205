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

namespace semisort {
// Traits of a user-defined key type for the C++ template entry points
// (include/semisort.hpp).  Specialize with
//   __device__ static uint64_t hash(const K&);           equal keys hash equally
//   __device__ static bool equal(const K&, const K&);    an equivalence
//   __device__ static bool less(const K&, const K&);     a strict weak order (semisort_<)
// Sec. 2.1 asks the user of a semisort for exactly these: a hash function
// family, an equality test and, for semisort_<, a comparison.
template <class K>
struct key_traits;
}  // namespace semisort

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

// Key traits used by the kernels.  The built-in types are specialized below;
// any other key type reads semisort::key_traits (its hash is mixed with the
// level salt, and equality always compares whole keys, so hash collisions
// never merge groups).  kIntegral: an unsigned integer of at most 8 bytes,
// which the semisort_< kernels may also treat as a number (lookup tables,
// interpolation buckets).
template <class K>
struct KeyT {
  static constexpr int kCode = -1;
  static constexpr bool kIntegral = false;
  __device__ __forceinline__ static uint64_t hash(const K& k, uint64_t salt, bool) {
    return mix64(semisort::key_traits<K>::hash(k) ^ salt);
  }
  __device__ __forceinline__ static bool eq(const K& a, const K& b) { return semisort::key_traits<K>::equal(a, b); }
  __device__ __forceinline__ static bool lt(const K& a, const K& b) { return semisort::key_traits<K>::less(a, b); }
};

template <>
struct KeyT<uint32_t> {
  static constexpr int kCode = 0;
  static constexpr bool kIntegral = true;
  __device__ __forceinline__ static uint64_t hash(uint32_t k, uint64_t salt, bool ident) {
    return ident ? (uint64_t)k << 32 : mix64((uint64_t)k ^ salt);
  }
  __device__ __forceinline__ static bool eq(uint32_t a, uint32_t b) { return a == b; }
  __device__ __forceinline__ static bool lt(uint32_t a, uint32_t b) { return a < b; }
};

template <>
struct KeyT<uint64_t> {
  static constexpr int kCode = 1;
  static constexpr bool kIntegral = true;
  __device__ __forceinline__ static uint64_t hash(uint64_t k, uint64_t salt, bool ident) {
    return ident ? k : mix64(k ^ salt);
  }
  __device__ __forceinline__ static bool eq(uint64_t a, uint64_t b) { return a == b; }
  __device__ __forceinline__ static bool lt(uint64_t a, uint64_t b) { return a < b; }
};

template <>
struct KeyT<k128> {
  static constexpr int kCode = 2;
  static constexpr bool kIntegral = false;
  __device__ __forceinline__ static uint64_t hash(k128 k, uint64_t salt, bool ident) {
    return ident ? k.hi : mix64(k.lo ^ mix64(k.hi ^ salt));
  }
  __device__ __forceinline__ static bool eq(k128 a, k128 b) { return a.lo == b.lo && a.hi == b.hi; }
  __device__ __forceinline__ static bool lt(k128 a, k128 b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
  }
};

// Heavy-key capacity of a segment with 2^lbits light buckets: min(n_L, 512).
__host__ __device__ __forceinline__ uint32_t hcap_of(uint32_t lbits) {
  const uint32_t nl = 1u << lbits;
  return nl < kMaxHeavy ? nl : kMaxHeavy;
}

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

// Maximum of v over the threads before this one (0 for thread 0), and
// minimum over the threads after it (0xFFFFFFFF for the last); `tmp` holds
// at least 32 words.  Both contain __syncthreads.
__device__ __forceinline__ uint32_t block_exclusive_max(uint32_t v, uint32_t* tmp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc = t > inc ? t : inc;
  }
  uint32_t ex = __shfl_up_sync(kFull, inc, 1);
  if (lane == 0) ex = 0;
  if (lane == 31) tmp[w] = inc;
  __syncthreads();
  for (int j = 0; j < w && j < nw; ++j) ex = tmp[j] > ex ? tmp[j] : ex;
  __syncthreads();
  return ex;
}
__device__ __forceinline__ uint32_t block_suffix_min(uint32_t v, uint32_t* tmp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_down_sync(kFull, inc, o);
    if (lane + o < 32) inc = t < inc ? t : inc;
  }
  uint32_t ex = __shfl_down_sync(kFull, inc, 1);
  if (lane == 31) ex = 0xFFFFFFFFu;
  if (lane == 0) tmp[w] = inc;
  __syncthreads();
  for (int j = w + 1; j < nw; ++j) ex = tmp[j] < ex ? tmp[j] : ex;
  __syncthreads();
  return ex;
}

__device__ __forceinline__ uint32_t block_reduce_sum(uint32_t v, uint32_t* tmp) {
  uint32_t t;
  block_exclusive_scan(v, tmp, &t);
  return t;
}

// ---------------------------------------------------------------------------
// Stable block-wide rank by a DBITS-bit digit without atomics or warp votes.
//
// T threads hold R items each in blocked order (thread t holds items
// t*R .. t*R+R-1, so item order = (thread, slot)).  Every thread counts its
// items in private 16-bit counters, two digits packed per 32-bit word and laid
// out [digit pair][thread]; one raking exclusive scan over that array in
// (digit pair, thread) order then gives, per (digit, thread), the number of
// items with a smaller digit plus the items of the same digit in earlier
// threads.  Adding the thread's own running count yields the stable rank.
// The two packed halves are scanned together; each half counts at most T*R
// items, so T*R must stay below 65536.  A padding word after every 32 keeps
// both the counting and the raking phases free of bank conflicts.
// ---------------------------------------------------------------------------
template <int T, int R, int DBITS>
struct BlockRank {
  static constexpr int D = 1 << DBITS;
  static constexpr int ROWS = D / 2;
  static constexpr int WORDS = ROWS * T;
  static constexpr int RAKE = ROWS;  // words raked per thread
  static constexpr int PWORDS = WORDS + (WORDS / 32) * 4;
  static_assert(T * R < 65536, "packed 16-bit counters");
  static_assert(RAKE % 4 == 0 && RAKE <= 32 && 32 % RAKE == 0, "rake range must stay inside a padded block");
  struct Smem {
    alignas(16) uint32_t c[PWORDS];
    uint32_t dofs[D];
    uint32_t scan_tmp[33];
  };
  // 4 padding words after every 32: keeps 16-byte alignment for the raking
  // loads and spreads both access patterns over all banks.
  __device__ __forceinline__ static int pidx(int f) { return f + ((f >> 5) << 2); }

  // Digit of item r: (val[r] >> shift) & (D - 1).
  __device__ static void rank(Smem& s, const uint32_t (&val)[R], int shift, uint32_t (&out)[R]) {
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < ROWS; ++i) s.c[pidx(i * T + t)] = 0;
    uint32_t pre[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t d = (val[r] >> shift) & (D - 1);
      const int idx = pidx((int)(d >> 1) * T + t);
      const uint32_t sh = (d & 1u) << 4;
      const uint32_t w = s.c[idx];
      pre[r] = (w >> sh) & 0xFFFFu;
      s.c[idx] = w + (1u << sh);
    }
    __syncthreads();
    uint4* rk4 = reinterpret_cast<uint4*>(&s.c[pidx(t * RAKE)]);
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < RAKE / 4; ++j) {
      const uint4 v = rk4[j];
      sum += v.x + v.y + v.z + v.w;
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(sum, s.scan_tmp, &total);
#pragma unroll
    for (int j = 0; j < RAKE / 4; ++j) {
      const uint4 v = rk4[j];
      uint4 o;
      o.x = run;
      run += v.x;
      o.y = run;
      run += v.y;
      o.z = run;
      run += v.z;
      o.w = run;
      run += v.w;
      rk4[j] = o;
    }
    __syncthreads();
    // per-digit offsets: even digit 2i adds the odd-digit totals of rows < i,
    // odd digit 2i+1 adds the even-digit totals of rows <= i
    for (int d = t; d < D; d += T) {
      const int i = d >> 1;
      if (d & 1) {
        const uint32_t S1 = (i + 1 < ROWS) ? s.c[pidx((i + 1) * T)] : total;
        s.dofs[d] = S1 & 0xFFFFu;
      } else {
        s.dofs[d] = s.c[pidx(i * T)] >> 16;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t d = (val[r] >> shift) & (D - 1);
      const uint32_t v = s.c[pidx((int)(d >> 1) * T + t)];
      out[r] = ((v >> ((d & 1u) << 4)) & 0xFFFFu) + s.dofs[d] + pre[r];
    }
    __syncthreads();
  }
};

// Conflict-free index for blocked reads of an array written at ranks.
__device__ __forceinline__ int bpad(int q) { return q + (q >> 5); }

// ---------------------------------------------------------------------------
// Records of the temporary arrays (array of structures, so a record is one
// contiguous access); V = void means keys only.
// ---------------------------------------------------------------------------
// Alignment of a record: the largest power of two (up to 16) that its size
// allows, so that one record moves with one vector load or store.
template <class K, class V>
struct RecAlign {
  static constexpr size_t bytes = sizeof(K) + sizeof(V);
  static constexpr size_t value = bytes > 8 ? 16 : (bytes > 4 ? 8 : 4);
};
template <class K, class V>
struct alignas(RecAlign<K, V>::value) RecT {
  K k;
  V v;
};
template <class K>
struct alignas(sizeof(K) >= 16 ? 16 : sizeof(K)) RecT<K, void> {
  K k;
};

// Slot of record i in a shared-memory staging buffer of RB-byte records.  An
// XOR swizzle inside every 128-byte row keeps both access patterns of the
// kernels free of bank conflicts: consecutive i (coalesced copies) and
// i = 16 t + r for t = 0..31 (thread t holding 16 consecutive records).
// PER = records each thread holds in the blocked pattern (a power of two).
template <int RB, int PER = 16>
__device__ __forceinline__ uint32_t sw(uint32_t i) {
  constexpr uint32_t L = RB >= 128 ? 1u : 128u / RB;  // records per 128-byte row
  constexpr int SH = PER == 16 ? 4 : PER == 8 ? 3 : PER == 4 ? 2 : 4;
  if constexpr (L <= 1)
    return i;
  else
    return (i & ~(L - 1)) | ((i ^ (i >> SH)) & (L - 1));
}

template <class V>
struct ValT {
  using type = V;
};
template <>
struct ValT<void> {
  using type = uint32_t;  // placeholder, never stored
};

// Bucketing hash of one recursion level: multiply-shift (Dietzfelbinger et
// al.) with a seeded odd multiplier per level; the light bucket is the top
// lbits bits (Sec. 3.1 takes the bucket from hash bits; a fresh multiplier
// per level plays the role of the next hash function of the family).
template <class K>
__device__ __forceinline__ uint64_t fold_key(const K& k) {
  return semisort::key_traits<K>::hash(k);
}
template <>
__device__ __forceinline__ uint64_t fold_key<uint32_t>(const uint32_t& k) { return k; }
template <>
__device__ __forceinline__ uint64_t fold_key<uint64_t>(const uint64_t& k) { return k; }
template <>
__device__ __forceinline__ uint64_t fold_key<k128>(const k128& k) { return k.lo ^ mix64(k.hi); }

}  // namespace ss
