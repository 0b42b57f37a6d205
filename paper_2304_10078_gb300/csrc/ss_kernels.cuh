// Kernels of the semisort pipeline (templated on key type K, value type V --
// void for keys only -- and the operation OP).  Included by one translation
// unit per key type through ss_launch.cuh.
//
// One recursion level of Algorithm 1 is the kernel sequence
//   plan -> sample -> count -> scan -> distribute -> scan_items -> emit
// over all segments of the level at once; a final `finish` kernel runs every
// base case (Sec. 3.3) and every copy-back (Sec. 3.4) collected on the way.
//
// Record layout: the caller's arrays are structure-of-arrays (keys[], vals[]);
// the two temporary arrays T and T2 hold records as array-of-structures
// (RecT<K,V>), so that one record is one contiguous access.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "ss_common.cuh"
#include "ss_learn.cuh"
#include "ss_plan.h"

namespace ss {

// ----------------------------------------------------------------------------
// Small helpers
// ----------------------------------------------------------------------------
__device__ __forceinline__ void set_error(Ctrl* c, uint32_t code) { atomicCAS(&c->error, 0u, code); }

__host__ __device__ __forceinline__ uint64_t level_salt(uint64_t seed, int level) {
  return mix64(seed ^ (0x9E3779B97F4A7C15ull * (uint64_t)(level + 1)));
}
__host__ __device__ __forceinline__ uint64_t refine_salt(uint64_t seed) { return mix64(seed ^ 0x5EF1CE5EF1CE0001ull); }

// Odd multiplier of a segment's bucketing hash: seeded by level and segment.
__host__ __device__ __forceinline__ uint64_t seg_mult(uint64_t seed, int level, uint64_t start) {
  return mix64(level_salt(seed, level) ^ (start * 0xD1B54A32D192ED03ull)) | 1ull;
}

__device__ __forceinline__ uint32_t ceil_log2_u32(uint32_t x) { return x <= 1 ? 0 : 32 - __clz(x - 1); }

// Buffers of one level (the launcher computes them).
struct LevelBufs {
  const void* src_k;  // SoA keys (src_aos == 0) or AoS records (src_aos == 1)
  const void* src_v;  // SoA values (src_aos == 0)
  void* dst;          // light buckets: AoS records (dst_aos == 1) or SoA keys
  void* dst_v;        // light buckets: SoA values (dst_aos == 0)
  void* hdst_k;       // heavy destination: SoA keys, or AoS records when hdst_aos
  void* hdst_v;
  uint32_t src_aos;
  uint32_t dst_aos;
  uint32_t hdst_aos;
  uint32_t dst_id;   // Buf id of dst
  uint32_t hdst_id;  // Buf id of the heavy destination
  int level;
};

__device__ __forceinline__ void* buf_ptr(const Work& w, uint32_t id) {
  return id == kBufIn ? const_cast<void*>(w.in_k) : id == kBufT ? w.t_k : id == kBufOut ? w.out_k : w.t2_k;
}

// Key access for SoA or AoS sources.
template <class K, class V>
__device__ __forceinline__ K load_key(const void* src, uint32_t aos, uint64_t i) {
  return aos ? reinterpret_cast<const RecT<K, V>*>(src)[i].k : reinterpret_cast<const K*>(src)[i];
}


// Heavy-key capacity of a segment (a power of two): hash-bucket segments keep
// n_L + capacity <= kMaxBuckets, range segments use hcap_of.
template <int OP>
__device__ __forceinline__ uint32_t seg_hcap(const Seg& sg) {
  return OP == kOpLess ? hcap_of(sg.lbits) : sg.nbcap - sg.nl;
}

// Bucket of key k in its segment (GetBucketId of Algorithm 1): the heavy
// bucket n_L + i if k is the i-th heavy key, else the light bucket given by
// the top lbits bits of the level hash.  hk/ht: the segment's heavy keys and
// its open-addressing table (4 slots per heavy key, so probes stay short).
// The light bucket is the hash scaled to [0, n_L): the top bits of the
// product when n_L is a power of two.
template <class K>
__device__ __forceinline__ uint32_t bucket_of(const K& k, uint64_t mult, uint32_t nl, uint32_t nh,
                                              const K* hk, const uint16_t* ht, uint32_t tmask,
                                              bool ident = false, uint32_t shift = 0) {
  const uint64_t f = fold_key<K>(k);
  const uint64_t h = f * mult;
  // identity hashing (semisort-i, Sec. 4.1): the key's own bits, lowest first,
  // each recursion level taking the next log2(n_L) bits (n_L a power of two)
  uint32_t b = ident ? (shift < 64 ? (uint32_t)(f >> shift) & (nl - 1) : 0u) : (uint32_t)__umul64hi(h, nl);
  if (nh) {
    uint32_t slot = (uint32_t)(h >> 20) & tmask;
    uint32_t e = ht[slot];
    while (e != 0xFFFFu) {
      if (KeyT<K>::eq(hk[e], k)) {
        b = nl + e;
        break;
      }
      slot = (slot + 1) & tmask;
      e = ht[slot];
    }
  }
  return b;
}

// semisort_< bucket of key k: with q sorted boundaries bnd[] (splitters and
// heavy keys, flags[i] = 1 for a heavy key), u = #boundaries <= k; range
// bucket 2u holds bnd[u-1] < k < bnd[u] (or bnd[u-1] <= k if bnd[u-1] is not
// heavy), equality bucket 2u-1 holds k == bnd[u-1] for a heavy boundary.  Bucket
// ids therefore increase with the key, so concatenating the buckets in id order
// is a key-ordered partition (samplesort with equality buckets).
template <class K>
__device__ __forceinline__ uint32_t bucket_less(const K& k, const K* bnd, const uint16_t* flags, uint32_t q) {
  uint32_t lo = 0, hi = q;  // upper bound: first boundary > k
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (KeyT<K>::lt(k, bnd[mid]))
      hi = mid;
    else
      lo = mid + 1;
  }
  if (lo > 0 && flags[lo - 1] && KeyT<K>::eq(bnd[lo - 1], k)) return 2 * lo - 1;
  return 2 * lo;
}

// semisort_< bucket through the top level's lookup table: the boundaries
// that can order a key are those of its cell, so the search covers only them.
template <class K>
__device__ __forceinline__ uint32_t bucket_less_tab(const K& k, const K* bnd, const uint16_t* flags,
                                                    const uint16_t* cell, uint64_t kmin, uint32_t shift) {
  const uint64_t kk = (uint64_t)k;
  uint64_t c = kk > kmin ? (kk - kmin) >> shift : 0;
  c = c < kTopCells - 1 ? c : kTopCells - 1;
  uint32_t lo = cell[c], hi = cell[c + 1];
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (KeyT<K>::lt(k, bnd[mid]))
      hi = mid;
    else
      lo = mid + 1;
  }
  if (lo > 0 && flags[lo - 1] && KeyT<K>::eq(bnd[lo - 1], k)) return 2 * lo - 1;
  return 2 * lo;
}

// The same search through a narrow level's key-cell table: 2^cbits cells
// over [kmin, kmin + 2^(shift + cbits)), keys outside clamped to the end cells.
template <class K>
__device__ __forceinline__ uint32_t bucket_less_cells(const K& k, const K* bnd, const uint16_t* flags,
                                                      const uint16_t* cell, uint64_t kmin, uint32_t shift,
                                                      uint32_t cbits) {
  const uint64_t kk = (uint64_t)k;
  uint64_t c = kk > kmin ? (kk - kmin) >> shift : 0;
  const uint64_t last = (1u << cbits) - 1;
  c = c < last ? c : last;
  uint32_t lo = cell[c], hi = cell[c + 1];
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (KeyT<K>::lt(k, bnd[mid]))
      hi = mid;
    else
      lo = mid + 1;
  }
  if (lo > 0 && flags[lo - 1] && KeyT<K>::eq(bnd[lo - 1], k)) return 2 * lo - 1;
  return 2 * lo;
}

// Whether the semisort_< top level uses the wide bucket space (2^16-key
// sample, up to 2^12 ranges, a lookup table over the key range): for
// unsigned integer keys of up to 8 bytes, whose wide distribute buffers fit in
// shared memory.
template <class K, int OP>
struct TopWide {
  static constexpr bool value = OP == kOpLess && KeyT<K>::kIntegral;
};

// Whether bucket b holds a single heavy key (final after distribution).
template <int OP>
__device__ __forceinline__ bool is_heavy(uint32_t b, uint32_t nl) {
  return OP == kOpLess ? (b & 1u) != 0 : b >= nl;
}

// Bucket of a key in segment sg (its tables already in shared memory).
template <class K, int OP>
__device__ __forceinline__ uint32_t bucket_in(const K& k, const Seg& sg, const K* hk, const uint16_t* ht,
                                              uint32_t tmask) {
  if constexpr (OP == kOpLess)
    return bucket_less<K>(k, hk, ht, sg.nh);
  else
    return bucket_of<K>(k, sg.mult, sg.nl, sg.nh, hk, ht, tmask, sg.ident != 0, sg.shift);
}

// ----------------------------------------------------------------------------
// init: reset the control block and seed level 0 (or a single base case).
// ----------------------------------------------------------------------------
static __global__ void __launch_bounds__(1024) k_init(Work w) {
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t carry[2];
  __shared__ uint32_t bad;
  Ctrl* c = w.ctrl;
  if (threadIdx.x == 0) {
    for (int l = 0; l < kMaxLevels; ++l) {
      c->nsegs[l] = 0;
      c->ntiles[l] = 0;
    }
    c->nfin = 0;
    c->error = 0;
    for (int i = 0; i < 16; ++i) c->stats[i] = 0;
    bad = 0;
    carry[0] = carry[1] = 0;
  }
  __syncthreads();
  if (w.n == 0) return;
  if (w.offsets == nullptr) {
    if (threadIdx.x != 0) return;
    if (w.n <= w.alpha) {
      Item it;
      it.start = 0;
      it.len = (uint32_t)w.n;
      it.kind = kItemRefine;
      it.buf = kBufIn;
      it.aux = it.aux2 = 0;
      it.level = 0;
      w.items[0] = it;
      c->nfin = 1;
    } else {
      Seg s = {};
      s.start = 0;
      s.len = (uint32_t)w.n;
      s.ident = w.ident;
      w.segs[0][0] = s;
      c->nsegs[0] = 1;
    }
    return;
  }
  // batched: check the offsets, then instances of at most alpha records become
  // base-case items and larger ones level-0 segments, both in instance order
  const uint64_t* off = w.offsets;
  const uint32_t ni = w.num_inst;
  for (uint32_t i = threadIdx.x; i < ni; i += blockDim.x)
    if (off[i] > off[i + 1]) bad = 1;
  if (threadIdx.x == 0 && (off[0] != 0 || off[ni] != w.n)) bad = 1;
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) set_error(c, 1 /*SS_ERR_INVALID_ARG*/);
    return;
  }
  for (uint32_t i0 = 0; i0 < ni; i0 += blockDim.x) {
    const uint32_t i = i0 + threadIdx.x;
    const uint64_t len = i < ni ? off[i + 1] - off[i] : 0;
    const uint32_t small = len > 0 && len <= w.alpha, big = len > w.alpha;
    uint32_t ts, tb;
    const uint32_t es = block_exclusive_scan(small, tmp, &ts);
    const uint32_t eb = block_exclusive_scan(big, tmp, &tb);
    if (small) {
      Item it;
      it.start = off[i];
      it.len = (uint32_t)len;
      it.kind = kItemRefine;
      it.buf = kBufIn;
      it.aux = it.aux2 = 0;
      it.level = kDirectLevel;
      w.items[carry[0] + es] = it;
    }
    if (big) {
      Seg s = {};
      s.start = off[i];
      s.len = (uint32_t)len;
      s.ident = w.ident;
      w.segs[0][carry[1] + eb] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry[0] += ts;
      carry[1] += tb;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    c->nfin = carry[0];
    c->nsegs[0] = carry[1];
  }
}

// ----------------------------------------------------------------------------
// plan: per segment of level `level`, pick n_L, cut it into subarrays, and
// lay out its rows of the count matrix.  One CTA.
// ----------------------------------------------------------------------------
template <int OP>
__global__ void __launch_bounds__(1024) k_plan(Work w, int level) {
  __shared__ uint64_t tmp64[33];
  __shared__ uint64_t carry[3];
  const uint32_t ns = w.ctrl->nsegs[level];
  if (ns == 0) return;
  if (threadIdx.x < 3) carry[threadIdx.x] = 0;
  __syncthreads();
  Seg* segs = w.segs[level];
  const uint32_t l = level == 0 ? w.l1 : w.l2;
  for (uint32_t b0 = 0; b0 < ns; b0 += blockDim.x) {
    const uint32_t s = b0 + threadIdx.x;
    const uint64_t base_t = carry[0], base_b = carry[1], base_c = carry[2];
    uint64_t nt = 0, nb2 = 0, cc = 0;
    Seg sg;
    if (s < ns) {
      sg = segs[s];
      uint32_t lb;
      const bool top_single = level == 0 && w.num_inst <= 1;
      if (top_single) {
        lb = w.lbits1;
      } else {
        const uint64_t want = (2ull * sg.len + w.alpha - 1) / w.alpha;
        lb = want <= 2 ? 1u : (uint32_t)(64 - __clzll(want - 1));
        lb = lb > (uint32_t)kMaxLightLog2 ? (uint32_t)kMaxLightLog2 : lb;
      }
      if (OP == kOpLess && !top_single && lb > kMaxLightLog2 - 1) lb = kMaxLightLog2 - 1;
      uint32_t nl = 1u << lb, hcap = hcap_of(lb);
      // hash buckets: a segment wanting more than 512 light buckets gets 768
      // (and room for 256 heavy keys), still 1024 bucket ids in all
      if (OP != kOpLess && !sg.ident && lb == (uint32_t)kMaxLightLog2 && (!top_single || w.auto_nl)) {
        const uint64_t want = (2ull * (top_single ? w.n : sg.len) + w.alpha - 1) / w.alpha;
        if (want > 512) {
          nl = 768;
          hcap = 256;
        }
      }
      sg.lbits = lb;
      sg.nl = nl;
      // semisort_<: q <= (n_L - 1) + n_L boundaries give 2q + 1 < 4 n_L bucket ids
      sg.nbcap = OP == kOpLess ? 4 * nl : nl + hcap;
      sg.nh = 0;
      sg.nb = nl;
      sg.mult = seg_mult(w.seed, level, sg.start);
      sg.ntiles = (uint32_t)((sg.len + (uint64_t)l - 1) / l);
      nt = sg.ntiles;
      nb2 = sg.nbcap;
      cc = (uint64_t)sg.nbcap * sg.ntiles;
    }
    uint64_t tt, tb, tc;
    const uint64_t pt = block_exclusive_scan64(nt, tmp64, &tt);
    const uint64_t pb = block_exclusive_scan64(nb2, tmp64, &tb);
    const uint64_t pc = block_exclusive_scan64(cc, tmp64, &tc);
    if (s < ns) {
      sg.first_tile = (uint32_t)(base_t + pt);
      sg.bbase = (uint32_t)(base_b + pb);
      sg.cbase = base_c + pc;
      if (base_t + pt + nt > w.tile_cap[level] || base_b + pb + nb2 > w.bucket_cap[level] ||
          base_c + pc + cc > w.c_cap[level]) {
        set_error(w.ctrl, 4 /*SS_ERR_CAPACITY*/);
        sg.ntiles = 0;
        sg.lbits = 0;  // marks the segment as skipped for every later kernel
      }
      segs[s] = sg;
      Tile* tiles = w.tiles[level];
      for (uint32_t t = 0; t < sg.ntiles; ++t) {
        Tile tl;
        tl.start = sg.start + (uint64_t)t * l;
        const uint64_t rem = sg.len - (uint64_t)t * l;
        tl.len = (uint32_t)(rem < l ? rem : l);
        tl.seg = s;
        tl.idx = t;
        tl.pad = 0;
        tiles[sg.first_tile + t] = tl;
      }
      // records distributed per level (levels 4 and deeper share the last entry)
      atomicAdd((unsigned long long*)&w.ctrl->stats[1 + (level < 3 ? level : 3)], (unsigned long long)sg.len);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry[0] += tt;
      carry[1] += tb;
      carry[2] += tc;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    w.ctrl->ntiles[level] = (uint32_t)carry[0];
    atomicMax((unsigned long long*)&w.ctrl->stats[0], (unsigned long long)(level + 1));
  }
}

// ----------------------------------------------------------------------------
// sample: Sampling and Bucketing (Sec. 3.1).  Per segment draw |S| keys at
// seeded random positions, sort them, and make every key seen at least
// tau = |S| / n_H,cap times heavy (a key expected to fill at least one light
// bucket).  Heavy keys get ids in ascending key order (deterministic) and an
// open-addressing lookup table with 4 slots per heavy key.  semisort_< also
// takes n_L - 1 splitters at evenly spaced sample ranks and merges them with
// the heavy keys into one sorted boundary list (equality buckets for heavy
// keys, samplesort-style).
// ----------------------------------------------------------------------------
// Largest sample count a range bucket of the learned splitters may hold
// before the sampled splitters replace them: twice the light keys' share of a
// range, plus four standard deviations of a sample count of that size (with
// 2^16 sample keys and 4096 ranges a range holds about 16 of them, and even
// exact splitters show a largest count near 31 from counting noise alone).
__device__ __forceinline__ uint32_t judge_limit(uint32_t share) {
  const float t = 2.0f * (float)(share > 1 ? share : 1);
  return (uint32_t)(t + 4.0f * sqrtf(t));
}

// First position of the sorted S[0, m) holding a key > k (upper) or >= k.
template <class K>
__device__ __forceinline__ uint32_t sorted_bound(const K* S, uint32_t m, const K& k, bool upper) {
  uint32_t lo = 0, hi = m;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (upper ? !KeyT<K>::lt(k, S[mid]) : KeyT<K>::lt(S[mid], k))
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

template <class K, class V, int OP>
__global__ void __launch_bounds__(1024) k_sample(Work w, LevelBufs lb, uint32_t s_cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  K* S = reinterpret_cast<K*>(smem);
  __shared__ uint32_t tab[4 * kMaxHeavy];
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t nh_sh;
  if (TopWide<K, OP>::value && lb.level == 0 && w.num_inst <= 1) return;  // the wide top level uses k_less_split
  const uint32_t ns = w.ctrl->nsegs[lb.level];
  for (uint32_t s = blockIdx.x; s < ns; s += gridDim.x) {
    const Seg sg = w.segs[lb.level][s];
    if (sg.lbits == 0) continue;
    const uint32_t hcap = seg_hcap<OP>(sg);
    uint32_t S_n = 16u * hcap;
    if (S_n > s_cap) S_n = s_cap;
    const uint32_t tau = S_n / hcap;
    const uint64_t base = mix64(level_salt(w.seed, lb.level) ^ (sg.start * 0xD1B54A32D192ED03ull) ^ 0x5A4Dull);
    for (uint32_t t = threadIdx.x; t < S_n; t += blockDim.x) {
      const uint64_t r = mix64(base + (uint64_t)(t + 1) * 0x9E3779B97F4A7C15ull);
      const uint64_t pos = __umul64hi(r, (uint64_t)sg.len);
      S[t] = load_key<K, V>(lb.src_k, lb.src_aos, sg.start + pos);
    }
    __syncthreads();
    // bitonic sort of S (S_n is a power of two)
    for (uint32_t k = 2; k <= S_n; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        for (uint32_t p = threadIdx.x; p < S_n / 2; p += blockDim.x) {
          const uint32_t i = (p / j) * 2 * j + (p % j);
          const uint32_t ixj = i + j;
          const bool up = (i & k) == 0;
          const K a = S[i], b = S[ixj];
          if (up ? KeyT<K>::lt(b, a) : KeyT<K>::lt(a, b)) {
            S[i] = b;
            S[ixj] = a;
          }
        }
        __syncthreads();
      }
    }
    // heavy keys: run starts whose run reaches length tau, in key order
    const uint32_t tsize = 4 * hcap;
    for (uint32_t t = threadIdx.x; t < tsize; t += blockDim.x) tab[t] = kEmpty;
    if (threadIdx.x == 0) nh_sh = 0;
    __syncthreads();
    K* hk = reinterpret_cast<K*>(w.hkeys[lb.level]) + sg.bbase;
    for (uint32_t t0 = 0; t0 < S_n; t0 += blockDim.x) {
      const uint32_t t = t0 + threadIdx.x;
      uint32_t f = 0;
      if (t < S_n && (t == 0 || !KeyT<K>::eq(S[t], S[t - 1])) && t + tau - 1 < S_n &&
          KeyT<K>::eq(S[t + tau - 1], S[t]))
        f = 1;
      uint32_t tot;
      const uint32_t ex = block_exclusive_scan(f, tmp, &tot);
      const uint32_t idx = nh_sh + ex;
      if (f && idx < hcap) hk[idx] = S[t];
      __syncthreads();
      if (threadIdx.x == 0) nh_sh += tot;
      __syncthreads();
    }
    const uint32_t nh = nh_sh < hcap ? nh_sh : hcap;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nh; i += blockDim.x) {
      const uint64_t h = fold_key<K>(hk[i]) * sg.mult;
      uint32_t slot = (uint32_t)(h >> 20) & (tsize - 1);
      while (atomicCAS(&tab[slot], kEmpty, i) != kEmpty) slot = (slot + 1) & (tsize - 1);
    }
    __syncthreads();
    uint16_t* ht = w.htab[lb.level] + 2ull * sg.bbase;
    if constexpr (OP == kOpLess) {
      const uint32_t nl = sg.nl;
      K* bnd = reinterpret_cast<K*>(w.splitters[lb.level]) + sg.bbase;
      // batched calls in learned mode: the shared CDF model's splitters for
      // this instance (the inverted splitters at 2^8 ranges, every
      // 2^(8 - lbits)-th of them), judged against the sampled ones below
      const LearnState* L = nullptr;
      if constexpr (KeyT<K>::kIntegral) {
        if (lb.level == 0 && w.num_inst > 1 && w.splitter_mode == 1) L = reinterpret_cast<const LearnState*>(w.learn);
      }
      const bool model = L != nullptr && L->usable && sg.lbits <= kBatchLearnLog2;
      auto cand = [&](uint32_t j, bool use_model) -> K {
        if (use_model) return reinterpret_cast<const K*>(L->splitters)[(j << (kBatchLearnLog2 - sg.lbits)) - 1];
        return S[(uint64_t)j * S_n / nl];
      };
      // merge the n_L - 1 candidate splitters (deduplicated) with the heavy
      // keys into the sorted boundaries; returns their number (thread 0)
      auto merge = [&](bool use_model) {
        if (threadIdx.x == 0) {
          uint32_t q = 0, j = 1, hi = 0;
          bool have_last = false;
          K last = S[0], prev = S[0];
          while (j < nl || hi < nh) {
            K cj = j < nl ? cand(j, use_model) : S[0];
            if (use_model && j < nl && j > 1 && KeyT<K>::lt(cj, prev)) cj = prev;  // FP32 rounding: keep it sorted
            K c;
            bool heavy;
            if (j < nl && (hi >= nh || KeyT<K>::lt(cj, hk[hi]))) {
              c = cj;
              heavy = false;
              prev = cj;
              ++j;
            } else if (j < nl && KeyT<K>::eq(cj, hk[hi])) {
              c = hk[hi];
              heavy = true;
              prev = cj;
              ++j;
              ++hi;
            } else {
              c = hk[hi];
              heavy = true;
              ++hi;
            }
            if (have_last && KeyT<K>::eq(c, last)) {
              if (heavy) ht[q - 1] = 1;
              continue;
            }
            bnd[q] = c;
            ht[q] = heavy ? 1 : 0;
            ++q;
            last = c;
            have_last = true;
          }
          nh_sh = q;
        }
        __syncthreads();
        return nh_sh;
      };
      // the largest range bucket of the boundaries on this segment's sample
      auto max_range = [&](uint32_t q) {
        if (threadIdx.x == 0) tmp[32] = 0;
        __syncthreads();
        uint32_t mx = 0;
        for (uint32_t u = threadIdx.x; u <= q; u += blockDim.x) {
          const uint32_t lo = u == 0 ? 0u : sorted_bound<K>(S, S_n, bnd[u - 1], ht[u - 1] != 0);
          const uint32_t hi = u == q ? S_n : sorted_bound<K>(S, S_n, bnd[u], false);
          mx = hi > lo && hi - lo > mx ? hi - lo : mx;
        }
        atomicMax(&tmp[32], mx);
        __syncthreads();
        const uint32_t r = tmp[32];
        __syncthreads();
        return r;
      };
      uint32_t q = merge(false);
      if (model) {
        const uint32_t max_s = max_range(q);
        // light sample keys: those not equal to a heavy key
        if (threadIdx.x == 0) tmp[32] = 0;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < nh; i += blockDim.x)
          atomicAdd(&tmp[32], sorted_bound<K>(S, S_n, hk[i], true) - sorted_bound<K>(S, S_n, hk[i], false));
        __syncthreads();
        const uint32_t heavy_n = tmp[32];
        __syncthreads();
        const uint32_t share = (S_n - heavy_n + nl - 1) / nl;
        q = merge(true);
        const uint32_t max_l = max_range(q);
        const bool reject = max_l > judge_limit(share) && max_l > max_s;
        if (reject) q = merge(false);
        if (threadIdx.x == 0 && !reject) atomicAdd((unsigned long long*)&w.ctrl->stats[12], 1ull);
      }
      // key-cell table (integer keys): 2 n_L cells of equal key width over
      // the range of the sample and the boundaries; cell c lists the
      // boundaries from cell[c] (those below the cell's first key) to
      // cell[c + 1], so a key's search covers only its own cell's boundaries
      uint32_t cbits = 0;
      if constexpr (KeyT<K>::kIntegral) {
        cbits = sg.lbits + 1;
        const uint64_t kmin = q && (uint64_t)bnd[0] < (uint64_t)S[0] ? (uint64_t)bnd[0] : (uint64_t)S[0];
        const uint64_t kmax =
            q && (uint64_t)bnd[q - 1] > (uint64_t)S[S_n - 1] ? (uint64_t)bnd[q - 1] : (uint64_t)S[S_n - 1];
        const uint64_t range = kmax - kmin;
        const uint32_t bits = range ? 64 - __clzll((long long)range) : 0;
        const uint32_t shift = bits > cbits ? bits - cbits : 0;
        uint16_t* cell = w.lcell[lb.level] + 2ull * sg.bbase;
        for (uint32_t c = threadIdx.x; c <= (1u << cbits); c += blockDim.x) {
          uint32_t v = q;
          const uint64_t off = c < (1u << cbits) ? (uint64_t)c << shift : ~0ull;
          if (off <= range) {
            const K start = (K)(kmin + off);
            uint32_t lo = 0, hi = q;  // boundaries below the cell's first key
            while (lo < hi) {
              const uint32_t mid = (lo + hi) >> 1;
              if (KeyT<K>::lt(bnd[mid], start))
                lo = mid + 1;
              else
                hi = mid;
            }
            v = lo;
          }
          cell[c] = (uint16_t)v;
        }
        if (threadIdx.x == 0) {
          w.segs[lb.level][s].mult = kmin;
          w.segs[lb.level][s].shift = shift;
        }
      }
      if (threadIdx.x == 0) {
        w.segs[lb.level][s].nh = q;
        w.segs[lb.level][s].nb = 2 * q + 1;
        w.segs[lb.level][s].cbits = cbits;
        if (lb.level == 0) w.ctrl->stats[7] = nh;
      }
    } else {
      for (uint32_t t = threadIdx.x; t < tsize; t += blockDim.x) ht[t] = (uint16_t)(tab[t] == kEmpty ? 0xFFFFu : tab[t]);
      if (threadIdx.x == 0) {
        w.segs[lb.level][s].nh = nh;
        w.segs[lb.level][s].nb = sg.nl + nh;
        if (lb.level == 0) w.ctrl->stats[7] = nh;
      }
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// semisort_< top level: a sample of kBigSample keys, sorted on the device.
// Each CTA gathers one run of the sample at seeded positions and sorts it in
// shared memory (bitonic); a merge kernel then places every key at its rank
// in the whole sample (positions inside its run plus, in every other run, the
// keys that order before it -- ties go to the earlier run), a stable merge.
// ----------------------------------------------------------------------------
template <class K>
struct BigRun {
  static constexpr uint32_t len = sizeof(K) >= 16 ? 8192u : 16384u;  // keys per sorted run
  static constexpr uint32_t runs = kBigSample / len;
};

template <class K>
__global__ void __launch_bounds__(1024) k_bigsample_sort(Work w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* S = reinterpret_cast<K*>(smem_raw);
  constexpr uint32_t L = BigRun<K>::len;
  const K* in = reinterpret_cast<const K*>(w.in_k);
  const uint64_t base = mix64(level_salt(w.seed, 0) ^ 0xB165A3F1E5EEDull);
  for (uint32_t t = threadIdx.x; t < L; t += blockDim.x) {
    const uint64_t gi = (uint64_t)blockIdx.x * L + t;
    const uint64_t r = mix64(base + (gi + 1) * 0x9E3779B97F4A7C15ull);
    S[t] = in[__umul64hi(r, w.n)];
  }
  __syncthreads();
  for (uint32_t k = 2; k <= L; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t p = threadIdx.x; p < L / 2; p += blockDim.x) {
        const uint32_t i = ((p & ~(j - 1)) << 1) | (p & (j - 1));
        const K a = S[i], b = S[i + j];
        if ((i & k) == 0 ? KeyT<K>::lt(b, a) : KeyT<K>::lt(a, b)) {
          S[i] = b;
          S[i + j] = a;
        }
      }
      __syncthreads();
    }
  }
  K* out = reinterpret_cast<K*>(w.bigs_tmp) + (uint64_t)blockIdx.x * L;
  for (uint32_t t = threadIdx.x; t < L; t += blockDim.x) out[t] = S[t];
}

template <class K>
__global__ void __launch_bounds__(256) k_bigsample_merge(Work w) {
  constexpr uint32_t L = BigRun<K>::len;
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kBigSample) return;
  const K* runs = reinterpret_cast<const K*>(w.bigs_tmp);
  const uint32_t r = e / L;
  const K key = runs[e];
  uint32_t rank = e % L;
  for (uint32_t q = 0; q < BigRun<K>::runs; ++q) {
    if (q == r) continue;
    const K* R = runs + (uint64_t)q * L;
    uint32_t lo = 0, hi = L;  // earlier runs: keys <= key; later runs: keys < key
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      const bool before = q < r ? !KeyT<K>::lt(key, R[mid]) : KeyT<K>::lt(R[mid], key);
      if (before)
        lo = mid + 1;
      else
        hi = mid;
    }
    rank += lo;
  }
  reinterpret_cast<K*>(w.bigs)[rank] = key;
}

// Boundaries of the semisort_< top level from the sorted sample: n_L - 1
// candidate splitters -- keys at evenly spaced sample ranks, or, in learned
// mode, the integer splitters inverted from the CDF model -- merged with the
// heavy keys (keys whose sample run reaches the expected size of one range
// bucket, at most min(n_L, 512) of them in key order) into one sorted list with
// a flag per heavy key (equality buckets, as in k_sample).  The sampled
// splitters judge the learned ones on the sample through the largest range
// bucket: the model is rejected (sampled splitters used) when its largest
// range bucket holds more than twice the light (non-heavy) sample keys'
// share of a range (plus the sample's counting noise, judge_limit) and more
// than the sampled splitters' largest one.
// stats[11]: 0 sampled, 1 learned, 2 learned rejected or not usable;
// stats[12]: the largest range bucket's sample count; stats[14]: the top
// level's n_L; stats[15]: Adam steps of the training.  One CTA.
template <class K>
__device__ __forceinline__ uint32_t sample_lower(const K* S, const K& k, bool upper) {
  uint32_t lo = 0, hi = kBigSample;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (upper ? !KeyT<K>::lt(k, S[mid]) : KeyT<K>::lt(S[mid], k))
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

template <class K>
__global__ void __launch_bounds__(1024) k_less_split(Work w, const LearnState* L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t nh_sh, q_sh, maxc_sh;
  Seg* sgp = w.segs[0];
  if (w.ctrl->nsegs[0] == 0 || sgp[0].lbits == 0) return;
  const uint32_t nl = 1u << sgp[0].lbits;
  const uint32_t hcap = hcap_of(sgp[0].lbits);
  const K* S = reinterpret_cast<const K*>(w.bigs);
  uint32_t tau = kBigSample / nl;
  if (tau < 2) tau = 2;
  K* cs = reinterpret_cast<K*>(smem_raw);  // n_L - 1 candidate splitters
  K* hs = cs + nl;                         // heavy keys (at most hcap)
  K* bs = hs + kMaxHeavy;                  // merged boundaries (< 2 n_L)
  uint16_t* fs = reinterpret_cast<uint16_t*>(bs + 2 * nl);
  bool learned = L != nullptr && L->usable;
  // heavy keys
  if (threadIdx.x == 0) nh_sh = 0;
  __syncthreads();
  for (uint32_t t0 = 0; t0 < kBigSample; t0 += blockDim.x) {
    const uint32_t t = t0 + threadIdx.x;
    const uint32_t f = (t < kBigSample && (t == 0 || !KeyT<K>::eq(S[t], S[t - 1])) && t + tau - 1 < kBigSample &&
                        KeyT<K>::eq(S[t + tau - 1], S[t]))
                           ? 1u
                           : 0u;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan(f, tmp, &tot);
    if (f && nh_sh + ex < hcap) hs[nh_sh + ex] = S[t];
    __syncthreads();
    if (threadIdx.x == 0) nh_sh += tot;
    __syncthreads();
  }
  const uint32_t nh = nh_sh < hcap ? nh_sh : hcap;
  // Learned mode judges both splitter sets on the sample: the sampled ones
  // first (their largest range bucket), then the learned ones, which are kept
  // unless their largest range bucket exceeds twice the light keys' share of
  // a range and also the sampled splitters' largest one; a rejected model
  // means a third pass rebuilds the sampled boundaries.
  const uint32_t share = (L != nullptr ? (L->light + nl - 1) / nl : kBigSample / nl);
  const int passes = learned ? 3 : 1;
  uint32_t max_sampled = 0;
  for (int attempt = 0; attempt < passes; ++attempt) {
    const bool use_model = learned && attempt == 1;
    for (uint32_t j = 1 + threadIdx.x; j < nl; j += blockDim.x)
      cs[j - 1] = use_model ? reinterpret_cast<const K*>(L->splitters)[j - 1] : S[(uint64_t)j * kBigSample / nl];
    __syncthreads();
    if (threadIdx.x == 0) {
      if (use_model)  // the bisection in FP32 may step back by a rounding: make the list non-decreasing
        for (uint32_t j = 1; j + 1 < nl; ++j)
          if (KeyT<K>::lt(cs[j], cs[j - 1])) cs[j] = cs[j - 1];
      // q <= (n_L - 1) + hcap < 2 n_L boundaries
      uint32_t q = 0, j = 0, hi = 0;
      bool have_last = false;
      K last = cs[0];
      while (j + 1 < nl || hi < nh) {
        K c;
        bool heavy;
        if (j + 1 < nl && (hi >= nh || KeyT<K>::lt(cs[j], hs[hi]))) {
          c = cs[j++];
          heavy = false;
        } else if (j + 1 < nl && KeyT<K>::eq(cs[j], hs[hi])) {
          c = hs[hi++];
          ++j;
          heavy = true;
        } else {
          c = hs[hi++];
          heavy = true;
        }
        if (have_last && KeyT<K>::eq(c, last)) {
          if (heavy) fs[q - 1] = 1;
          continue;
        }
        bs[q] = c;
        fs[q] = heavy ? 1 : 0;
        ++q;
        last = c;
        have_last = true;
      }
      q_sh = q;
      maxc_sh = 0;
    }
    __syncthreads();
    const uint32_t q = q_sh;
    // sample count of every range bucket u (keys between boundaries u-1 and u)
    uint32_t mx = 0;
    for (uint32_t u = threadIdx.x; u <= q; u += blockDim.x) {
      const uint32_t lo = u == 0 ? 0u : sample_lower<K>(S, bs[u - 1], fs[u - 1] != 0);
      const uint32_t hi = u == q ? kBigSample : sample_lower<K>(S, bs[u], false);
      const uint32_t c = hi > lo ? hi - lo : 0u;
      mx = c > mx ? c : mx;
    }
    atomicMax(&maxc_sh, mx);
    __syncthreads();
    if (attempt == 0 && learned) {
      max_sampled = maxc_sh;
      __syncthreads();
      continue;
    }
    if (attempt == 1) {
      const bool reject = maxc_sh > judge_limit(share) && maxc_sh > max_sampled;
      if (!reject) break;
      learned = false;  // fall back to the sampled splitters (rebuilt by the third pass)
      __syncthreads();
    }
  }
  const uint32_t q = q_sh;
  K* bnd = reinterpret_cast<K*>(w.splitters[0]) + sgp[0].bbase;
  uint16_t* fl = w.htab[0] + 2ull * sgp[0].bbase;
  for (uint32_t u = threadIdx.x; u < q; u += blockDim.x) {
    bnd[u] = bs[u];
    fl[u] = fs[u];
  }
  // lookup table: cells of 2^shift keys from the sample minimum, 4096 cells
  // spanning the sample's key range; cell[c] = boundaries below cell c's start
  {
    const uint64_t kmin = (uint64_t)S[0], range = (uint64_t)S[kBigSample - 1] - kmin;
    const uint32_t bits = range ? 64 - __clzll((long long)range) : 0;
    const uint32_t shift = bits > 12 ? bits - 12 : 0;
    TopTable* T = w.toptab;
    for (uint32_t c = threadIdx.x; c <= kTopCells; c += blockDim.x) {
      uint32_t lo = 0;
      if (c == kTopCells || (c > 0 && ((uint64_t)c << shift) > ~0ull - kmin)) {
        lo = q;
      } else if (c > 0) {
        const uint64_t start = kmin + ((uint64_t)c << shift);  // first key of cell c
        uint32_t hi = q;
        while (lo < hi) {
          const uint32_t mid = (lo + hi) >> 1;
          if ((uint64_t)bs[mid] < start)
            lo = mid + 1;
          else
            hi = mid;
        }
      }
      T->cell[c] = (uint16_t)lo;
    }
    if (threadIdx.x == 0) {
      T->kmin = kmin;
      T->shift = shift;
      T->q = q;
    }
  }
  if (threadIdx.x == 0) {
    sgp[0].nh = q;
    sgp[0].nb = 2 * q + 1;
    w.ctrl->stats[7] = nh;
    w.ctrl->stats[11] = L == nullptr ? 0u : learned ? 1u : 2u;
    w.ctrl->stats[12] = maxc_sh;
    w.ctrl->stats[14] = nl;
    w.ctrl->stats[15] = L == nullptr ? 0u : L->steps_done;
  }
}

// Shared memory of k_less_split for keys of type K.
template <class K>
constexpr size_t less_split_smem() {
  return ((size_t)(1u << kLessTopLog2) + kMaxHeavy + 2 * (1u << kLessTopLog2)) * sizeof(K) +
         2 * (1u << kLessTopLog2) * sizeof(uint16_t);
}

// Load a segment's heavy keys and table (semisort_<: boundaries and flags)
// into shared memory.
template <class K, int OP>
__device__ __forceinline__ void load_heavy(const Work& w, int level, const Seg& sg, K* hk, uint16_t* ht) {
  if (OP == kOpLess) {
    const K* gb = reinterpret_cast<const K*>(w.splitters[level]) + sg.bbase;
    const uint16_t* gf = w.htab[level] + 2ull * sg.bbase;
    for (uint32_t i = threadIdx.x; i < sg.nh; i += blockDim.x) {
      hk[i] = gb[i];
      ht[i] = gf[i];
    }
  } else if (sg.nh) {
    const uint32_t tsize = 4 * seg_hcap<OP>(sg);
    const K* ghk = reinterpret_cast<const K*>(w.hkeys[level]) + sg.bbase;
    const uint16_t* ght = w.htab[level] + 2ull * sg.bbase;
    for (uint32_t i = threadIdx.x; i < sg.nh; i += blockDim.x) hk[i] = ghk[i];
    for (uint32_t i = threadIdx.x; i < tsize; i += blockDim.x) ht[i] = ght[i];
  }
}

// ----------------------------------------------------------------------------
// count: the counting matrix C of Blocked Distributing (Sec. 3.2).  One CTA
// per subarray; plain shared-memory atomic increments (their order does not
// matter for a count).  Collect-reduce also sums the values of heavy records
// per subarray here, so they are never moved (Sec. 3.5).
// ----------------------------------------------------------------------------
constexpr int kCountThreads = 512;

// Bucket-id space of a level: the wide semisort_< top level (BIG) or the rest.
// Cells of a narrow semisort_< level's key-cell table: 2 n_L <= 512.
constexpr uint32_t kSegCells = 2u << (kMaxLightLog2 - 1);

template <bool BIG>
struct Space {
  static constexpr uint32_t kIds = BIG ? kBigBuckets : kMaxBuckets;   // bucket ids
  static constexpr uint32_t kBnd = BIG ? kBigBounds : kMaxHeavy;      // heavy keys / boundaries
  static constexpr uint32_t kTab = kBnd > 4 * kMaxHeavy ? kBnd : 4 * kMaxHeavy;  // table / flags
};

template <class K, int OP, bool BIG>
struct CountSmem {
  uint32_t hist[Space<BIG>::kIds];
  K hk[Space<BIG>::kBnd];
  uint16_t ht[Space<BIG>::kTab];
  // collect-reduce: per-subarray sums of the heavy keys' values, eight copies
  // per key (picked by lane) so that a warp's records of one key collide at
  // most four ways in the shared-memory atomics
  unsigned long long hsum[OP == kOpReduce ? kMaxHeavy * 8 : 1];
  uint16_t cell[BIG ? kTopCells + 1 : OP == kOpLess ? kSegCells + 1 : 1];
};

// The wide top level's lookup table into shared memory.
template <bool BIG>
__device__ __forceinline__ void load_cells(const Work& w, uint16_t* cell, uint64_t* kmin, uint32_t* shift) {
  if constexpr (BIG) {
    for (uint32_t i = threadIdx.x; i <= kTopCells; i += blockDim.x) cell[i] = w.toptab->cell[i];
    *kmin = w.toptab->kmin;
    *shift = w.toptab->shift;
  }
}

// A narrow semisort_< level's key-cell table into shared memory (integer
// keys; sg.cbits == 0: the segment has none and the search covers all its
// boundaries).
template <class K, int OP, bool BIG>
__device__ __forceinline__ void load_seg_cells(const Work& w, int level, const Seg& sg, uint16_t* cell) {
  if constexpr (!BIG && OP == kOpLess && KeyT<K>::kIntegral) {
    if (sg.cbits) {
      const uint16_t* g = w.lcell[level] + 2ull * sg.bbase;
      for (uint32_t i = threadIdx.x; i <= (1u << sg.cbits); i += blockDim.x) cell[i] = g[i];
    }
  }
}

// Bucket of a key at a narrow level: through the segment's key-cell table
// when it has one.
template <class K, int OP>
__device__ __forceinline__ uint32_t bucket_narrow(const K& k, const Seg& sg, const K* hk, const uint16_t* ht,
                                                  uint32_t tmask, const uint16_t* cell) {
  if constexpr (OP == kOpLess && KeyT<K>::kIntegral) {
    if (sg.cbits) return bucket_less_cells<K>(k, hk, ht, cell, sg.mult, sg.shift, sg.cbits);
  }
  return bucket_in<K, OP>(k, sg, hk, ht, tmask);
}

// U: keys in flight per thread -- 16 from the caller's key array (level 0),
// 4 from the temporaries' 16-byte records (deeper levels, where the smaller
// register footprint keeps four CTAs per SM), as measured.
template <class K, class V, int OP, bool BIG, int U>
__global__ void __launch_bounds__(kCountThreads) k_count(Work w, LevelBufs lb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CountSmem<K, OP, BIG>& cs = *reinterpret_cast<CountSmem<K, OP, BIG>*>(smem_raw);
  uint32_t* hist = cs.hist;
  K* hk = cs.hk;
  uint16_t* ht = cs.ht;
  unsigned long long* hsum = cs.hsum;
  const uint32_t nt = w.ctrl->ntiles[lb.level];
  for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
    const Tile tl = w.tiles[lb.level][t];
    const Seg sg = w.segs[lb.level][tl.seg];
    const uint32_t nl = sg.nl;
    const uint32_t nb = sg.nb;
    const uint32_t tmask = 4 * seg_hcap<OP>(sg) - 1;
    load_heavy<K, OP>(w, lb.level, sg, hk, ht);
    uint64_t tkmin = 0;
    uint32_t tshift = 0;
    load_cells<BIG && OP == kOpLess>(w, cs.cell, &tkmin, &tshift);
    load_seg_cells<K, OP, BIG>(w, lb.level, sg, cs.cell);
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
    if (OP == kOpReduce)
      for (uint32_t b = threadIdx.x; b < sg.nh * 8; b += blockDim.x) hsum[b] = 0;
    __syncthreads();
    const uint32_t per = blockDim.x * U;
    for (uint32_t i0 = 0; i0 < tl.len; i0 += per) {
      K key[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t i = i0 + u * blockDim.x + threadIdx.x;
        if (i < tl.len) key[u] = load_key<K, V>(lb.src_k, lb.src_aos, tl.start + i);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t i = i0 + u * blockDim.x + threadIdx.x;
        if (i < tl.len) {
          uint32_t b;
          if constexpr (BIG && OP == kOpLess)
            b = bucket_less_tab<K>(key[u], hk, ht, cs.cell, tkmin, tshift);
          else
            b = bucket_narrow<K, OP>(key[u], sg, hk, ht, tmask, cs.cell);
          atomicAdd(&hist[b], 1u);
          if constexpr (OP == kOpReduce) {
            if (b >= nl) {
              uint64_t v;
              if (lb.src_aos)
                v = (uint64_t)reinterpret_cast<const RecT<K, uint64_t>*>(lb.src_k)[tl.start + i].v;
              else
                v = reinterpret_cast<const uint64_t*>(lb.src_v)[tl.start + i];
              atomicAdd(&hsum[(b - nl) * 8 + (threadIdx.x & 7)], (unsigned long long)v);
            }
          }
        }
      }
    }
    __syncthreads();
    uint32_t* C = w.C[lb.level] + sg.cbase;
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) C[(uint64_t)b * sg.ntiles + tl.idx] = hist[b];
    if (OP == kOpReduce) {
      uint64_t* HP = w.hpart[lb.level] + sg.cbase;
      for (uint32_t b = threadIdx.x; b < sg.nh; b += blockDim.x) {
        unsigned long long t = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) t += hsum[b * 8 + c];
        HP[(uint64_t)b * sg.ntiles + tl.idx] = t;
      }
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// scan: column-major prefix sum X of C (Sec. 3.2): within each bucket row an
// exclusive prefix over subarrays, then bucket offsets from the row totals.
// Also counts the finish items and next-level segments each segment will
// emit.  One CTA per segment.
// ----------------------------------------------------------------------------
// Items a bucket produces besides the refine windows: heavy buckets give a
// copy-back (records left in the temporary array) or a heavy output
// (collect-reduce / histogram); light buckets above alpha give a next-level
// segment.  Light buckets of at most alpha records are covered by windows.
template <int OP>
__device__ __forceinline__ void items_of_bucket(uint32_t b, uint32_t nl, uint32_t sz, uint32_t alpha, bool last,
                                                uint32_t hdst_id, uint32_t* nf, uint32_t* nx) {
  *nf = 0;
  *nx = 0;
  if (!sz) return;
  if (is_heavy<OP>(b, nl)) {
    if (OP == kOpReduce || OP == kOpHist)
      *nf = 1;
    else if (hdst_id != kBufOut)
      *nf = (sz + kCopyChunk - 1) / kCopyChunk;
  } else if (sz > alpha && !last) {
    *nx = 1;
  }
}

// Refine windows of one segment: runs of adjacent light buckets of at most
// alpha records each, merged greedily in bucket order while the run stays
// within alpha records.  Equal keys never straddle buckets, so refining a
// window is the same as refining each of its buckets (Sec. 3.3) one after
// the other; for semisort_< the buckets are key ranges in increasing order, so
// sorting a window is the same as sorting its buckets in turn.  A non-empty
// heavy bucket ends the current window (its records sit between light ones in
// the semisort_< layout).  Run by one thread; writes the items when `items`
// is non-null.
template <int OP>
__device__ __forceinline__ uint32_t refine_windows(const uint32_t* bsize, const uint32_t* boff, uint32_t nl,
                                                   uint32_t nb, uint32_t alpha, bool last, uint64_t seg_start,
                                                   uint32_t buf, int level, Item* items, uint32_t first,
                                                   uint32_t cap) {
  uint32_t cnt = 0, wstart = 0, wlen = 0;
  bool open = false;
  auto flush = [&]() {
    if (items && first + cnt < cap) {
      Item it;
      it.start = seg_start + wstart;
      it.len = wlen;
      it.kind = kItemRefine;
      it.buf = buf;
      it.aux = it.aux2 = 0;
      it.level = level;
      items[first + cnt] = it;
    }
    ++cnt;
    open = false;
  };
  for (uint32_t b = 0; b < nb; ++b) {
    const uint32_t sz = bsize[b];
    if (sz == 0) continue;
    if (is_heavy<OP>(b, nl)) {
      if (open) flush();
      continue;
    }
    if (sz > alpha) {
      if (open) flush();
      if (last) {  // no level left: an oversized base case (reported as a depth error)
        wstart = boff[b];
        wlen = sz;
        flush();
      }
      continue;
    }
    if (open && wlen + sz > alpha) flush();
    if (!open) {
      wstart = boff[b];
      wlen = 0;
      open = true;
    }
    wlen += sz;
  }
  if (open) flush();
  return cnt;
}

template <int OP>
__global__ void __launch_bounds__(1024) k_scan(Work w, LevelBufs lb) {
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t carry;
  __shared__ uint32_t szs[OP == kOpLess ? kBigBuckets : kMaxBuckets];  // bucket sizes
  const uint32_t ns = w.ctrl->nsegs[lb.level];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const bool last_level = lb.level == kMaxLevels - 1;
  for (uint32_t s = blockIdx.x; s < ns; s += gridDim.x) {
    const Seg sg = w.segs[lb.level][s];
    if (sg.lbits == 0) {
      if (threadIdx.x == 0) {
        w.segs[lb.level][s].cnt_fin = 0;
        w.segs[lb.level][s].cnt_next = 0;
      }
      continue;
    }
    const uint32_t nl = sg.nl;
    const uint32_t nb = sg.nb;
    uint32_t* C = w.C[lb.level] + sg.cbase;
    uint32_t* bsize = w.bsize[lb.level] + sg.bbase;
    uint32_t* boff = w.boff[lb.level] + sg.bbase;
    for (uint32_t b = wid; b < nb; b += nw) {
      uint32_t* row = C + (uint64_t)b * sg.ntiles;
      uint32_t run = 0;
      for (uint32_t i0 = 0; i0 < sg.ntiles; i0 += 32) {
        const uint32_t i = i0 + lane;
        const uint32_t v = i < sg.ntiles ? row[i] : 0;
        const uint32_t inc = warp_inclusive_scan(v);
        if (i < sg.ntiles) row[i] = run + inc - v;
        run += __shfl_sync(kFull, inc, 31);
      }
      if (lane == 0) {
        bsize[b] = run;
        szs[b] = run;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    uint32_t nfin = 0, nnext = 0, lmax = 0;
    for (uint32_t b0 = 0; b0 < nb; b0 += blockDim.x) {
      const uint32_t b = b0 + threadIdx.x;
      const uint32_t sz = b < nb ? bsize[b] : 0;
      const bool heavy = is_heavy<OP>(b, nl);
      if (!heavy && sz > lmax) lmax = sz;
      // Collect-reduce and histogram never move heavy records (Sec. 3.5).
      const uint32_t lay = (heavy && (OP == kOpReduce || OP == kOpHist)) ? 0 : sz;
      uint32_t tot;
      const uint32_t ex = block_exclusive_scan(lay, tmp, &tot);
      if (b < nb) boff[b] = carry + ex;
      __syncthreads();
      if (threadIdx.x == 0) carry += tot;
      __syncthreads();
      if (b < nb) {
        uint32_t f, x;
        items_of_bucket<OP>(b, nl, sz, w.alpha, last_level, lb.hdst_id, &f, &x);
        nfin += f;
        nnext += x;
      }
    }
    const uint32_t tf = block_reduce_sum(nfin, tmp);
    const uint32_t tn = block_reduce_sum(nnext, tmp);
    if (lb.level == 0) atomicMax((unsigned long long*)&w.ctrl->stats[13], (unsigned long long)lmax);
    if (threadIdx.x == 0) {
      const uint32_t nw = refine_windows<OP>(szs, boff, nl, nb, w.alpha, last_level, sg.start, lb.dst_id,
                                             lb.level, nullptr, 0, 0);
      w.segs[lb.level][s].cnt_fin = tf + nw;
      w.segs[lb.level][s].cnt_next = tn;
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// distribute: the second pass of Blocked Distributing (Sec. 3.2).  Each CTA
// walks its subarray chunk by chunk in input order.  A chunk of records is
// copied once, coalesced, into a swizzled shared buffer; every thread then
// takes 16 consecutive records from it, computes their buckets and ranks them
// stably by bucket id (BlockRank, two 5-bit passes, no atomics).  The output
// pass walks the chunk in rank order, so each bucket's records leave as one
// contiguous run at X[bucket][subarray] + (records of that bucket already
// written): stable, and no two CTAs ever write the same slot (race-free).
// Light records go to the level's temporary array (records), heavy records
// straight to their final place.
//
// Latency hiding: the chunk after the current one is prefetched into L2 when
// the current one starts, and its loads into registers are issued before the
// current chunk's output phase, so the copy into shared memory that follows
// waits for nothing.  Bucket runs of the ranked chunk are found in one pass
// in blocked order with a suffix minimum over threads (no per-record loop
// over neighbours).
// ----------------------------------------------------------------------------
constexpr int kDT = 256;
constexpr int kDR = 16;
constexpr int kDCH = kDT * kDR;  // 4096 records per chunk
using DRank = BlockRank<kDT, kDR, 5>;

template <class K, class V, bool BIG, int OP>
struct DistSmem {
  RecT<K, V> S[kDCH];                // the chunk, swizzled (sw)
  typename DRank::Smem rk;
  uint32_t px[kDCH + kDCH / 32];     // (bucket << 16 | chunk index) at rank, padded (bpad)
  uint32_t cur[Space<BIG>::kIds];    // next write offset per bucket within the segment
  K hk[Space<BIG>::kBnd];
  uint16_t ht[Space<BIG>::kTab];
  uint16_t cell[BIG ? kTopCells + 1 : OP == kOpLess ? kSegCells + 1 : 1];
};

// Record i of a level's source (caller SoA at level 0, AoS records after).
template <class K, class V>
__device__ __forceinline__ RecT<K, V> read_src(const LevelBufs& lb, uint64_t i) {
  RecT<K, V> r;
  if (lb.src_aos) {
    r = reinterpret_cast<const RecT<K, V>*>(lb.src_k)[i];
  } else {
    r.k = reinterpret_cast<const K*>(lb.src_k)[i];
    if constexpr (!std::is_same<V, void>::value) r.v = reinterpret_cast<const V*>(lb.src_v)[i];
  }
  return r;
}

// Coalesced copy of `len` records starting at global index g into S; eight
// independent loads per thread are in flight before the first store.
template <int NT, class K, class V, class Src, int PER = 16, int B = 8>
__device__ __forceinline__ void load_chunk(RecT<K, V>* S, uint32_t len, Src src) {
  using Rec = RecT<K, V>;
  for (uint32_t i0 = 0; i0 < len; i0 += B * NT) {
    Rec t[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const uint32_t i = i0 + u * NT + threadIdx.x;
      if (i < len) t[u] = src(i);
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const uint32_t i = i0 + u * NT + threadIdx.x;
      if (i < len) S[sw<sizeof(Rec), PER>(i)] = t[u];
    }
  }
}


// Asynchronous global -> shared copy of `bytes` (4, 8 or 16, both addresses
// aligned to it) that bypasses registers; async_wait() waits for all of the
// thread's copies (a barrier must follow before other threads read them).
template <int bytes>
__device__ __forceinline__ void async_copy(void* smem_dst, const void* gmem_src) {
  static_assert(bytes == 4 || bytes == 8 || bytes == 16, "cp.async size");
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem_dst);
  if constexpr (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem_src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sa), "l"(gmem_src), "n"(bytes) : "memory");
}
__device__ __forceinline__ void async_wait() {
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Hash-bucket ids of a thread's kDR records in one pass: every light bucket
// first (no branches), then the first heavy-table probe of every record as
// independent loads, then the rare longer probe chains.
template <class K, class V>
__device__ __forceinline__ void bucket_ids_hash(const RecT<K, V>* S, uint32_t c0t, uint32_t clen, const Seg& sg,
                                                const K* hk, const uint16_t* ht, uint32_t tmask,
                                                uint32_t (&bid)[kDR]) {
  constexpr int RB = sizeof(RecT<K, V>);
  K key[kDR];
  uint32_t slot[kDR];
  const bool ident = sg.ident != 0;
#pragma unroll
  for (int r = 0; r < kDR; ++r) {
    key[r] = S[sw<RB>(c0t + r)].k;
    const uint64_t f = fold_key<K>(key[r]);
    const uint64_t h = f * sg.mult;
    bid[r] = ident ? (sg.shift < 64 ? (uint32_t)(f >> sg.shift) & (sg.nl - 1) : 0u) : (uint32_t)__umul64hi(h, sg.nl);
    slot[r] = (uint32_t)(h >> 20) & tmask;
  }
  if (sg.nh) {
    uint32_t e[kDR];
#pragma unroll
    for (int r = 0; r < kDR; ++r) e[r] = ht[slot[r]];
#pragma unroll
    for (int r = 0; r < kDR; ++r) {
      uint32_t s = slot[r], x = e[r];
      while (x != 0xFFFFu) {
        if (KeyT<K>::eq(hk[x], key[r])) {
          bid[r] = sg.nl + x;
          break;
        }
        s = (s + 1) & tmask;
        x = ht[s];
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kDR; ++r)
    if (c0t + r >= clen) bid[r] = 0x7FFFu;
}

// L2 prefetch of records [start, start + len) of a level's source (one
// prefetch per 128-byte line, every address inside the range).
template <class K, class V>
__device__ __forceinline__ void prefetch_src(const LevelBufs& lb, uint64_t start, uint32_t len) {
  auto pf = [&](const void* p0, uint64_t bytes) {
    const char* p = reinterpret_cast<const char*>(p0);
    const uint32_t lines = (uint32_t)((bytes + 127) / 128);
    for (uint32_t l = threadIdx.x; l < lines; l += blockDim.x) {
      uint64_t off = (uint64_t)l * 128;
      if (off >= bytes) off = bytes - 1;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(p + off));
    }
  };
  if (len == 0) return;
  if (lb.src_aos) {
    pf(reinterpret_cast<const RecT<K, V>*>(lb.src_k) + start, (uint64_t)len * sizeof(RecT<K, V>));
  } else {
    pf(reinterpret_cast<const K*>(lb.src_k) + start, (uint64_t)len * sizeof(K));
    if constexpr (!std::is_same<V, void>::value)
      pf(reinterpret_cast<const V*>(lb.src_v) + start, (uint64_t)len * sizeof(V));
  }
}

template <class K, class V, int OP, bool BIG>
__global__ void __launch_bounds__(kDT, 2) k_distribute(Work w, LevelBufs lb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DistSmem<K, V, BIG, OP>& sm = *reinterpret_cast<DistSmem<K, V, BIG, OP>*>(smem_raw);
  using Rec = RecT<K, V>;
  constexpr int RB = sizeof(Rec);
  constexpr bool kVals = !std::is_same<V, void>::value;
  using VV = typename ValT<V>::type;
  // records per thread carried in registers from one chunk to the next
  constexpr int kPF = RB <= 16 ? kDR : kDR / 2;
  const uint32_t nt = w.ctrl->ntiles[lb.level];
  constexpr bool kMoveHeavy = (OP == kOpEqual || OP == kOpLess);
  Rec* dst = reinterpret_cast<Rec*>(lb.dst);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t c0t = tid * kDR;
  uint32_t t = blockIdx.x;
  if (t >= nt) return;

  // A chunk moves global -> registers (issue) -> shared memory (commit); the
  // issue of chunk c + 1 comes before chunk c's output phase, so its loads
  // are in flight while chunk c is written out.
  Rec R[kPF];
  auto issue = [&](uint64_t base, uint32_t len) {
#pragma unroll
    for (int u = 0; u < kPF; ++u) {
      const uint32_t i = u * kDT + tid;
      Rec v{};
      if (i < len) v = read_src<K, V>(lb, base + i);
      R[u] = v;
    }
  };
  auto commit = [&](uint64_t base, uint32_t len) {
#pragma unroll
    for (int u = 0; u < kPF; ++u) {
      const uint32_t i = u * kDT + tid;
      if (i < len) sm.S[sw<RB>(i)] = R[u];
    }
    for (uint32_t i = kPF * kDT + tid; i < len; i += kDT) sm.S[sw<RB>(i)] = read_src<K, V>(lb, base + i);
  };
  // the first non-empty tile at or after tile index u of this CTA's sequence
  auto first_chunk = [&](uint32_t u, uint64_t* base, uint32_t* len) {
    *base = 0;
    *len = 0;
    for (; u < nt; u += gridDim.x) {
      const Tile tu = w.tiles[lb.level][u];
      if (tu.len) {
        *base = tu.start;
        *len = tu.len < (uint32_t)kDCH ? tu.len : (uint32_t)kDCH;
        return;
      }
    }
  };
  {
    uint64_t b0;
    uint32_t l0;
    first_chunk(t, &b0, &l0);
    issue(b0, l0);
    commit(b0, l0);
  }
  for (; t < nt; t += gridDim.x) {
    const Tile tl = w.tiles[lb.level][t];
    const Seg sg = w.segs[lb.level][tl.seg];
    const uint32_t nl = sg.nl;
    const uint32_t nb = sg.nb;
    const uint32_t tmask = 4 * seg_hcap<OP>(sg) - 1;
    load_heavy<K, OP>(w, lb.level, sg, sm.hk, sm.ht);
    uint64_t tkmin = 0;
    uint32_t tshift = 0;
    load_cells<BIG && OP == kOpLess>(w, sm.cell, &tkmin, &tshift);
    load_seg_cells<K, OP, BIG>(w, lb.level, sg, sm.cell);
    {
      const uint32_t* X = w.C[lb.level] + sg.cbase;
      const uint32_t* boff = w.boff[lb.level] + sg.bbase;
      for (uint32_t b = tid; b < nb; b += kDT) sm.cur[b] = boff[b] + X[(uint64_t)b * sg.ntiles + tl.idx];
    }
    const int passes = nb > 1024 ? 3 : nb > 32 ? 2 : 1;
    for (uint32_t c0 = 0; c0 < tl.len; c0 += kDCH) {
      const uint32_t clen = tl.len - c0 < (uint32_t)kDCH ? tl.len - c0 : (uint32_t)kDCH;
      // the chunk that follows this one: the tile's next chunk, or the first
      // chunk of this CTA's next tile
      uint64_t nbase = 0;
      uint32_t nlen = 0;
      if (c0 + kDCH < tl.len) {
        nbase = tl.start + c0 + kDCH;
        nlen = tl.len - (c0 + kDCH) < (uint32_t)kDCH ? tl.len - (c0 + kDCH) : (uint32_t)kDCH;
      } else {
        first_chunk(t + gridDim.x, &nbase, &nlen);
      }
      __syncthreads();  // the chunk is in S; tables and cursors are loaded
      prefetch_src<K, V>(lb, nbase, nlen);
      uint32_t bid[kDR], rk[kDR];
      // invalid slots get id 2^15 - 1: every 5-bit digit is 31, and as the last
      // items in blocked order they rank after every valid record
      if constexpr (OP != kOpLess && sizeof(K) <= 8) {
        bucket_ids_hash<K, V>(sm.S, c0t, clen, sg, sm.hk, sm.ht, tmask, bid);
      } else {
#pragma unroll
        for (int r = 0; r < kDR; ++r) {
          if (c0t + r >= clen) {
            bid[r] = 0x7FFFu;
          } else if constexpr (BIG) {
            bid[r] = bucket_less_tab<K>(sm.S[sw<RB>(c0t + r)].k, sm.hk, sm.ht, sm.cell, tkmin, tshift);
          } else {
            bid[r] = bucket_narrow<K, OP>(sm.S[sw<RB>(c0t + r)].k, sg, sm.hk, sm.ht, tmask, sm.cell);
          }
        }
      }
      DRank::rank(sm.rk, bid, 0, rk);
#pragma unroll
      for (int r = 0; r < kDR; ++r) sm.px[bpad(rk[r])] = (bid[r] << 16) | (c0t + r);
      // further passes as straight-line code with constant digit positions
      // (a loop over passes would keep the arrays in local memory)
      auto pass = [&](int shift) {
        __syncthreads();
        uint32_t x[kDR];
#pragma unroll
        for (int r = 0; r < kDR; ++r) x[r] = sm.px[bpad(c0t + r)];
        DRank::rank(sm.rk, x, shift, rk);
#pragma unroll
        for (int r = 0; r < kDR; ++r) sm.px[bpad(rk[r])] = x[r];
      };
      if (passes > 1) pass(21);
      if (BIG && passes > 2) pass(26);
      __syncthreads();
      // Bucket runs of the ranked chunk, found in blocked order: thread t
      // looks at sorted positions c0t .. c0t + 15.  smask marks run starts,
      // emask run starts and the chunk end (clen).  A run ends at the next
      // marked position: in this thread's range, else the first marked
      // position of a later thread (a suffix minimum over threads).
      uint32_t smask = 0, emask = 0, fb = 0xFFFFu;
      {
        uint32_t prev = c0t > 0 ? sm.px[bpad(c0t - 1)] >> 16 : 0xFFFFFFFFu;
#pragma unroll
        for (int r = 0; r < kDR; ++r) {
          const uint32_t p = c0t + r;
          const uint32_t b = sm.px[bpad(p)] >> 16;
          const bool st = p < clen && b != prev;
          const bool en = st || p == clen;
          smask |= st ? 1u << r : 0u;
          emask |= en ? 1u << r : 0u;
          prev = b;
        }
        if (emask) fb = c0t + (__ffs(emask) - 1);
      }
      uint32_t nf;  // first marked position of the threads after this one
      {
        uint32_t v = fb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t u = __shfl_down_sync(kFull, v, o);
          if (lane + o < 32) v = u < v ? u : v;
        }
        const uint32_t after = __shfl_down_sync(kFull, v, 1);
        if (lane == 0) sm.rk.scan_tmp[wid] = v;
        __syncthreads();
        nf = lane < 31 ? after : 0xFFFFu;
        for (int j = wid + 1; j < kDT / 32; ++j) {
          const uint32_t y = sm.rk.scan_tmp[j];
          nf = y < nf ? y : nf;
        }
        if (nf > clen) nf = clen;  // a full chunk's end lies past every thread's range
      }
      // run starts: turn the bucket's running offset into the base of this chunk
      for (uint32_t m = smask; m; m &= m - 1) {
        const int r = __ffs(m) - 1;
        const uint32_t p = c0t + r;
        sm.cur[sm.px[bpad(p)] >> 16] -= p;
      }
      __syncthreads();
      // the next chunk's loads are in flight during the output phase
      issue(nbase, nlen);
      for (uint32_t p = tid; p < clen; p += kDT) {
        const uint32_t x = sm.px[bpad(p)];
        const uint32_t b = x >> 16;
        const uint64_t pos = sg.start + sm.cur[b] + p;
        const Rec rec = sm.S[sw<RB>(x & 0xFFFFu)];
        if (!is_heavy<OP>(b, nl)) {
          if (lb.dst_aos) {
            dst[pos] = rec;
          } else {
            reinterpret_cast<K*>(lb.dst)[pos] = rec.k;
            if constexpr (kVals) reinterpret_cast<VV*>(lb.dst_v)[pos] = rec.v;
          }
        } else if constexpr (kMoveHeavy) {
          if (lb.hdst_aos) {
            reinterpret_cast<Rec*>(lb.hdst_k)[pos] = rec;
          } else {
            reinterpret_cast<K*>(lb.hdst_k)[pos] = rec.k;
            if constexpr (kVals) reinterpret_cast<VV*>(lb.hdst_v)[pos] = rec.v;
          }
        }
      }
      __syncthreads();
      // run ends: the next chunk continues after this chunk's run
      for (uint32_t m = smask; m; m &= m - 1) {
        const int r = __ffs(m) - 1;
        const uint32_t p = c0t + r;
        const uint32_t later = emask >> r >> 1;
        const uint32_t e = later ? p + __ffs(later) : nf;
        sm.cur[sm.px[bpad(p)] >> 16] += e;
      }
      commit(nbase, nlen);
    }
    __syncthreads();  // cursors of this tile are final before the next tile's
  }
}

// ----------------------------------------------------------------------------
// scan_items: one CTA.  Exclusive scans over the segments' item counts give
// every segment its slice of the finish list and of the next level.
// ----------------------------------------------------------------------------
static __global__ void __launch_bounds__(1024) k_scan_items(Work w, int level) {
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t carry[2];
  const uint32_t ns = w.ctrl->nsegs[level];
  if (ns == 0) return;
  if (threadIdx.x == 0) {
    carry[0] = w.ctrl->nfin;
    carry[1] = 0;
  }
  __syncthreads();
  Seg* segs = w.segs[level];
  for (uint32_t b0 = 0; b0 < ns; b0 += blockDim.x) {
    const uint32_t s = b0 + threadIdx.x;
    const uint32_t f = s < ns ? segs[s].cnt_fin : 0;
    const uint32_t x = s < ns ? segs[s].cnt_next : 0;
    uint32_t tf, tx;
    const uint32_t ef = block_exclusive_scan(f, tmp, &tf);
    const uint32_t ex = block_exclusive_scan(x, tmp, &tx);
    if (s < ns) {
      segs[s].fin_off = carry[0] + ef;
      segs[s].next_off = carry[1] + ex;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry[0] += tf;
      carry[1] += tx;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (carry[0] > w.item_cap) set_error(w.ctrl, 4);
    w.ctrl->nfin = carry[0] < w.item_cap ? carry[0] : w.item_cap;
    if (level + 1 < kMaxLevels) {
      const uint32_t cap = w.seg_cap[level + 1];
      if (carry[1] > cap) set_error(w.ctrl, 4);
      w.ctrl->nsegs[level + 1] = carry[1] < cap ? carry[1] : cap;
    }
  }
}

// ----------------------------------------------------------------------------
// emit: write the finish items (base cases, copy-backs, heavy outputs) and
// the next level's segments, in bucket order.  One CTA per segment.
// ----------------------------------------------------------------------------
template <int OP>
__global__ void __launch_bounds__(1024) k_emit(Work w, LevelBufs lb) {
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t carry[2];
  __shared__ uint32_t szs[OP == kOpLess ? kBigBuckets : kMaxBuckets];  // bucket sizes
  const uint32_t ns = w.ctrl->nsegs[lb.level];
  const bool last_level = lb.level == kMaxLevels - 1;
  for (uint32_t s = blockIdx.x; s < ns; s += gridDim.x) {
    const Seg sg = w.segs[lb.level][s];
    if (sg.lbits == 0) continue;
    const uint32_t nl = sg.nl;
    const uint32_t nb = sg.nb;
    const uint32_t* bsize = w.bsize[lb.level] + sg.bbase;
    const uint32_t* boff = w.boff[lb.level] + sg.bbase;
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) szs[b] = bsize[b];
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t nw = refine_windows<OP>(szs, boff, nl, nb, w.alpha, last_level, sg.start, lb.dst_id,
                                             lb.level, w.items, sg.fin_off, w.item_cap);
      for (uint32_t b = 0; b < nb; ++b)
        if (!is_heavy<OP>(b, nl) && szs[b] > w.alpha && last_level) set_error(w.ctrl, 8 /*SS_ERR_DEPTH*/);
      carry[0] = sg.fin_off + nw;
      carry[1] = sg.next_off;
    }
    __syncthreads();
    for (uint32_t b0 = 0; b0 < nb; b0 += blockDim.x) {
      const uint32_t b = b0 + threadIdx.x;
      const uint32_t sz = b < nb ? bsize[b] : 0;
      const bool heavy = is_heavy<OP>(b, nl);
      uint32_t nf = 0, nx = 0;
      if (b < nb) items_of_bucket<OP>(b, nl, sz, w.alpha, last_level, lb.hdst_id, &nf, &nx);
      uint32_t tf, tx;
      const uint32_t ef = block_exclusive_scan(nf, tmp, &tf);
      const uint32_t ex = block_exclusive_scan(nx, tmp, &tx);
      const uint64_t start = sg.start + (b < nb ? boff[b] : 0);
      if (nf) {
        const uint32_t i0 = carry[0] + ef;
        if (heavy && (OP == kOpReduce || OP == kOpHist)) {
          if (i0 < w.item_cap) {
            Item it;
            it.start = sg.start;  // (locates the instance of a batched call)
            it.len = sz;
            it.kind = kItemHeavyOut;
            it.buf = 0;
            it.aux = s;
            it.aux2 = b - nl;
            it.level = lb.level;
            w.items[i0] = it;
          }
        } else if (heavy) {
          for (uint32_t c = 0; c < nf; ++c) {
            if (i0 + c >= w.item_cap) break;
            Item it;
            it.start = start + (uint64_t)c * kCopyChunk;
            const uint32_t rem = sz - c * kCopyChunk;
            it.len = rem < kCopyChunk ? rem : kCopyChunk;
            it.kind = kItemCopy;
            it.buf = lb.hdst_id;
            it.aux = it.aux2 = 0;
            it.level = lb.level;
            w.items[i0 + c] = it;
          }
        }
      }
      if (nx && lb.level + 1 < kMaxLevels) {
        const uint32_t j = carry[1] + ex;
        if (j < w.seg_cap[lb.level + 1]) {
          Seg ns2 = {};
          ns2.start = start;
          ns2.len = sz;
          ns2.shift = sg.shift + sg.lbits;
          ns2.ident = sg.ident;
          w.segs[lb.level + 1][j] = ns2;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        carry[0] += tf;
        carry[1] += tx;
      }
      __syncthreads();
    }
  }
}

// ----------------------------------------------------------------------------
// finish (semisort_=): the base case of Sec. 3.3 for every light bucket of at
// most alpha records, and the copy-back of Sec. 3.4 for heavy buckets left in
// the temporary array.
//
// Base case: the window's records are copied once, coalesced, into a swizzled
// shared buffer.  Rounds of minimum reductions into a shared-memory hash table
// give every record the index of its key's first occurrence in the window
// (first_occurrences; the label does not depend on scheduling).  A scan over first occurrences turns
// labels into group ids 0..G-1 in first-occurrence order; ranking the records
// stably by group id (BlockRank, ceil(log2 G)/5 passes) puts every group in one
// run, groups in first-occurrence order and records of a group in input order
// -- the same result as the chained hash table of Sec. 3.3.  The output is
// written in rank order, coalesced, from the shared buffer.
// ----------------------------------------------------------------------------
constexpr int kRT = 256;
constexpr int kRR = 16;
constexpr int kRefMax = kRT * kRR;  // alpha upper bound (4096)
using RRank = BlockRank<kRT, kRR, 5>;

// First occurrences in a base-case window (the grouping step of the semisort_=
// and collect-reduce base cases, Sec. 3.3 and Sec. 3.5): for every record c
// of the window the smallest index o with key(o) == key(c).
//
// Rounds of minimum reductions into a shared-memory table of 2^tbits words
// (all kEmpty on entry, left dirty): in round k every record without a label
// reduces (tag_k << 12 | c) into the slot of its key under the round's hash;
// after a barrier the slot holds the smallest index o among the records that
// met there.  All records of one key meet in the same slot, so a record whose
// key equals key(o) takes o as its label (its key's first occurrence); the
// others move on to the next round's hash.  Tags fall from round to round, so
// values a slot kept from earlier rounds lose every minimum and the table is
// never cleared.  Every round settles at least the key of each slot used, so
// the rounds end.  No record waits on another record's result inside a
// round, which keeps the shared-memory atomics pipelined.
//
// Records are held kRR per thread in blocked order (c = c0t + r).  keyat(c)
// reads the key of record c; lab(r, o) receives the label of each valid
// record.  Contains barriers: every thread of the block calls it.
__device__ __forceinline__ uint64_t round_mult(uint64_t salt, uint32_t round) {
  return (salt | 1) * (0x9E3779B97F4A7C15ull * (2ull * round + 1) | 1);
}
template <class K, class KeyAt, class Lab>
__device__ __forceinline__ void first_occurrences(uint32_t* table, uint32_t tbits, uint32_t m, uint32_t c0t,
                                                  uint64_t salt, KeyAt keyat, Lab lab) {
  auto slot = [&](const K& key, uint64_t mul) { return (uint32_t)((fold_key<K>(key) * mul) >> (64 - tbits)); };
  uint32_t pend = 0;  // bit r: record c0t + r has no label yet
#pragma unroll
  for (int r = 0; r < kRR; ++r) pend |= (c0t + r < m) ? 1u << r : 0u;
  for (uint32_t round = 0;; ++round) {
    const uint64_t mul = round_mult(salt, round);
    const uint32_t tag = (0xFFFFEu - round) << 12;  // below kEmpty for every round and index
#pragma unroll
    for (int r = 0; r < kRR; ++r)
      if (pend >> r & 1u) atomicMin(&table[slot(keyat(c0t + r), mul)], tag | (c0t + r));
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRR; ++r) {
      if (pend >> r & 1u) {
        const K key = keyat(c0t + r);
        const uint32_t o = table[slot(key, mul)] & 0xFFFu;
        if (KeyT<K>::eq(keyat(o), key)) {
          lab(r, o);
          pend &= ~(1u << r);
        }
      }
    }
    if (!__syncthreads_or(pend != 0)) break;
  }
}

template <class K, class V>
struct RefSmem {
  RecT<K, V> S[kRefMax];  // the window, swizzled (sw)
  union {
    uint32_t table[2 * kRefMax];
    typename RRank::Smem rk;
  } u;
  uint32_t px[kRefMax + kRefMax / 32];  // group id by first occurrence; then (group << 16 | index) at rank
  uint32_t scan_tmp[33];
};

// Read record c of an item: AoS temporary, or the caller's SoA input.
template <class K, class V>
__device__ __forceinline__ RecT<K, V> load_rec(const Work& w, uint32_t buf, uint64_t c) {
  RecT<K, V> r;
  if (buf == kBufIn) {
    r.k = reinterpret_cast<const K*>(w.in_k)[c];
    if constexpr (!std::is_same<V, void>::value) r.v = reinterpret_cast<const V*>(w.in_v)[c];
  } else if (buf == kBufOut) {  // records a level left in the caller's output (Sec. 3.4)
    r.k = reinterpret_cast<const K*>(w.out_k)[c];
    if constexpr (!std::is_same<V, void>::value) r.v = reinterpret_cast<const V*>(w.out_v)[c];
  } else {
    r = reinterpret_cast<const RecT<K, V>*>(buf_ptr(w, buf))[c];
  }
  return r;
}

template <class K, class V>
__device__ __forceinline__ void store_out(const Work& w, uint64_t pos, const RecT<K, V>& r) {
  reinterpret_cast<K*>(w.out_k)[pos] = r.k;
  if constexpr (!std::is_same<V, void>::value) reinterpret_cast<V*>(w.out_v)[pos] = r.v;
}

// Copy-back of Sec. 3.4: records of an item from the temporary array to the
// output, eight independent loads per thread in flight.
template <int NT, class K, class V>
__device__ __forceinline__ void copy_item(const Work& w, const Item& it) {
  constexpr int B = 2;
  for (uint32_t i0 = 0; i0 < it.len; i0 += B * NT) {
    RecT<K, V> t[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const uint32_t i = i0 + u * NT + threadIdx.x;
      if (i < it.len) t[u] = load_rec<K, V>(w, it.buf, it.start + i);
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const uint32_t i = i0 + u * NT + threadIdx.x;
      if (i < it.len) store_out<K, V>(w, it.start + i, t[u]);
    }
  }
}

// Stable rank of the window's items by bits [16, 16 + 5 passes) of g[] (at
// most three passes): (id << 16 | index) ends up at rank in px.  The passes
// are straight-line code with constant digit positions; a loop over a runtime
// pass count keeps g[] and the rank's arrays in local memory.
__device__ __forceinline__ void rank_window(typename RRank::Smem& rs, uint32_t* px, const uint32_t (&g)[kRR],
                                            uint32_t passes, uint32_t c0t) {
  {
    uint32_t rk[kRR];
    RRank::rank(rs, g, 16, rk);
#pragma unroll
    for (int r = 0; r < kRR; ++r) px[bpad(rk[r])] = g[r];
  }
  auto pass = [&](int shift) {
    __syncthreads();
    uint32_t x[kRR], rk[kRR];
#pragma unroll
    for (int r = 0; r < kRR; ++r) x[r] = px[bpad(c0t + r)];
    RRank::rank(rs, x, shift, rk);
#pragma unroll
    for (int r = 0; r < kRR; ++r) px[bpad(rk[r])] = x[r];
  };
  if (passes > 1) pass(21);
  if (passes > 2) pass(26);
  __syncthreads();
}

// A base-case window into the swizzled shared buffer: records of a
// temporary array (16-byte records) by asynchronous copies, all of a thread's
// copies in flight at once; other windows through registers.
template <class K, class V>
__device__ __forceinline__ void load_window(RecT<K, V>* S, const Work& w, const Item& it) {
  using Rec = RecT<K, V>;
  constexpr int RB = sizeof(Rec);
  if (RB == 16 && it.buf != kBufIn && it.buf != kBufOut) {
    const Rec* src = reinterpret_cast<const Rec*>(buf_ptr(w, it.buf)) + it.start;
    for (uint32_t i = threadIdx.x; i < it.len; i += blockDim.x) async_copy<16>(&S[sw<RB>(i)], src + i);
    async_wait();
  } else {
    auto ld = [&](uint32_t i) { return load_rec<K, V>(w, it.buf, it.start + i); };
    load_chunk<kRT, K, V, decltype(ld), 16, 4>(S, it.len, ld);
  }
}

// L2 prefetch of a refine window's records.
template <class K, class V>
__device__ __forceinline__ void prefetch_item(const Work& w, const Item& it) {
  auto pf = [&](const void* p0, uint64_t bytes) {
    const char* p = reinterpret_cast<const char*>(p0);
    const uint32_t lines = (uint32_t)((bytes + 127) / 128);
    for (uint32_t l = threadIdx.x; l < lines; l += blockDim.x) {
      uint64_t off = (uint64_t)l * 128;
      if (off >= bytes) off = bytes - 1;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(p + off));
    }
  };
  if (it.len == 0) return;
  if (it.buf == kBufIn || it.buf == kBufOut) {
    const void* kp = it.buf == kBufIn ? w.in_k : w.out_k;
    const void* vp = it.buf == kBufIn ? w.in_v : w.out_v;
    pf(reinterpret_cast<const K*>(kp) + it.start, (uint64_t)it.len * sizeof(K));
    if constexpr (!std::is_same<V, void>::value)
      pf(reinterpret_cast<const V*>(vp) + it.start, (uint64_t)it.len * sizeof(V));
  } else {
    pf(reinterpret_cast<const RecT<K, V>*>(buf_ptr(w, it.buf)) + it.start, (uint64_t)it.len * sizeof(RecT<K, V>));
  }
}

// The refine window that follows item x in a CTA's sequence, if it is a
// base case (copy items are not prefetched).
__device__ __forceinline__ bool next_window(const Work& w, uint32_t x, uint32_t nfin, Item* out) {
  if (x >= nfin) return false;
  *out = w.items[x];
  return out->kind == kItemRefine && out->len <= (uint32_t)kRefMax;
}

template <class K, class V>
__global__ void __launch_bounds__(kRT, 2) k_finish_equal(Work w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RefSmem<K, V>& sm = *reinterpret_cast<RefSmem<K, V>*>(smem_raw);
  using Rec = RecT<K, V>;
  constexpr int RB = sizeof(Rec);
  const uint32_t nfin = w.ctrl->nfin;
  const int tid = threadIdx.x;
  const uint32_t c0t = tid * kRR;
  const uint64_t salt = refine_salt(w.seed);
  for (uint32_t itx = blockIdx.x; itx < nfin; itx += gridDim.x) {
    const Item it = w.items[itx];
    if (it.kind == kItemCopy) {
      copy_item<kRT, K, V>(w, it);
      if (tid == 0) atomicAdd((unsigned long long*)&w.ctrl->stats[6], (unsigned long long)it.len);
      continue;
    }
    const uint32_t m = it.len;
    if (m > (uint32_t)kRefMax) {
      if (tid == 0) set_error(w.ctrl, 8);
      continue;
    }
    Item nx;
    if (next_window(w, itx + gridDim.x, nfin, &nx)) prefetch_item<K, V>(w, nx);
    uint32_t ts = 64;
    while (ts < 2 * m) ts <<= 1;
    load_window<K, V>(sm.S, w, it);
    for (uint32_t i = tid; i < ts; i += kRT) sm.u.table[i] = kEmpty;
    __syncthreads();
    first_occurrences<K>(sm.u.table, 31 - __clz(ts), m, c0t, salt,
                         [&](uint32_t i) { return sm.S[sw<RB>(i)].k; },
                         [&](int r, uint32_t o) { sm.px[bpad(c0t + r)] = o; });
    // labels (first occurrences, in px) -> group ids in first-occurrence
    // order (kept per first occurrence in the table region)
    uint32_t nfirst = 0;
#pragma unroll
    for (int r = 0; r < kRR; ++r) {
      const uint32_t c = c0t + r;
      nfirst += (c < m && sm.px[bpad(c)] == c) ? 1u : 0u;
    }
    uint32_t G;
    uint32_t g0 = block_exclusive_scan(nfirst, sm.scan_tmp, &G);  // its barriers end the table reads
    if (tid == 0) {
      atomicAdd((unsigned long long*)&w.ctrl->stats[5], (unsigned long long)m);
      atomicAdd((unsigned long long*)&w.ctrl->stats[9], 1ull);
      atomicMax((unsigned long long*)&w.ctrl->stats[8], (unsigned long long)m);
    }
    if (G == m) {
      // every key distinct: the window is already semisorted
      if (tid == 0) atomicAdd((unsigned long long*)&w.ctrl->stats[10], (unsigned long long)m);
      for (uint32_t p = tid; p < m; p += kRT) store_out<K, V>(w, it.start + p, sm.S[sw<RB>(p)]);
      __syncthreads();
      continue;
    }
#pragma unroll
    for (int r = 0; r < kRR; ++r) {
      const uint32_t c = c0t + r;
      if (c < m && sm.px[bpad(c)] == c) sm.u.table[c] = g0++;
    }
    __syncthreads();
    // stable LSD ranking by group id, 5 bits per pass; padding items get
    // group 0xFFF and, last in blocked order, rank after every record
    uint32_t g[kRR];
#pragma unroll
    for (int r = 0; r < kRR; ++r) {
      const uint32_t c = c0t + r;
      g[r] = ((c < m ? sm.u.table[sm.px[bpad(c)]] : 0xFFFu) << 16) | c;
    }
    const uint32_t gbits = ceil_log2_u32(G) < 1 ? 1 : ceil_log2_u32(G);
    const uint32_t passes = (gbits + 4) / 5;
    __syncthreads();  // group ids read: px and the hash table region are free
    rank_window(sm.u.rk, sm.px, g, passes, c0t);
    for (uint32_t p = tid; p < m; p += kRT) store_out<K, V>(w, it.start + p, sm.S[sw<RB>(sm.px[bpad(p)] & 0xFFFFu)]);
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// finish (semisort_<): the base case of Sec. 3.3 with a sort by key, and the
// copy-backs of Sec. 3.4.  A window's records are staged once in shared
// memory.  For keys up to 8 bytes every record gets an interpolation bucket,
// the top 15 bits of (key - window minimum), a non-decreasing function of the
// key; a stable rank by it (at most three 5-bit passes) leaves the window
// ordered by bucket with input order inside each bucket.  Runs of equal
// buckets that hold an inversion are then ordered in parallel: every record
// counts the records of its run that precede it by (key, window index).
// Runs are short unless keys repeat (then they are already in order) or
// cluster; a window with an unordered run longer than 64 records -- and every
// window of 128-bit or user-defined keys -- is sorted instead by Batcher's
// bitonic network on (key, position in the window).  Either way the output
// is the stable sort of the window.
// ----------------------------------------------------------------------------
template <class K, class V>
struct LessSmem {
  RecT<K, V> S[kRefMax];  // the window, swizzled (sw)
  union {
    typename RRank::Smem rk;
    uint16_t idx[kRefMax];                 // bitonic: positions in the window
    uint32_t px2[kRefMax + kRefMax / 32];  // the final order, padded (bpad)
  } u;
  uint32_t px[kRefMax + kRefMax / 32];  // (bucket << 16 | index) at rank, padded (bpad)
  uint8_t runinv[kRefMax];              // per run start: the run holds an inversion
  uint32_t scan_tmp[33];
  unsigned long long mn[32], mx[32];
};

template <class K, class V>
__global__ void __launch_bounds__(kRT, 2) k_finish_less(Work w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LessSmem<K, V>& sm = *reinterpret_cast<LessSmem<K, V>*>(smem_raw);
  using Rec = RecT<K, V>;
  constexpr int RB = sizeof(Rec);
  const uint32_t nfin = w.ctrl->nfin;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t c0t = tid * kRR;
  for (uint32_t itx = blockIdx.x; itx < nfin; itx += gridDim.x) {
    const Item it = w.items[itx];
    if (it.kind == kItemCopy) {
      copy_item<kRT, K, V>(w, it);
      if (tid == 0) atomicAdd((unsigned long long*)&w.ctrl->stats[6], (unsigned long long)it.len);
      continue;
    }
    const uint32_t m = it.len;
    if (m > (uint32_t)kRefMax) {
      if (tid == 0) set_error(w.ctrl, 8);
      continue;
    }
    {
      Item nx;  // the next window streams into L2 while this one is sorted
      if (next_window(w, itx + gridDim.x, nfin, &nx)) prefetch_item<K, V>(w, nx);
    }
    load_window<K, V>(sm.S, w, it);
    if (tid == 0) {
      atomicAdd((unsigned long long*)&w.ctrl->stats[5], (unsigned long long)m);
      atomicAdd((unsigned long long*)&w.ctrl->stats[9], 1ull);
      atomicMax((unsigned long long*)&w.ctrl->stats[8], (unsigned long long)m);
    }
    __syncthreads();
    if constexpr (KeyT<K>::kIntegral) {
      // key range of the window
      unsigned long long lo = ~0ull, hi = 0;
#pragma unroll
      for (int r = 0; r < kRR; ++r) {
        if (c0t + r < m) {
          const unsigned long long k = (uint64_t)sm.S[sw<RB>(c0t + r)].k;
          lo = k < lo ? k : lo;
          hi = k > hi ? k : hi;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(kFull, lo, o), b = __shfl_xor_sync(kFull, hi, o);
        lo = a < lo ? a : lo;
        hi = b > hi ? b : hi;
      }
      if (lane == 0) {
        sm.mn[wid] = lo;
        sm.mx[wid] = hi;
      }
      __syncthreads();
      lo = ~0ull;
      hi = 0;
      for (int i = 0; i < kRT / 32; ++i) {
        lo = sm.mn[i] < lo ? sm.mn[i] : lo;
        hi = sm.mx[i] > hi ? sm.mx[i] : hi;
      }
      const uint64_t range = hi - lo;
      const uint32_t bits = range ? 64 - __clzll((long long)range) : 0;
      const uint32_t shift = bits > 15 ? bits - 15 : 0;
      const uint32_t nbits = bits - shift;  // bucket ids < 2^nbits <= 2^15
      if (nbits == 0) {
        // all keys equal: the window is already sorted
        for (uint32_t p = tid; p < m; p += kRT) store_out<K, V>(w, it.start + p, sm.S[sw<RB>(p)]);
        __syncthreads();
        continue;
      }
      uint32_t g[kRR];
#pragma unroll
      for (int r = 0; r < kRR; ++r) {
        const uint32_t c = c0t + r;
        const uint32_t ib = c < m ? (uint32_t)(((uint64_t)sm.S[sw<RB>(c)].k - lo) >> shift) : 0x7FFFu;
        g[r] = (ib << 16) | c;
      }
      rank_window(sm.u.rk, sm.px, g, (nbits + 4) / 5, c0t);
      // Runs of equal buckets are in window order.  With shift 0 a bucket
      // holds one key value and the rank is already the sort; otherwise find
      // the inversions (a key below its predecessor's in the same run), in
      // blocked order.
      auto key_at = [&](uint32_t x) { return sm.S[sw<RB>(x & 0xFFFFu)].k; };
      uint32_t headm = 0, invm = 0;
      if (shift > 0) {
        uint32_t pb = 0xFFFFFFFFu;
        K pk{};
        if (c0t > 0 && c0t - 1 < m) {
          const uint32_t x = sm.px[bpad(c0t - 1)];
          pb = x >> 16;
          pk = key_at(x);
        }
#pragma unroll
        for (int r = 0; r < kRR; ++r) {
          const uint32_t p = c0t + r;
          if (p < m) {
            const uint32_t x = sm.px[bpad(p)];
            const K k = key_at(x);
            const bool head = (x >> 16) != pb;
            headm |= head ? 1u << r : 0u;
            invm |= (!head && KeyT<K>::lt(k, pk)) ? 1u << r : 0u;
            pb = x >> 16;
            pk = k;
          }
        }
      }
      if (!__syncthreads_or(invm != 0)) {
        for (uint32_t p = tid; p < m; p += kRT)
          store_out<K, V>(w, it.start + p, sm.S[sw<RB>(sm.px[bpad(p)] & 0xFFFFu)]);
        __syncthreads();
        continue;
      }
      // Run bounds: the run of position p starts at the last head at or
      // before p and ends before the first head after p (block-wide max and
      // suffix-min scans over the threads' head positions).
      const uint32_t hfirst = headm ? c0t + __ffs(headm) - 1 : 0xFFFFFFFFu;
      const uint32_t hlast = headm ? c0t + 31 - __clz(headm) : 0u;
      uint32_t rs = block_exclusive_max(hlast, sm.scan_tmp);
      uint32_t nh = block_suffix_min(hfirst, sm.scan_tmp);
      nh = nh < m ? nh : m;
#pragma unroll
      for (int r = 0; r < kRR; ++r)
        if (headm >> r & 1u) sm.runinv[c0t + r] = 0;
      __syncthreads();
      uint32_t rsr[kRR];
#pragma unroll
      for (int r = 0; r < kRR; ++r) {
        if (headm >> r & 1u) rs = c0t + r;
        rsr[r] = rs;
        if (invm >> r & 1u) sm.runinv[rs] = 1;
      }
      __syncthreads();
      // Every record of a run with an inversion takes its place in the run
      // by (key, window index): the records of the run before it with a key
      // not above its own, and those after it with a smaller key, precede
      // it.  Runs longer than kRunMax go to the bitonic network instead.
      constexpr uint32_t kRunMax = 64;
      uint32_t longrun = 0;
      uint32_t re = nh;
#pragma unroll
      for (int r = kRR - 1; r >= 0; --r) {
        const uint32_t p = c0t + r;
        if (p >= m) continue;
        const uint32_t x = sm.px[bpad(p)];
        uint32_t pos = p;
        if (sm.runinv[rsr[r]]) {
          if (re - rsr[r] > kRunMax) {
            longrun = 1;
          } else {
            const K kp = key_at(x);
            pos = rsr[r];
            for (uint32_t q = rsr[r]; q < re; ++q) {
              if (q == p) continue;
              const K kq = key_at(sm.px[bpad(q)]);
              pos += q < p ? (KeyT<K>::lt(kp, kq) ? 0u : 1u) : (KeyT<K>::lt(kq, kp) ? 1u : 0u);
            }
          }
        }
        sm.u.px2[bpad(pos)] = x;
        if (headm >> r & 1u) re = p;
      }
      if (!__syncthreads_or(longrun)) {
        for (uint32_t p = tid; p < m; p += kRT)
          store_out<K, V>(w, it.start + p, sm.S[sw<RB>(sm.u.px2[bpad(p)] & 0xFFFFu)]);
        __syncthreads();
        continue;
      }
    }
    // bitonic network on (key, position), positions only move
    uint32_t P = 2;
    while (P < m) P <<= 1;
    for (uint32_t c = tid; c < P; c += kRT) sm.u.idx[c] = (uint16_t)c;  // positions >= m: padding, last
    __syncthreads();
    for (uint32_t k = 2; k <= P; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        for (uint32_t p = tid; p < P / 2; p += kRT) {
          const uint32_t i = ((p & ~(j - 1)) << 1) | (p & (j - 1));
          const uint32_t ixj = i + j;
          const uint32_t ia = sm.u.idx[i], ib = sm.u.idx[ixj];
          bool gt;  // (key, position) of slot i above that of slot i + j
          if (ia >= m || ib >= m) {
            gt = ia > ib;
          } else {
            const K ka = sm.S[sw<RB>(ia)].k, kb = sm.S[sw<RB>(ib)].k;
            gt = KeyT<K>::lt(kb, ka) || (KeyT<K>::eq(ka, kb) && ia > ib);
          }
          if (gt == ((i & k) == 0)) {
            sm.u.idx[i] = (uint16_t)ib;
            sm.u.idx[ixj] = (uint16_t)ia;
          }
        }
        __syncthreads();
      }
    }
    for (uint32_t p = tid; p < m; p += kRT) store_out<K, V>(w, it.start + p, sm.S[sw<RB>(sm.u.idx[p])]);
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// finish (collect-reduce, histogram; Sec. 3.5).  Refine windows: a shared-
// memory hash table finds each key's first occurrence (first_occurrences, as
// in the semisort_= base case); first occurrences numbered in
// window order give group ids, and the values (collect-reduce) or ones
// (histogram) are added per group.  The G distinct (key, sum) pairs are
// written compacted over the window's own first G slots (its records are no
// longer needed; the caller's input is never written, a window of it goes to
// T instead), histogram counts to the same positions of scratch32.  Heavy
// outputs: collect-reduce adds the per-subarray partial sums of the count
// pass, a histogram count is the heavy bucket's size.  item_out receives the
// number of outputs of each item; a scan and a pack kernel then place them.
// Unsigned wraparound addition is associative and commutative, so the sums do
// not depend on the order of the atomic adds.
// ----------------------------------------------------------------------------
template <class K>
struct RedSmem {
  K keys[kRefMax];
  uint32_t table[2 * kRefMax];
  unsigned long long acc[kRefMax];
  uint16_t gid[kRefMax];
  uint16_t fo[kRefMax];
  uint32_t scan_tmp[33];
  unsigned long long red[32];
};

__device__ __forceinline__ uint32_t compact_buf(uint32_t buf) { return buf == kBufIn ? (uint32_t)kBufT : buf; }

template <class K, class V, int OP>
__global__ void __launch_bounds__(kRT, 2) k_finish_reduce(Work w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RedSmem<K>& sm = *reinterpret_cast<RedSmem<K>*>(smem_raw);
  using Rec = RecT<K, V>;
  const uint32_t nfin = w.ctrl->nfin;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t c0t = tid * kRR;
  const uint64_t salt = refine_salt(w.seed);
  for (uint32_t itx = blockIdx.x; itx < nfin; itx += gridDim.x) {
    const Item it = w.items[itx];
    if (it.kind == kItemHeavyOut) {
      if constexpr (OP == kOpReduce) {
        const Seg sg = w.segs[it.level][it.aux];
        const uint64_t* HP = w.hpart[it.level] + sg.cbase + (uint64_t)it.aux2 * sg.ntiles;
        unsigned long long v = 0;
        for (uint32_t t = tid; t < sg.ntiles; t += kRT) v += HP[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (lane == 0) sm.red[wid] = v;
        __syncthreads();
        if (tid == 0) {
          unsigned long long t = 0;
          for (int i = 0; i < kRT / 32; ++i) t += sm.red[i];
          w.item_aux[itx] = t;
        }
        __syncthreads();
      }
      if (tid == 0) w.item_out[itx] = 1;
      continue;
    }
    const uint32_t m = it.len;
    if (m > (uint32_t)kRefMax) {
      if (tid == 0) {
        set_error(w.ctrl, 8);
        w.item_out[itx] = 0;
      }
      continue;
    }
    {
      Item nx;  // the next window streams into L2 while this one is reduced
      if (next_window(w, itx + gridDim.x, nfin, &nx)) prefetch_item<K, V>(w, nx);
    }
    uint32_t ts = 64;
    while (ts < 2 * m) ts <<= 1;
    if (sizeof(K) == 8 && it.buf != kBufIn) {
      // keys of a temporary array's records: asynchronous 8-byte copies
      const Rec* src = reinterpret_cast<const Rec*>(buf_ptr(w, it.buf)) + it.start;
      for (uint32_t c = tid; c < m; c += kRT) async_copy<8>(&sm.keys[c], &src[c].k);
      async_wait();
    } else {
      for (uint32_t c = tid; c < m; c += kRT)
        sm.keys[c] = it.buf == kBufIn ? reinterpret_cast<const K*>(w.in_k)[it.start + c]
                                      : reinterpret_cast<const Rec*>(buf_ptr(w, it.buf))[it.start + c].k;
    }
    for (uint32_t i = tid; i < ts; i += kRT) sm.table[i] = kEmpty;
    __syncthreads();
    uint32_t lab[kRR];
#pragma unroll
    for (int r = 0; r < kRR; ++r) lab[r] = 0;
    first_occurrences<K>(sm.table, 31 - __clz(ts), m, c0t, salt, [&](uint32_t i) { return sm.keys[i]; },
                         [&](int r, uint32_t o) { lab[r] = o; });
    uint32_t nfirst = 0;
#pragma unroll
    for (int r = 0; r < kRR; ++r) {
      const uint32_t c = c0t + r;
      nfirst += (c < m && lab[r] == c) ? 1u : 0u;
    }
    uint32_t G;
    uint32_t g0 = block_exclusive_scan(nfirst, sm.scan_tmp, &G);
    if (G == m) {
      // every key distinct: each record is its own group, and the compacted
      // window is the window itself -- already in place in a temporary
      // array; a window of the caller's input is copied to T
      if (it.buf == kBufIn) {
        Rec* cb = reinterpret_cast<Rec*>(buf_ptr(w, compact_buf(it.buf)));
        for (uint32_t c = tid; c < m; c += kRT) {
          Rec o;
          o.k = sm.keys[c];
          if constexpr (OP == kOpReduce) o.v = reinterpret_cast<const uint64_t*>(w.in_v)[it.start + c];
          cb[it.start + c] = o;
        }
      }
      if constexpr (OP == kOpHist)
        for (uint32_t c = tid; c < m; c += kRT) w.scratch32[it.start + c] = 1u;
      if (tid == 0) {
        w.item_out[itx] = G;
        atomicAdd((unsigned long long*)&w.ctrl->stats[5], (unsigned long long)m);
        atomicAdd((unsigned long long*)&w.ctrl->stats[9], 1ull);
        atomicMax((unsigned long long*)&w.ctrl->stats[8], (unsigned long long)m);
        atomicAdd((unsigned long long*)&w.ctrl->stats[10], (unsigned long long)m);
      }
      __syncthreads();
      continue;
    }
#pragma unroll
    for (int r = 0; r < kRR; ++r) {
      const uint32_t c = c0t + r;
      if (c < m && lab[r] == c) {
        sm.gid[c] = (uint16_t)g0;
        sm.fo[g0] = (uint16_t)c;
        sm.acc[g0] = 0;
        ++g0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRR; ++r) {
      const uint32_t c = c0t + r;
      if (c < m) {
        unsigned long long v = 1;
        if constexpr (OP == kOpReduce) {
          v = it.buf == kBufIn ? reinterpret_cast<const uint64_t*>(w.in_v)[it.start + c]
                               : (uint64_t)reinterpret_cast<const Rec*>(buf_ptr(w, it.buf))[it.start + c].v;
        }
        atomicAdd(&sm.acc[sm.gid[lab[r]]], v);
      }
    }
    __syncthreads();  // every record of the window has been read
    Rec* cb = reinterpret_cast<Rec*>(buf_ptr(w, compact_buf(it.buf)));
    for (uint32_t g = tid; g < G; g += kRT) {
      Rec o;
      o.k = sm.keys[sm.fo[g]];
      if constexpr (OP == kOpReduce) o.v = (uint64_t)sm.acc[g];
      cb[it.start + g] = o;
      if constexpr (OP == kOpHist) w.scratch32[it.start + g] = (uint32_t)sm.acc[g];
    }
    if (tid == 0) {
      w.item_out[itx] = G;
      atomicAdd((unsigned long long*)&w.ctrl->stats[5], (unsigned long long)m);
      atomicAdd((unsigned long long*)&w.ctrl->stats[9], 1ull);
      atomicMax((unsigned long long*)&w.ctrl->stats[8], (unsigned long long)m);
      if (G == m) atomicAdd((unsigned long long*)&w.ctrl->stats[10], (unsigned long long)m);
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// Output placement for collect-reduce / histogram (the packing step of
// Sec. 3.5): an exclusive scan of item_out in item order (three kernels:
// chunk totals, one-CTA scan of the totals, chunk-local scans), then a pack
// kernel that copies each item's outputs to the caller's arrays.  Item order
// is deterministic, so the output order is too.
// ----------------------------------------------------------------------------
constexpr uint32_t kScanChunk = 4096;  // items per CTA (1024 threads x 4)

static __global__ void __launch_bounds__(1024) k_iscan_a(Work w) {
  __shared__ uint64_t tmp[33];
  const uint32_t nfin = w.ctrl->nfin;
  const uint64_t c0 = (uint64_t)blockIdx.x * kScanChunk;
  if (c0 >= nfin) return;
  uint64_t s = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const uint64_t i = c0 + threadIdx.x * 4 + r;
    if (i < nfin) s += w.item_out[i];
  }
  uint64_t tot;
  block_exclusive_scan64(s, tmp, &tot);
  if (threadIdx.x == 0) w.block_sums[blockIdx.x] = tot;
}

static __global__ void __launch_bounds__(1024) k_iscan_b(Work w) {
  __shared__ uint64_t tmp[33];
  __shared__ uint64_t carry;
  const uint32_t nfin = w.ctrl->nfin;
  const uint32_t nch = (nfin + kScanChunk - 1) / kScanChunk;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t b0 = 0; b0 < nch; b0 += blockDim.x) {
    const uint32_t b = b0 + threadIdx.x;
    const uint64_t v = b < nch ? w.block_sums[b] : 0;
    uint64_t tot;
    const uint64_t ex = block_exclusive_scan64(v, tmp, &tot);
    if (b < nch) w.block_sums[b] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && w.offsets == nullptr) {
    *w.num_unique = carry;
    if (carry > w.out_capacity) set_error(w.ctrl, 4 /*SS_ERR_CAPACITY*/);
  }
}

static __global__ void __launch_bounds__(1024) k_iscan_c(Work w) {
  __shared__ uint64_t tmp[33];
  const uint32_t nfin = w.ctrl->nfin;
  const uint64_t c0 = (uint64_t)blockIdx.x * kScanChunk;
  if (c0 >= nfin) return;
  uint64_t v[4], s = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const uint64_t i = c0 + threadIdx.x * 4 + r;
    v[r] = i < nfin ? w.item_out[i] : 0;
    s += v[r];
  }
  uint64_t tot;
  uint64_t run = w.block_sums[blockIdx.x] + block_exclusive_scan64(s, tmp, &tot);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const uint64_t i = c0 + threadIdx.x * 4 + r;
    if (i < nfin) w.item_pos[i] = run;
    run += v[r];
  }
}

// Batched collect-reduce / histogram output placement.  Within each item
// class (base-case items of small instances, then the items of distribution
// levels 0..3, in the order the list holds them) the items are grouped by
// instance in instance order, so an instance's outputs in one class occupy one
// range of the item scan.  Per (class, instance): the outputs and the first
// scan position (order-independent atomics, so deterministic); then one scan
// over instances gives every instance its output offset and every (class,
// instance) its base: instance offset + outputs of earlier classes.
__device__ __forceinline__ uint32_t item_class(const Item& it) {
  return it.level == kDirectLevel ? 0u : it.level + 1u;
}
__device__ __forceinline__ uint32_t instance_of(const Work& w, uint64_t start) {
  uint32_t lo = 0, hi = w.num_inst;  // last instance whose first record <= start
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (w.offsets[mid] <= start)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

static __global__ void k_inst_reset(Work w) {
  const uint32_t m = kItemClasses * w.num_inst;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    w.inst_base[i] = 0;
    w.inst_first[i] = ~0ull;
  }
}

static __global__ void k_inst_accum(Work w) {
  const uint32_t nfin = w.ctrl->nfin;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nfin; i += gridDim.x * blockDim.x) {
    const Item it = w.items[i];
    const uint32_t k = item_class(it) * w.num_inst + instance_of(w, it.start);
    atomicAdd((unsigned long long*)&w.inst_base[k], (unsigned long long)w.item_out[i]);
    atomicMin((unsigned long long*)&w.inst_first[k], (unsigned long long)w.item_pos[i]);
  }
}

static __global__ void __launch_bounds__(1024) k_inst_scan(Work w) {
  __shared__ uint64_t tmp[33];
  __shared__ uint64_t carry;
  const uint32_t ni = w.num_inst;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t i0 = 0; i0 < ni; i0 += blockDim.x) {
    const uint32_t i = i0 + threadIdx.x;
    uint64_t u[kItemClasses], tot = 0;
#pragma unroll
    for (uint32_t c = 0; c < kItemClasses; ++c) {
      u[c] = i < ni ? w.inst_base[(uint64_t)c * ni + i] : 0;
      tot += u[c];
    }
    uint64_t all;
    const uint64_t ex = carry + block_exclusive_scan64(tot, tmp, &all);
    if (i < ni) {
      w.num_unique[i] = tot;
      w.inst_off_out[i] = ex;
      uint64_t b = ex;
#pragma unroll
      for (uint32_t c = 0; c < kItemClasses; ++c) {
        w.inst_base[(uint64_t)c * ni + i] = b;
        b += u[c];
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += all;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    w.inst_off_out[ni] = carry;
    if (carry > w.out_capacity) set_error(w.ctrl, 4 /*SS_ERR_CAPACITY*/);
  }
}

// One warp per item.  Outputs at positions >= capacity are not written.
template <class K, class V, int OP>
__global__ void __launch_bounds__(256) k_pack(Work w) {
  using Rec = RecT<K, V>;
  const uint32_t nfin = w.ctrl->nfin;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  K* uk = reinterpret_cast<K*>(w.out_k);
  const uint64_t cap = w.out_capacity;
  for (uint32_t itx = gw; itx < nfin; itx += nwarps) {
    const Item it = w.items[itx];
    uint64_t pos = w.item_pos[itx];
    if (w.offsets) {
      const uint32_t k = item_class(it) * w.num_inst + instance_of(w, it.start);
      pos = w.inst_base[k] + (pos - w.inst_first[k]);
    }
    if (it.kind == kItemHeavyOut) {
      if (lane == 0 && pos < cap) {
        const Seg sg = w.segs[it.level][it.aux];
        uk[pos] = reinterpret_cast<const K*>(w.hkeys[it.level])[sg.bbase + it.aux2];
        if constexpr (OP == kOpReduce)
          reinterpret_cast<uint64_t*>(w.sums_out)[pos] = w.item_aux[itx];
        else
          reinterpret_cast<uint32_t*>(w.sums_out)[pos] = it.len;
      }
      continue;
    }
    const uint32_t cnt = (uint32_t)w.item_out[itx];
    const Rec* cb = reinterpret_cast<const Rec*>(buf_ptr(w, compact_buf(it.buf)));
    for (uint32_t g = lane; g < cnt; g += 32) {
      if (pos + g >= cap) break;
      const Rec r = cb[it.start + g];
      uk[pos + g] = r.k;
      if constexpr (OP == kOpReduce)
        reinterpret_cast<uint64_t*>(w.sums_out)[pos + g] = (uint64_t)r.v;
      else
        reinterpret_cast<uint32_t*>(w.sums_out)[pos + g] = w.scratch32[it.start + g];
    }
  }
}

}  // namespace ss
