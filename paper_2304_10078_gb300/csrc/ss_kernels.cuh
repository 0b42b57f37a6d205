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
  const void* src_v;  // SoA values (level 0 only)
  void* dst;          // AoS records: light buckets
  void* hdst_k;       // heavy destination: SoA keys, or AoS records when hdst_aos
  void* hdst_v;
  uint32_t src_aos;
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

__host__ __device__ __forceinline__ uint32_t hcap_of(uint32_t lbits) {
  const uint32_t nl = 1u << lbits;
  return nl < kMaxHeavy ? nl : kMaxHeavy;
}

// Bucket of key k in its segment (GetBucketId of Algorithm 1): the heavy
// bucket n_L + i if k is the i-th heavy key, else the light bucket given by
// the top lbits bits of the level hash.  hk/ht: the segment's heavy keys and
// its open-addressing table (4 slots per heavy key, so probes stay short).
template <class K>
__device__ __forceinline__ uint32_t bucket_of(const K& k, uint64_t mult, uint32_t lbits, uint32_t nh,
                                              const K* hk, const uint16_t* ht, uint32_t tmask) {
  const uint64_t h = fold_key<K>(k) * mult;
  uint32_t b = (uint32_t)(h >> (64 - lbits));
  if (nh) {
    uint32_t slot = (uint32_t)(h >> 20) & tmask;
    uint32_t e = ht[slot];
    while (e != 0xFFFFu) {
      if (KeyT<K>::eq(hk[e], k)) {
        b = (1u << lbits) + e;
        break;
      }
      slot = (slot + 1) & tmask;
      e = ht[slot];
    }
  }
  return b;
}

// ----------------------------------------------------------------------------
// init: reset the control block and seed level 0 (or a single base case).
// ----------------------------------------------------------------------------
__global__ void k_init(Work w) {
  if (threadIdx.x != 0) return;
  Ctrl* c = w.ctrl;
  for (int l = 0; l < kMaxLevels; ++l) {
    c->nsegs[l] = 0;
    c->ntiles[l] = 0;
  }
  c->nfin = 0;
  c->error = 0;
  for (int i = 0; i < 16; ++i) c->stats[i] = 0;
  if (w.n == 0) return;
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
    w.segs[0][0] = s;
    c->nsegs[0] = 1;
  }
}

// ----------------------------------------------------------------------------
// plan: per segment of level `level`, pick n_L, cut it into subarrays, and
// lay out its rows of the count matrix.  One CTA.
// ----------------------------------------------------------------------------
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
      if (level == 0) {
        lb = w.lbits1;
      } else {
        const uint64_t want = (2ull * sg.len + w.alpha - 1) / w.alpha;
        lb = want <= 2 ? 1u : (uint32_t)(64 - __clzll(want - 1));
        lb = lb > (uint32_t)kMaxLightLog2 ? (uint32_t)kMaxLightLog2 : lb;
      }
      const uint32_t nl = 1u << lb;
      sg.lbits = lb;
      sg.nbcap = nl + hcap_of(lb);
      sg.nh = 0;
      sg.mult = seg_mult(w.seed, level, sg.start);
      sg.ntiles = (uint32_t)((sg.len + (uint64_t)l - 1) / l);
      nt = sg.ntiles;
      nb2 = 2ull * nl;
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
      atomicAdd((unsigned long long*)&w.ctrl->stats[1 + level], (unsigned long long)sg.len);
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
// open-addressing lookup table with 4 slots per heavy key.
// ----------------------------------------------------------------------------
template <class K, class V>
__global__ void __launch_bounds__(1024) k_sample(Work w, LevelBufs lb, uint32_t s_cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  K* S = reinterpret_cast<K*>(smem);
  __shared__ uint32_t tab[4 * kMaxHeavy];
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t nh_sh;
  const uint32_t ns = w.ctrl->nsegs[lb.level];
  for (uint32_t s = blockIdx.x; s < ns; s += gridDim.x) {
    const Seg sg = w.segs[lb.level][s];
    if (sg.lbits == 0) continue;
    const uint32_t hcap = hcap_of(sg.lbits);
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
    for (uint32_t t = threadIdx.x; t < tsize; t += blockDim.x) ht[t] = (uint16_t)(tab[t] == kEmpty ? 0xFFFFu : tab[t]);
    if (threadIdx.x == 0) {
      w.segs[lb.level][s].nh = nh;
      if (lb.level == 0) w.ctrl->stats[7] = nh;
    }
    __syncthreads();
  }
}

// Load a segment's heavy keys and table into shared memory.
template <class K>
__device__ __forceinline__ void load_heavy(const Work& w, int level, const Seg& sg, K* hk, uint16_t* ht) {
  if (sg.nh) {
    const uint32_t tsize = 4 * hcap_of(sg.lbits);
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

template <class K, class V, int OP>
__global__ void __launch_bounds__(kCountThreads) k_count(Work w, LevelBufs lb) {
  __shared__ uint32_t hist[kMaxBuckets];
  __shared__ K hk[kMaxHeavy];
  __shared__ uint16_t ht[4 * kMaxHeavy];
  __shared__ unsigned long long hsum[OP == kOpReduce ? kMaxHeavy : 1];
  const uint32_t nt = w.ctrl->ntiles[lb.level];
  for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
    const Tile tl = w.tiles[lb.level][t];
    const Seg sg = w.segs[lb.level][tl.seg];
    const uint32_t nl = 1u << sg.lbits;
    const uint32_t nb = nl + sg.nh;
    const uint32_t tmask = 4 * hcap_of(sg.lbits) - 1;
    load_heavy<K>(w, lb.level, sg, hk, ht);
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
    if (OP == kOpReduce)
      for (uint32_t b = threadIdx.x; b < sg.nh; b += blockDim.x) hsum[b] = 0;
    __syncthreads();
    constexpr int U = 4;
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
          const uint32_t b = bucket_of<K>(key[u], sg.mult, sg.lbits, sg.nh, hk, ht, tmask);
          atomicAdd(&hist[b], 1u);
          if constexpr (OP == kOpReduce) {
            if (b >= nl) {
              uint64_t v;
              if (lb.src_aos)
                v = (uint64_t)reinterpret_cast<const RecT<K, uint64_t>*>(lb.src_k)[tl.start + i].v;
              else
                v = reinterpret_cast<const uint64_t*>(lb.src_v)[tl.start + i];
              atomicAdd(&hsum[b - nl], (unsigned long long)v);
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
      for (uint32_t b = threadIdx.x; b < sg.nh; b += blockDim.x) HP[(uint64_t)b * sg.ntiles + tl.idx] = hsum[b];
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
  if (b >= nl) {
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
// the other.  Run by one thread; writes the items when `items` is non-null.
__device__ __forceinline__ uint32_t refine_windows(const uint32_t* bsize, const uint32_t* boff, uint32_t nl,
                                                   uint32_t alpha, bool last, uint64_t seg_start, uint32_t buf,
                                                   int level, Item* items, uint32_t first, uint32_t cap) {
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
  for (uint32_t b = 0; b < nl; ++b) {
    const uint32_t sz = bsize[b];
    if (sz == 0) continue;
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
    const uint32_t nl = 1u << sg.lbits;
    const uint32_t nb = nl + sg.nh;
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
      if (lane == 0) bsize[b] = run;
    }
    __syncthreads();
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    uint32_t nfin = 0, nnext = 0;
    for (uint32_t b0 = 0; b0 < nb; b0 += blockDim.x) {
      const uint32_t b = b0 + threadIdx.x;
      const uint32_t sz = b < nb ? bsize[b] : 0;
      const bool heavy = b >= nl;
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
    if (threadIdx.x == 0) {
      const uint32_t nw = refine_windows(bsize, boff, nl, w.alpha, last_level, sg.start, lb.dst_id, lb.level,
                                         nullptr, 0, 0);
      w.segs[lb.level][s].cnt_fin = tf + nw;
      w.segs[lb.level][s].cnt_next = tn;
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// distribute: the second pass of Blocked Distributing (Sec. 3.2).  Each CTA
// walks its subarray chunk by chunk in input order.  Inside a chunk the
// records are ranked stably by bucket id (BlockRank, two 5-bit passes, no
// atomics), staged in shared memory in bucket order, and written as
// contiguous runs at X[bucket][subarray] + (records of that bucket already
// written): stable, and no two CTAs ever write the same slot (race-free).
// Light records go to the level's temporary array (records), heavy records
// straight to their final place.
// ----------------------------------------------------------------------------
constexpr int kDT = 256;
constexpr int kDR = 16;
constexpr int kDCH = kDT * kDR;  // 4096 records per chunk
using DRank = BlockRank<kDT, kDR, 5>;

template <class K, class V>
struct DistSmem {
  union {
    struct {
      typename DRank::Smem rk;
      uint32_t tmp[kDCH + kDCH / 32];
    } a;
    RecT<K, V> stage[kDCH];
  } u;
  uint16_t fpos[kDCH];
  uint16_t sbid[kDCH];
  uint32_t running[kMaxBuckets];
  uint32_t base[kMaxBuckets];
  K hk[kMaxHeavy];
  uint16_t ht[4 * kMaxHeavy];
};

template <class K, class V, int OP>
__global__ void __launch_bounds__(kDT, 2) k_distribute(Work w, LevelBufs lb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DistSmem<K, V>& sm = *reinterpret_cast<DistSmem<K, V>*>(smem_raw);
  using Rec = RecT<K, V>;
  constexpr bool kVals = !std::is_same<V, void>::value;
  using VV = typename ValT<V>::type;
  const uint32_t nt = w.ctrl->ntiles[lb.level];
  constexpr bool kMoveHeavy = (OP == kOpEqual || OP == kOpLess);
  Rec* dst = reinterpret_cast<Rec*>(lb.dst);
  const int tid = threadIdx.x;
  const uint32_t c0t = tid * kDR;
  for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
    const Tile tl = w.tiles[lb.level][t];
    const Seg sg = w.segs[lb.level][tl.seg];
    const uint32_t nl = 1u << sg.lbits;
    const uint32_t nb = nl + sg.nh;
    const uint32_t tmask = 4 * hcap_of(sg.lbits) - 1;
    load_heavy<K>(w, lb.level, sg, sm.hk, sm.ht);
    {
      const uint32_t* X = w.C[lb.level] + sg.cbase;
      const uint32_t* boff = w.boff[lb.level] + sg.bbase;
      for (uint32_t b = tid; b < nb; b += kDT) sm.running[b] = boff[b] + X[(uint64_t)b * sg.ntiles + tl.idx];
    }
    __syncthreads();
    const bool two_pass = nb > 32;
    for (uint32_t c0 = 0; c0 < tl.len; c0 += kDCH) {
      const uint32_t clen = tl.len - c0 < (uint32_t)kDCH ? tl.len - c0 : (uint32_t)kDCH;
      const uint64_t gbase = tl.start + c0;
      uint32_t bid[kDR], rk[kDR];
      {
        K key[kDR];
#pragma unroll
        for (int r = 0; r < kDR; ++r)
          if (c0t + r < clen) key[r] = load_key<K, V>(lb.src_k, lb.src_aos, gbase + c0t + r);
        // invalid slots get the largest bucket id: both 5-bit digits are 31, so they rank last
#pragma unroll
        for (int r = 0; r < kDR; ++r)
          bid[r] = c0t + r < clen ? bucket_of<K>(key[r], sg.mult, sg.lbits, sg.nh, sm.hk, sm.ht, tmask)
                                  : (kMaxBuckets - 1);
      }
      DRank::rank(sm.u.a.rk, bid, 0, rk);
      if (!two_pass) {
#pragma unroll
        for (int r = 0; r < kDR; ++r) {
          sm.fpos[c0t + r] = (uint16_t)rk[r];
          sm.sbid[rk[r]] = (uint16_t)bid[r];
        }
      } else {
#pragma unroll
        for (int r = 0; r < kDR; ++r) sm.u.a.tmp[bpad(rk[r])] = (bid[r] << 16) | (c0t + r);
        __syncthreads();
        uint32_t x[kDR];
#pragma unroll
        for (int r = 0; r < kDR; ++r) x[r] = sm.u.a.tmp[bpad(c0t + r)];
        DRank::rank(sm.u.a.rk, x, 21, rk);
#pragma unroll
        for (int r = 0; r < kDR; ++r) {
          sm.fpos[x[r] & 0xFFFFu] = (uint16_t)rk[r];
          sm.sbid[rk[r]] = (uint16_t)(x[r] >> 16);
        }
      }
      __syncthreads();
      // stage records in bucket order (the rank scratch is dead now); the
      // records are read again (cache hits) rather than held in registers
#pragma unroll
      for (int r = 0; r < kDR; ++r) {
        const uint32_t c = c0t + r;
        if (c < clen) {
          Rec rec;
          if (lb.src_aos) {
            rec = reinterpret_cast<const Rec*>(lb.src_k)[gbase + c];
          } else {
            rec.k = reinterpret_cast<const K*>(lb.src_k)[gbase + c];
            if constexpr (kVals) rec.v = reinterpret_cast<const VV*>(lb.src_v)[gbase + c];
          }
          sm.u.stage[sm.fpos[c]] = rec;
        }
      }
      for (uint32_t p = tid; p < clen; p += kDT) {
        const uint32_t b = sm.sbid[p];
        if (p == 0 || sm.sbid[p - 1] != b) sm.base[b] = sm.running[b] - p;
      }
      __syncthreads();
      for (uint32_t p = tid; p < clen; p += kDT) {
        const uint32_t b = sm.sbid[p];
        const uint32_t rel = sm.base[b] + p;
        const uint64_t pos = sg.start + rel;
        const Rec rec = sm.u.stage[p];
        if (b < nl) {
          dst[pos] = rec;
        } else if constexpr (kMoveHeavy) {
          if (lb.hdst_aos) {
            reinterpret_cast<Rec*>(lb.hdst_k)[pos] = rec;
          } else {
            reinterpret_cast<K*>(lb.hdst_k)[pos] = rec.k;
            if constexpr (kVals) reinterpret_cast<VV*>(lb.hdst_v)[pos] = rec.v;
          }
        }
        if (p == clen - 1 || sm.sbid[p + 1] != b) sm.running[b] = rel + 1;
      }
      __syncthreads();
    }
  }
}

// ----------------------------------------------------------------------------
// scan_items: one CTA.  Exclusive scans over the segments' item counts give
// every segment its slice of the finish list and of the next level.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_scan_items(Work w, int level) {
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
  const uint32_t ns = w.ctrl->nsegs[lb.level];
  const bool last_level = lb.level == kMaxLevels - 1;
  for (uint32_t s = blockIdx.x; s < ns; s += gridDim.x) {
    const Seg sg = w.segs[lb.level][s];
    if (sg.lbits == 0) continue;
    const uint32_t nl = 1u << sg.lbits;
    const uint32_t nb = nl + sg.nh;
    const uint32_t* bsize = w.bsize[lb.level] + sg.bbase;
    const uint32_t* boff = w.boff[lb.level] + sg.bbase;
    if (threadIdx.x == 0) {
      const uint32_t nw = refine_windows(bsize, boff, nl, w.alpha, last_level, sg.start, lb.dst_id, lb.level,
                                         w.items, sg.fin_off, w.item_cap);
      for (uint32_t b = 0; b < nl; ++b)
        if (bsize[b] > w.alpha && last_level) set_error(w.ctrl, 8 /*SS_ERR_DEPTH*/);
      carry[0] = sg.fin_off + nw;
      carry[1] = sg.next_off;
    }
    __syncthreads();
    for (uint32_t b0 = 0; b0 < nb; b0 += blockDim.x) {
      const uint32_t b = b0 + threadIdx.x;
      const uint32_t sz = b < nb ? bsize[b] : 0;
      const bool heavy = b >= nl;
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
            it.start = 0;
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
// Base case: a shared-memory hash table maps each key to the index of its
// first occurrence in the bucket (insert by atomicCAS, then atomicMin, so the
// label does not depend on scheduling).  A scan over first occurrences turns
// labels into group ids 0..G-1 in first-occurrence order; ranking the records
// stably by group id (BlockRank, ceil(log2 G)/5 passes) puts every group in one
// run, groups in first-occurrence order and records of a group in input order
// -- the same result as the chained hash table of Sec. 3.3.
// ----------------------------------------------------------------------------
constexpr int kRT = 256;
constexpr int kRR = 16;
constexpr int kRefMax = kRT * kRR;  // alpha upper bound (4096)
using RRank = BlockRank<kRT, kRR, 5>;

template <class K, class V>
struct RefSmem {
  union {
    struct {
      K keys[kRefMax];
      uint32_t table[2 * kRefMax];
    } h;
    struct {
      typename RRank::Smem rk;
      uint32_t tmp[kRefMax + kRefMax / 32];
    } a;
    RecT<K, V> stage[kRefMax];
  } u;
  uint16_t fpos[kRefMax];
  uint16_t gid[kRefMax];
  uint32_t scan_tmp[33];
};

// Read record c of an item: AoS temporary, or the caller's SoA input.
template <class K, class V>
__device__ __forceinline__ RecT<K, V> load_rec(const Work& w, uint32_t buf, uint64_t c) {
  RecT<K, V> r;
  if (buf == kBufIn) {
    r.k = reinterpret_cast<const K*>(w.in_k)[c];
    if constexpr (!std::is_same<V, void>::value) r.v = reinterpret_cast<const V*>(w.in_v)[c];
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

template <class K, class V>
__global__ void __launch_bounds__(kRT, 2) k_finish_equal(Work w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RefSmem<K, V>& sm = *reinterpret_cast<RefSmem<K, V>*>(smem_raw);
  const uint32_t nfin = w.ctrl->nfin;
  const int tid = threadIdx.x;
  const uint32_t c0t = tid * kRR;
  const uint64_t salt = refine_salt(w.seed);
  for (uint32_t itx = blockIdx.x; itx < nfin; itx += gridDim.x) {
    const Item it = w.items[itx];
    if (it.kind == kItemCopy) {
      for (uint32_t i = tid; i < it.len; i += kRT)
        store_out<K, V>(w, it.start + i, load_rec<K, V>(w, it.buf, it.start + i));
      if (tid == 0) atomicAdd((unsigned long long*)&w.ctrl->stats[6], (unsigned long long)it.len);
      continue;
    }
    const uint32_t m = it.len;
    if (m > (uint32_t)kRefMax) {
      if (tid == 0) set_error(w.ctrl, 8);
      continue;
    }
    uint32_t ts = 64;
    while (ts < 2 * m) ts <<= 1;
    uint32_t slot[kRR];
    for (uint32_t c = tid; c < m; c += kRT)
      sm.u.h.keys[c] = it.buf == kBufIn ? reinterpret_cast<const K*>(w.in_k)[it.start + c]
                                        : reinterpret_cast<const RecT<K, V>*>(buf_ptr(w, it.buf))[it.start + c].k;
    for (uint32_t i = tid; i < ts; i += kRT) sm.u.h.table[i] = kEmpty;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRR; ++r) {
      const uint32_t c = c0t + r;
      slot[r] = 0;
      if (c < m) {
        const K key = sm.u.h.keys[c];
        const uint64_t h = KeyT<K>::hash(key, salt, false);
        uint32_t s = (uint32_t)h & (ts - 1);
        while (true) {
          uint32_t e = sm.u.h.table[s];
          if (e == kEmpty) {
            e = atomicCAS(&sm.u.h.table[s], kEmpty, c);
            if (e == kEmpty) break;
          }
          if (KeyT<K>::eq(sm.u.h.keys[e], key)) {
            atomicMin(&sm.u.h.table[s], c);
            break;
          }
          s = (s + 1) & (ts - 1);
        }
        slot[r] = s;
      }
    }
    __syncthreads();
    // first-occurrence labels -> group ids in first-occurrence order
    uint32_t lab[kRR];
    uint32_t nfirst = 0;
#pragma unroll
    for (int r = 0; r < kRR; ++r) {
      const uint32_t c = c0t + r;
      lab[r] = c < m ? sm.u.h.table[slot[r]] : 0;
      nfirst += (c < m && lab[r] == c) ? 1u : 0u;
    }
    uint32_t G;
    uint32_t g0 = block_exclusive_scan(nfirst, sm.scan_tmp, &G);
#pragma unroll
    for (int r = 0; r < kRR; ++r) {
      const uint32_t c = c0t + r;
      if (c < m && lab[r] == c) sm.gid[c] = (uint16_t)g0++;
    }
    __syncthreads();
    if (tid == 0) {
      atomicAdd((unsigned long long*)&w.ctrl->stats[5], (unsigned long long)m);
      atomicAdd((unsigned long long*)&w.ctrl->stats[9], 1ull);
      atomicMax((unsigned long long*)&w.ctrl->stats[8], (unsigned long long)m);
    }
    if (G == m) {
      // every key distinct: the bucket is already semisorted
      if (tid == 0) atomicAdd((unsigned long long*)&w.ctrl->stats[10], (unsigned long long)m);
      for (uint32_t c = tid; c < m; c += kRT) store_out<K, V>(w, it.start + c, load_rec<K, V>(w, it.buf, it.start + c));
      __syncthreads();
      continue;
    }
    // stable LSD ranking by group id, 5 bits per pass
    uint32_t g[kRR], rk[kRR], orig[kRR];
#pragma unroll
    for (int r = 0; r < kRR; ++r) {
      g[r] = c0t + r < m ? sm.gid[lab[r]] : 0xFFFu;
      orig[r] = c0t + r;
    }
    const uint32_t gbits = ceil_log2_u32(G) < 1 ? 1 : ceil_log2_u32(G);
    const uint32_t passes = (gbits + 4) / 5;
    __syncthreads();  // the hash table region becomes rank scratch
    for (uint32_t pz = 0; pz < passes; ++pz) {
      RRank::rank(sm.u.a.rk, g, 5 * pz, rk);
      if (pz + 1 < passes) {
#pragma unroll
        for (int r = 0; r < kRR; ++r) sm.u.a.tmp[bpad(rk[r])] = (g[r] << 16) | orig[r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kRR; ++r) {
          const uint32_t x = sm.u.a.tmp[bpad(c0t + r)];
          g[r] = x >> 16;
          orig[r] = x & 0xFFFFu;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < kRR; ++r)
      if (orig[r] < m) sm.fpos[orig[r]] = (uint16_t)rk[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRR; ++r) {
      const uint32_t c = c0t + r;
      if (c < m) sm.u.stage[sm.fpos[c]] = load_rec<K, V>(w, it.buf, it.start + c);
    }
    __syncthreads();
    for (uint32_t p = tid; p < m; p += kRT) store_out<K, V>(w, it.start + p, sm.u.stage[p]);
    __syncthreads();
  }
}

}  // namespace ss
