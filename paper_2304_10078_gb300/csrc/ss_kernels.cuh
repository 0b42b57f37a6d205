// Kernels of the semisort pipeline and its host-side launcher (templated on
// key type K, value type V and operation OP).  Included by one translation
// unit per key type.
//
// One recursion level of Algorithm 1 is the kernel sequence
//   plan -> sample -> count -> scan -> distribute -> scan_items -> emit
// over all segments of the level at once; a final `finish` kernel runs every
// base case (Sec. 3.3) and every copy-back (Sec. 3.4) collected on the way.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

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
__host__ __device__ __forceinline__ uint64_t refine_salt(uint64_t seed) {
  return mix64(seed ^ 0x5EF1CE5EF1CE0001ull);
}

__device__ __forceinline__ uint32_t ceil_log2_u32(uint32_t x) { return x <= 1 ? 0 : 32 - __clz(x - 1); }

// Buffers of one level (host computes them; see buffer rules in the launcher).
struct LevelBufs {
  const void* src_k;
  const void* src_v;
  void* dst_k;
  void* dst_v;
  void* hdst_k;
  void* hdst_v;
  uint32_t dst_id;   // Buf id of dst
  uint32_t hdst_id;  // Buf id of the heavy destination
  int level;
  uint64_t salt;
};

template <class K>
__device__ __forceinline__ const K* kptr(const void* p) { return reinterpret_cast<const K*>(p); }

__device__ __forceinline__ void* buf_k(const Work& w, uint32_t id) {
  return id == kBufIn ? const_cast<void*>(w.in_k) : id == kBufT ? w.t_k : id == kBufOut ? w.out_k : w.t2_k;
}
__device__ __forceinline__ void* buf_v(const Work& w, uint32_t id) {
  return id == kBufIn ? const_cast<void*>(w.in_v) : id == kBufT ? w.t_v : id == kBufOut ? w.out_v : w.t2_v;
}

// Bucket of key k in its segment (GetBucketId of Algorithm 1): the heavy
// bucket n_L + i if k is the i-th heavy key, else the light bucket given by
// the level hash.  hk/ht: the segment's heavy keys and open-addressing table.
template <class K>
__device__ __forceinline__ uint32_t bucket_of(const K& k, uint64_t salt, uint32_t lbits, uint32_t nh,
                                              const K* hk, const uint32_t* ht, uint32_t tmask) {
  const uint64_t h = KeyT<K>::hash(k, salt, false);
  if (nh) {
    uint32_t slot = (uint32_t)(h ^ (h >> 29)) & tmask;
    while (true) {
      const uint32_t e = ht[slot];
      if (e == kEmpty) break;
      if (KeyT<K>::eq(hk[e], k)) return (1u << lbits) + e;
      slot = (slot + 1) & tmask;
    }
  }
  return light_bucket(h, lbits);
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
        uint64_t want = (2ull * sg.len + w.alpha - 1) / w.alpha;
        lb = want <= 2 ? 1u : (uint32_t)(64 - __clzll(want - 1));
        lb = lb > (uint32_t)kMaxLightLog2 ? (uint32_t)kMaxLightLog2 : lb;
      }
      const uint32_t nl = 1u << lb;
      const uint32_t hcap = nl < kMaxHeavy ? nl : kMaxHeavy;
      sg.lbits = lb;
      sg.nbcap = nl + hcap;
      sg.nh = 0;
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
// tau = |S|/n_H,cap times heavy.  Heavy keys get ids in ascending key order
// (deterministic) and an open-addressing lookup table.
// ----------------------------------------------------------------------------
template <class K>
__global__ void __launch_bounds__(1024) k_sample(Work w, LevelBufs lb, uint32_t s_cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  K* S = reinterpret_cast<K*>(smem);
  __shared__ uint32_t tab[2 * kMaxHeavy];
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t nh_sh;
  const uint32_t ns = w.ctrl->nsegs[lb.level];
  const K* src = kptr<K>(lb.src_k);
  for (uint32_t s = blockIdx.x; s < ns; s += gridDim.x) {
    Seg sg = w.segs[lb.level][s];
    if (sg.lbits == 0) continue;
    const uint32_t nl = 1u << sg.lbits;
    const uint32_t hcap = nl < kMaxHeavy ? nl : kMaxHeavy;
    uint32_t S_n = 16u * hcap;
    if (S_n > s_cap) S_n = s_cap;
    const uint32_t tau = S_n / hcap;
    const uint64_t base = mix64(lb.salt ^ (sg.start * 0xD1B54A32D192ED03ull));
    for (uint32_t t = threadIdx.x; t < S_n; t += blockDim.x) {
      const uint64_t r = mix64(base + (uint64_t)(t + 1) * 0x9E3779B97F4A7C15ull);
      const uint64_t pos = __umul64hi(r, (uint64_t)sg.len);
      S[t] = src[sg.start + pos];
    }
    __syncthreads();
    // bitonic sort of S (S_n is a power of two)
    for (uint32_t k = 2; k <= S_n; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        for (uint32_t p = threadIdx.x; p < S_n / 2; p += blockDim.x) {
          const uint32_t i = (p / j) * 2 * j + (p % j);
          const uint32_t ixj = i + j;
          const bool up = (i & k) == 0;
          K a = S[i], b = S[ixj];
          if (up ? KeyT<K>::lt(b, a) : KeyT<K>::lt(a, b)) {
            S[i] = b;
            S[ixj] = a;
          }
        }
        __syncthreads();
      }
    }
    // heavy keys: run starts whose run reaches length tau
    const uint32_t tsize = 2 * hcap;
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
    uint32_t nh = nh_sh < hcap ? nh_sh : hcap;
    __syncthreads();
    __threadfence_block();
    // insert heavy ids into the shared table, then publish it
    for (uint32_t i = threadIdx.x; i < nh; i += blockDim.x) {
      const K key = hk[i];
      const uint64_t h = KeyT<K>::hash(key, lb.salt, false);
      uint32_t slot = (uint32_t)(h ^ (h >> 29)) & (tsize - 1);
      while (atomicCAS(&tab[slot], kEmpty, i) != kEmpty) slot = (slot + 1) & (tsize - 1);
    }
    __syncthreads();
    uint32_t* ht = w.htab[lb.level] + sg.bbase;
    for (uint32_t t = threadIdx.x; t < tsize; t += blockDim.x) ht[t] = tab[t];
    if (threadIdx.x == 0) {
      w.segs[lb.level][s].nh = nh;
      if (lb.level == 0) w.ctrl->stats[7] = nh;
    }
    __syncthreads();
  }
}

// Load a segment's heavy keys and table into shared memory.
template <class K>
__device__ __forceinline__ void load_heavy(const Work& w, int level, const Seg& sg, K* hk, uint32_t* ht) {
  const uint32_t nl = 1u << sg.lbits;
  const uint32_t tsize = 2 * (nl < kMaxHeavy ? nl : kMaxHeavy);
  if (sg.nh) {
    const K* ghk = reinterpret_cast<const K*>(w.hkeys[level]) + sg.bbase;
    const uint32_t* ght = w.htab[level] + sg.bbase;
    for (uint32_t i = threadIdx.x; i < sg.nh; i += blockDim.x) hk[i] = ghk[i];
    for (uint32_t i = threadIdx.x; i < tsize; i += blockDim.x) ht[i] = ght[i];
  }
}

// ----------------------------------------------------------------------------
// count: the counting matrix C of Blocked Distributing (Sec. 3.2).  One CTA
// per subarray; equal bucket ids within a warp are combined with
// __match_any_sync before the shared-memory increment.
// ----------------------------------------------------------------------------
template <class K, int OP>
__global__ void __launch_bounds__(512) k_count(Work w, LevelBufs lb) {
  __shared__ uint32_t hist[(1 << kMaxLightLog2) + kMaxHeavy];
  __shared__ K hk[kMaxHeavy];
  __shared__ uint32_t ht[2 * kMaxHeavy];
  const uint32_t nt = w.ctrl->ntiles[lb.level];
  const K* src = kptr<K>(lb.src_k);
  const int lane = threadIdx.x & 31;
  for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
    const Tile tl = w.tiles[lb.level][t];
    const Seg sg = w.segs[lb.level][tl.seg];
    const uint32_t nl = 1u << sg.lbits;
    const uint32_t nb = nl + sg.nh;
    const uint32_t tmask = 2 * (nl < kMaxHeavy ? nl : kMaxHeavy) - 1;
    load_heavy<K>(w, lb.level, sg, hk, ht);
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    constexpr int R = 8;
    const uint32_t per = blockDim.x * R;
    for (uint32_t i0 = 0; i0 < tl.len; i0 += per) {
      K key[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t i = i0 + r * blockDim.x + threadIdx.x;
        if (i < tl.len) key[r] = src[tl.start + i];
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t i = i0 + r * blockDim.x + threadIdx.x;
        const bool valid = i < tl.len;
        uint32_t b = 0xFFFFFFFFu;
        if (valid) b = bucket_of<K>(key[r], lb.salt, sg.lbits, sg.nh, hk, ht, tmask);
        const uint32_t peers = __match_any_sync(kFull, b);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&hist[b], (uint32_t)__popc(peers));
      }
    }
    __syncthreads();
    uint32_t* C = w.C[lb.level] + sg.cbase;
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) C[(uint64_t)b * sg.ntiles + tl.idx] = hist[b];
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// scan: column-major prefix sum X of C (Sec. 3.2): within each bucket row an
// exclusive prefix over subarrays, then bucket offsets from the row totals.
// Also counts the finish items and next-level segments each segment will
// emit.  One CTA per segment.
// ----------------------------------------------------------------------------
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
      uint32_t sz = b < nb ? bsize[b] : 0;
      const bool heavy = b >= nl;
      // Collect-reduce and histogram never move heavy records (Sec. 3.5).
      const uint32_t lay = (heavy && (OP == kOpReduce || OP == kOpHist)) ? 0 : sz;
      uint32_t tot;
      const uint32_t ex = block_exclusive_scan(lay, tmp, &tot);
      if (b < nb) boff[b] = carry + ex;
      __syncthreads();
      if (threadIdx.x == 0) carry += tot;
      __syncthreads();
      if (b < nb && sz) {
        if (heavy) {
          if (OP == kOpReduce || OP == kOpHist)
            nfin += 1;
          else if (lb.hdst_id != kBufOut)
            nfin += (sz + kCopyChunk - 1) / kCopyChunk;
        } else if (sz <= w.alpha || last_level) {
          nfin += 1;
        } else {
          nnext += 1;
        }
      }
    }
    const uint32_t tf = block_reduce_sum(nfin, tmp);
    const uint32_t tn = block_reduce_sum(nnext, tmp);
    if (threadIdx.x == 0) {
      w.segs[lb.level][s].cnt_fin = tf;
      w.segs[lb.level][s].cnt_next = tn;
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// distribute: the second pass of Blocked Distributing (Sec. 3.2).  Each CTA
// walks its subarray chunk by chunk in input order.  Inside a chunk records
// are ranked stably by bucket (block_rank8, one or two 8-bit passes), staged
// in shared memory in bucket order, and written as contiguous runs at
// X[bucket][subarray] + (records of that bucket already written), so the
// output is stable and no two CTAs write the same slot (race-free).
// ----------------------------------------------------------------------------
constexpr int kDistThreads = 512;
constexpr int kDistR = 8;
constexpr int kDistChunk = kDistThreads * kDistR;  // 4096 records

template <class K>
struct DistSmem {
  uint64_t stage[kDistChunk * (sizeof(K) > 8 ? 2 : 1)];
  uint16_t sbid[kDistChunk];
  uint16_t fpos[kDistChunk];
  uint16_t tbid[kDistChunk];
  uint16_t tidx[kDistChunk];
  uint16_t hist[(kDistThreads / 32) * 256];
  uint32_t dsum[256 + 33];
  uint32_t running[(1 << kMaxLightLog2) + kMaxHeavy];
  uint16_t rstart[(1 << kMaxLightLog2) + kMaxHeavy];
  K hk[kMaxHeavy];
  uint32_t ht[2 * kMaxHeavy];
};

template <class K, class V, int OP>
__global__ void __launch_bounds__(kDistThreads, 2) k_distribute(Work w, LevelBufs lb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DistSmem<K>& sm = *reinterpret_cast<DistSmem<K>*>(smem_raw);
  constexpr int NW = kDistThreads / 32;
  constexpr int R = kDistR;
  const uint32_t nt = w.ctrl->ntiles[lb.level];
  const K* src_k = kptr<K>(lb.src_k);
  const V* src_v = reinterpret_cast<const V*>(lb.src_v);
  K* dst_k = reinterpret_cast<K*>(lb.dst_k);
  V* dst_v = reinterpret_cast<V*>(lb.dst_v);
  K* hdst_k = reinterpret_cast<K*>(lb.hdst_k);
  V* hdst_v = reinterpret_cast<V*>(lb.hdst_v);
  const bool move_vals = (OP == kOpEqual || OP == kOpLess || OP == kOpReduce) && w.has_vals;
  const bool move_heavy = (OP == kOpEqual || OP == kOpLess);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
    const Tile tl = w.tiles[lb.level][t];
    const Seg sg = w.segs[lb.level][tl.seg];
    const uint32_t nl = 1u << sg.lbits;
    const uint32_t nb = nl + sg.nh;
    const uint32_t tmask = 2 * (nl < kMaxHeavy ? nl : kMaxHeavy) - 1;
    load_heavy<K>(w, lb.level, sg, sm.hk, sm.ht);
    {
      const uint32_t* X = w.C[lb.level] + sg.cbase;
      const uint32_t* boff = w.boff[lb.level] + sg.bbase;
      for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x)
        sm.running[b] = boff[b] + X[(uint64_t)b * sg.ntiles + tl.idx];
    }
    __syncthreads();
    const bool two_pass = nb > 256;
    for (uint32_t c0 = 0; c0 < tl.len; c0 += kDistChunk) {
      const uint32_t clen = tl.len - c0 < (uint32_t)kDistChunk ? tl.len - c0 : (uint32_t)kDistChunk;
      const uint64_t gbase = tl.start + c0;
      K key[R];
      uint32_t bid[R], d[R], rk[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t ci = wid * 32 * R + r * 32 + lane;
        if (ci < clen) {
          key[r] = src_k[gbase + ci];
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t ci = wid * 32 * R + r * 32 + lane;
        bid[r] = ci < clen ? bucket_of<K>(key[r], lb.salt, sg.lbits, sg.nh, sm.hk, sm.ht, tmask) : 0xFFFFu;
        d[r] = bid[r] & 255u;
      }
      block_rank8<NW, R>(d, rk, sm.hist, sm.dsum);
      if (!two_pass) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const uint32_t ci = wid * 32 * R + r * 32 + lane;
          sm.fpos[ci] = (uint16_t)rk[r];
          sm.sbid[rk[r]] = (uint16_t)bid[r];
        }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const uint32_t ci = wid * 32 * R + r * 32 + lane;
          sm.tbid[rk[r]] = (uint16_t)bid[r];
          sm.tidx[rk[r]] = (uint16_t)ci;
        }
        __syncthreads();
        uint32_t b2[R], i2[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const uint32_t q = wid * 32 * R + r * 32 + lane;
          b2[r] = sm.tbid[q];
          i2[r] = sm.tidx[q];
          d[r] = b2[r] >> 8;
        }
        block_rank8<NW, R>(d, rk, sm.hist, sm.dsum);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          sm.fpos[i2[r]] = (uint16_t)rk[r];
          sm.sbid[rk[r]] = (uint16_t)b2[r];
        }
      }
      __syncthreads();
      for (uint32_t p = threadIdx.x; p < clen; p += blockDim.x) {
        const uint32_t b = sm.sbid[p];
        if (p == 0 || sm.sbid[p - 1] != b) sm.rstart[b] = (uint16_t)p;
      }
      // keys into bucket order
      K* stage_k = reinterpret_cast<K*>(sm.stage);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t ci = wid * 32 * R + r * 32 + lane;
        if (ci < clen) stage_k[sm.fpos[ci]] = key[r];
      }
      __syncthreads();
      for (uint32_t p = threadIdx.x; p < clen; p += blockDim.x) {
        const uint32_t b = sm.sbid[p];
        const uint64_t dst = sg.start + sm.running[b] + (p - sm.rstart[b]);
        if (b < nl)
          dst_k[dst] = stage_k[p];
        else if (move_heavy)
          hdst_k[dst] = stage_k[p];
      }
      __syncthreads();
      if (move_vals) {
        V* stage_v = reinterpret_cast<V*>(sm.stage);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const uint32_t ci = wid * 32 * R + r * 32 + lane;
          if (ci < clen) stage_v[sm.fpos[ci]] = src_v[gbase + ci];
        }
        __syncthreads();
        for (uint32_t p = threadIdx.x; p < clen; p += blockDim.x) {
          const uint32_t b = sm.sbid[p];
          const uint64_t dst = sg.start + sm.running[b] + (p - sm.rstart[b]);
          if (b < nl)
            dst_v[dst] = stage_v[p];
          else if (move_heavy)
            hdst_v[dst] = stage_v[p];
        }
        __syncthreads();
      }
      for (uint32_t p = threadIdx.x; p < clen; p += blockDim.x) {
        const uint32_t b = sm.sbid[p];
        if (p == clen - 1 || sm.sbid[p + 1] != b) sm.running[b] += p - sm.rstart[b] + 1;
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
      carry[0] = sg.fin_off;
      carry[1] = sg.next_off;
    }
    __syncthreads();
    for (uint32_t b0 = 0; b0 < nb; b0 += blockDim.x) {
      const uint32_t b = b0 + threadIdx.x;
      const uint32_t sz = b < nb ? bsize[b] : 0;
      const bool heavy = b >= nl;
      uint32_t nf = 0, nx = 0;
      if (b < nb && sz) {
        if (heavy) {
          if (OP == kOpReduce || OP == kOpHist)
            nf = 1;
          else if (lb.hdst_id != kBufOut)
            nf = (sz + kCopyChunk - 1) / kCopyChunk;
        } else if (sz <= w.alpha || last_level) {
          nf = 1;
        } else {
          nx = 1;
        }
      }
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
        } else {
          if (i0 < w.item_cap) {
            Item it;
            it.start = start;
            it.len = sz;
            it.kind = kItemRefine;
            it.buf = lb.dst_id;
            it.aux = it.aux2 = 0;
            it.level = lb.level;
            w.items[i0] = it;
          }
          if (sz > w.alpha) set_error(w.ctrl, 8 /*SS_ERR_DEPTH*/);
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
// label does not depend on scheduling).  Sorting the records stably by that
// label (block_rank8 passes) puts every group in one run, groups in
// first-occurrence order and records of a group in input order -- the same
// result as the chained hash table of Sec. 3.3.
// ----------------------------------------------------------------------------
constexpr int kRefThreads = 512;
constexpr int kRefR = 8;
constexpr int kRefMax = kRefThreads * kRefR;  // alpha upper bound (4096)

template <class K>
struct RefSmem {
  uint64_t stage[kRefMax * (sizeof(K) > 8 ? 2 : 1)];  // keys in input order, later staging
  uint32_t table[2 * kRefMax];
  uint16_t fpos[kRefMax];
  uint16_t tbid[kRefMax];
  uint16_t tidx[kRefMax];
  uint16_t hist[(kRefThreads / 32) * 256];
  uint32_t dsum[256 + 33];
  uint32_t flag[2];
};

template <class K, class V>
__device__ void copy_item(const Work& w, const Item& it) {
  const K* sk = reinterpret_cast<const K*>(buf_k(w, it.buf));
  K* dk = reinterpret_cast<K*>(w.out_k);
  for (uint32_t i = threadIdx.x; i < it.len; i += blockDim.x) dk[it.start + i] = sk[it.start + i];
  if (w.has_vals) {
    const V* sv = reinterpret_cast<const V*>(buf_v(w, it.buf));
    V* dv = reinterpret_cast<V*>(w.out_v);
    for (uint32_t i = threadIdx.x; i < it.len; i += blockDim.x) dv[it.start + i] = sv[it.start + i];
  }
}

template <class K, class V>
__global__ void __launch_bounds__(kRefThreads, 2) k_finish_equal(Work w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RefSmem<K>& sm = *reinterpret_cast<RefSmem<K>*>(smem_raw);
  constexpr int NW = kRefThreads / 32;
  constexpr int R = kRefR;
  const uint32_t nfin = w.ctrl->nfin;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint64_t salt = refine_salt(w.seed);
  K* sk = reinterpret_cast<K*>(sm.stage);
  for (uint32_t itx = blockIdx.x; itx < nfin; itx += gridDim.x) {
    const Item it = w.items[itx];
    if (it.kind == kItemCopy) {
      copy_item<K, V>(w, it);
      if (threadIdx.x == 0) atomicAdd((unsigned long long*)&w.ctrl->stats[6], (unsigned long long)it.len);
      continue;
    }
    const uint32_t m = it.len;
    if (m > (uint32_t)kRefMax) {
      if (threadIdx.x == 0) set_error(w.ctrl, 8);
      continue;
    }
    const K* src_k = reinterpret_cast<const K*>(buf_k(w, it.buf));
    const V* src_v = reinterpret_cast<const V*>(buf_v(w, it.buf));
    K* out_k = reinterpret_cast<K*>(w.out_k);
    V* out_v = reinterpret_cast<V*>(w.out_v);
    const bool inplace = it.buf == kBufOut || (it.buf == kBufIn && w.in_k == w.out_k);
    uint32_t ts = 64;
    while (ts < 2 * m) ts <<= 1;
    K key[R];
    uint32_t slot[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t j = wid * 32 * R + r * 32 + lane;
      if (j < m) {
        key[r] = src_k[it.start + j];
        sk[j] = key[r];
      }
    }
    for (uint32_t i = threadIdx.x; i < ts; i += blockDim.x) sm.table[i] = kEmpty;
    if (threadIdx.x == 0) {
      sm.flag[0] = 0;
      sm.flag[1] = 0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t j = wid * 32 * R + r * 32 + lane;
      if (j < m) {
        const uint64_t h = KeyT<K>::hash(key[r], salt, false);
        uint32_t s = (uint32_t)h & (ts - 1);
        while (true) {
          uint32_t e = sm.table[s];
          if (e == kEmpty) {
            e = atomicCAS(&sm.table[s], kEmpty, j);
            if (e == kEmpty) break;
          }
          if (KeyT<K>::eq(sk[e], key[r])) {
            atomicMin(&sm.table[s], j);
            break;
          }
          s = (s + 1) & (ts - 1);
        }
        slot[r] = s;
      }
    }
    __syncthreads();
    uint32_t lab[R];
    uint32_t firsts = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t j = wid * 32 * R + r * 32 + lane;
      lab[r] = j < m ? sm.table[slot[r]] : 0xFFFFu;
      firsts += (j < m && lab[r] == j) ? 1u : 0u;
    }
    const uint32_t groups = block_reduce_sum(firsts, sm.dsum + 256);
    if (threadIdx.x == 0) {
      atomicAdd((unsigned long long*)&w.ctrl->stats[5], (unsigned long long)m);
      atomicAdd((unsigned long long*)&w.ctrl->stats[9], 1ull);
      atomicMax((unsigned long long*)&w.ctrl->stats[8], (unsigned long long)m);
    }
    if (groups == m) {
      // every key distinct: the bucket is already semisorted
      if (threadIdx.x == 0) atomicAdd((unsigned long long*)&w.ctrl->stats[10], (unsigned long long)m);
      if (!inplace) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const uint32_t j = wid * 32 * R + r * 32 + lane;
          if (j < m) out_k[it.start + j] = key[r];
        }
        if (w.has_vals)
          for (uint32_t j = threadIdx.x; j < m; j += blockDim.x) out_v[it.start + j] = src_v[it.start + j];
      } else if (threadIdx.x == 0) {
        atomicAdd((unsigned long long*)&w.ctrl->stats[11], (unsigned long long)m);
      }
      __syncthreads();
      continue;
    }
    // stable sort by first-occurrence label
    uint32_t d[R], rk[R];
#pragma unroll
    for (int r = 0; r < R; ++r) d[r] = lab[r] & 255u;
    block_rank8<NW, R>(d, rk, sm.hist, sm.dsum);
    if (m <= 256) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t j = wid * 32 * R + r * 32 + lane;
        if (j < m) sm.fpos[j] = (uint16_t)rk[r];
      }
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t j = wid * 32 * R + r * 32 + lane;
        sm.tbid[rk[r]] = (uint16_t)lab[r];
        sm.tidx[rk[r]] = (uint16_t)j;
      }
      __syncthreads();
      uint32_t i2[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t q = wid * 32 * R + r * 32 + lane;
        d[r] = (uint32_t)sm.tbid[q] >> 8;
        i2[r] = sm.tidx[q];
      }
      block_rank8<NW, R>(d, rk, sm.hist, sm.dsum);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (i2[r] < m) sm.fpos[i2[r]] = (uint16_t)rk[r];
    }
    __syncthreads();
    // values must be read before any write when refining in place
    V val[R];
    if (w.has_vals) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t j = wid * 32 * R + r * 32 + lane;
        if (j < m) val[r] = src_v[it.start + j];
      }
    }
    uint32_t moved = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t j = wid * 32 * R + r * 32 + lane;
      if (j < m) {
        sk[sm.fpos[j]] = key[r];
        moved += sm.fpos[j] != j;
      }
    }
    const uint32_t any_moved = block_reduce_sum(moved, sm.dsum + 256);
    if (inplace && any_moved == 0) {
      if (threadIdx.x == 0) atomicAdd((unsigned long long*)&w.ctrl->stats[11], (unsigned long long)m);
      continue;
    }
    for (uint32_t p = threadIdx.x; p < m; p += blockDim.x) out_k[it.start + p] = sk[p];
    if (w.has_vals) {
      __syncthreads();
      V* sv = reinterpret_cast<V*>(sm.stage);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t j = wid * 32 * R + r * 32 + lane;
        if (j < m) sv[sm.fpos[j]] = val[r];
      }
      __syncthreads();
      for (uint32_t p = threadIdx.x; p < m; p += blockDim.x) out_v[it.start + p] = sv[p];
    }
    __syncthreads();
  }
}

}  // namespace ss
