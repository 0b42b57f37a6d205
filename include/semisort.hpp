/*
 * semisort.hpp -- C++ template entry points of the GB300 semisort library for
 * user-defined key types, value types and monoids.
 *
 * Sec. 2.1 of the paper states the problems for any key type with a
 * user-supplied hash function family and equality test (and a comparison for
 * semisort_<), and collect-reduce for any monoid (op, identity); Sec. 3.5
 * notes that a stable semisort lets op be non-commutative.  The C ABI
 * (semisort.h) fixes the built-in key types and the + monoid; this header
 * instantiates the same kernels for the caller's own types.  It is
 * header-only: include it in a .cu file compiled by nvcc for sm_103a
 * (-gencode arch=compute_103a,code=sm_103a -std=c++17 --expt-relaxed-constexpr).
 *
 * Key type K: trivially copyable, at most 16 bytes, with a specialization of
 * semisort::key_traits<K> providing
 *     __device__ static uint64_t hash(const K&);         equal keys hash equally
 *     __device__ static bool equal(const K&, const K&);
 *     __device__ static bool less(const K&, const K&);   strict weak order (semisort_less)
 * declared before the first use of these templates.  Hash collisions are
 * harmless: grouping always compares whole keys.  Value type V: trivially
 * copyable, at most 16 bytes (or void: keys only).  A (key, value) record is
 * held in at most 32 bytes.
 *
 * Conventions are those of semisort.h: device pointers owned by the caller,
 * arrays aligned to their element type, a 16-byte-aligned workspace sized by
 * the matching *_workspace_size, stream-ordered calls that never synchronize
 * with the host and never allocate, in-place calls allowed (keys_out == keys
 * together with vals_out == vals).  Return values report argument errors;
 * device-side failures set the workspace flag read by ss_last_device_error.
 */
#ifndef SEMISORT_HPP_
#define SEMISORT_HPP_

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "semisort.h"
#include "../paper_2304_10078_gb300/csrc/ss_fold.cuh"
#include "../paper_2304_10078_gb300/csrc/ss_launch.cuh"
#include "../paper_2304_10078_gb300/csrc/ss_plan_host.h"

namespace semisort {
namespace detail {

template <class V>
constexpr int vbytes() {
  if constexpr (std::is_same<V, void>::value)
    return 0;
  else
    return (int)sizeof(V);
}

inline int num_sms() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 152;
  return v;
}

template <class K, class V>
constexpr bool supported() {
  return std::is_trivially_copyable<K>::value && sizeof(K) <= 16 && sizeof(ss::RecT<K, V>) <= 32 &&
         (std::is_same<V, void>::value || std::is_trivially_copyable<V>::value);
}

template <class K, class V>
ss_status plan(int op, uint64_t n, const ss_options* opt, ss::Plan* P) {
  return ss::plan_workspace(op, (int)sizeof(K), vbytes<V>(), sizeof(ss::RecT<K, V>), ss::KeyT<K>::kIntegral, n, opt,
                            num_sms(), P);
}

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }
inline bool disjoint(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x + na <= y || y + nb <= x;
}

template <class K, class V, int OP>
ss_status run(const K* keys, const V* vals, K* keys_out, V* vals_out, uint64_t n, void* ws, size_t ws_bytes,
              const ss_options* opt, cudaStream_t st) {
  static_assert(supported<K, V>(), "key/value types: trivially copyable, keys <= 16 bytes, records <= 32 bytes");
  constexpr bool kVals = !std::is_same<V, void>::value;
  if (n == 0) return SS_OK;
  if (!keys || !keys_out || !ws || !aligned(ws, 16)) return SS_ERR_INVALID_ARG;
  if (!aligned(keys, alignof(K)) || !aligned(keys_out, alignof(K))) return SS_ERR_INVALID_ARG;
  const size_t kb = n * sizeof(K);
  if (keys != keys_out && !disjoint(keys, kb, keys_out, kb)) return SS_ERR_INVALID_ARG;
  if constexpr (kVals) {
    if ((vals == nullptr) != (vals_out == nullptr)) return SS_ERR_INVALID_ARG;
    if (vals) {
      const size_t vb = n * sizeof(V);
      if (!aligned(vals, alignof(V)) || !aligned(vals_out, alignof(V))) return SS_ERR_INVALID_ARG;
      if ((keys == keys_out) != (vals == vals_out)) return SS_ERR_INVALID_ARG;
      if (vals != vals_out && !disjoint(vals, vb, vals_out, vb)) return SS_ERR_INVALID_ARG;
    }
  }
  if (opt && opt->splitter_mode != 0) return SS_ERR_UNSUPPORTED;  // learned splitters: built-in integer keys only
  if (opt && (opt->flags & (SS_FLAG_IDENTITY_HASH | SS_FLAG_HASH_BUCKETS))) return SS_ERR_UNSUPPORTED;  // built-in keys only
  ss::Plan P;
  const ss_status s = plan<K, V>(OP, n, opt, &P);
  if (s != SS_OK) return s;
  if (ws_bytes < P.total) return SS_ERR_WORKSPACE_TOO_SMALL;
  if (!disjoint(ws, P.total, keys, kb) || !disjoint(ws, P.total, keys_out, kb)) return SS_ERR_INVALID_ARG;
  ss::Work w;
  memset(&w, 0, sizeof(w));
  ss::fill_work(P, ws, &w);
  w.seed = opt ? opt->seed : 0;
  w.in_k = keys;
  w.in_v = vals;
  w.out_k = keys_out;
  w.out_v = vals_out;
  w.has_vals = vals != nullptr;
  w.auto_nl = (opt && opt->n_light_log2) ? 0u : 1u;
  w.swap = (opt && (opt->flags & SS_FLAG_SWAP_OUTPUT)) ? 1u : 0u;
  int launches = 0;
  ss::LaunchCfg c{num_sms(), nullptr, &launches};
  const cudaError_t e = ss::launch_pipeline<K, V, OP>(P, w, st, c);
  return e == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

// Layout of the collect-reduce workspace after the semisort_= workspace.
template <class K, class V>
struct FoldLayout {
  size_t semi, keys, vals, starts, base, flags, head, tail, total;
  uint32_t ntiles;
  explicit FoldLayout(size_t semi_bytes, uint64_t n) {
    ntiles = (uint32_t)((n + ss::kFoldTile - 1) / ss::kFoldTile);
    size_t o = ss::al(semi_bytes);
    semi = 0;
    keys = o;
    o = ss::al(o + n * sizeof(K));
    vals = o;
    o = ss::al(o + n * sizeof(V));
    starts = o;
    o = ss::al(o + (size_t)ntiles * 4);
    base = o;
    o = ss::al(o + (size_t)ntiles * 8);
    flags = o;
    o = ss::al(o + (size_t)ntiles * 4);
    head = o;
    o = ss::al(o + (size_t)ntiles * sizeof(V));
    tail = o;
    o = ss::al(o + (size_t)ntiles * sizeof(V));
    total = o;
  }
};

}  // namespace detail

/* Bytes of workspace for semisort_equal (op SS_OP_SEMISORT_EQUAL) or
 * semisort_less (SS_OP_SEMISORT_LESS) on n records of key type K and value
 * type V (void: keys only); 0 on an unsupported size or op. */
template <class K, class V>
size_t workspace_size(ss_op op, uint64_t n, const ss_options* opt = nullptr) {
  if (op != SS_OP_SEMISORT_EQUAL && op != SS_OP_SEMISORT_LESS) return 0;
  ss::Plan P;
  return detail::plan<K, V>(op, n, opt, &P) == SS_OK ? P.total : 0;
}

/* semisort_= for key type K (semisort::key_traits<K>): records with equal
 * keys become contiguous, in input order (stable); group order unspecified
 * but fixed for a given seed.  vals/vals_out may be null with V = void. */
template <class K, class V>
ss_status semisort_equal(const K* keys, const V* vals, K* keys_out, V* vals_out, uint64_t n, void* ws,
                         size_t ws_bytes, const ss_options* opt, cudaStream_t stream) {
  return detail::run<K, V, ss::kOpEqual>(keys, vals, keys_out, vals_out, n, ws, ws_bytes, opt, stream);
}

/* semisort_< for key type K: the stable sort by key_traits<K>::less (range
 * buckets cut by sampled splitters, heavy keys in equality buckets, a stable
 * comparison sort per base case). */
template <class K, class V>
ss_status semisort_less(const K* keys, const V* vals, K* keys_out, V* vals_out, uint64_t n, void* ws,
                        size_t ws_bytes, const ss_options* opt, cudaStream_t stream) {
  return detail::run<K, V, ss::kOpLess>(keys, vals, keys_out, vals_out, n, ws, ws_bytes, opt, stream);
}

/* Bytes of workspace for collect_reduce on n records. */
template <class K, class V>
size_t collect_reduce_workspace_size(uint64_t n, const ss_options* opt = nullptr) {
  const size_t semi = workspace_size<K, V>(SS_OP_SEMISORT_EQUAL, n, opt);
  if (!semi && n) return 0;
  return detail::FoldLayout<K, V>(semi, n).total;
}

/* collect-reduce with the monoid (op, identity) (Sec. 2.1): one output
 * (key, v_1 op v_2 op ... op v_m) per distinct key, the values of a key
 * combined in input order, so op needs to be associative but not
 * commutative (Sec. 3.5).  Op is a functor with
 *     __device__ V operator()(const V& a, const V& b) const;
 * and identity its neutral element.  Runs as semisort_= (stable) into the
 * workspace, then an ordered segmented fold over the groups.  Writes the
 * number of distinct keys to *d_num_unique (device pointer) and the first
 * `capacity` outputs to ukeys_out / sums_out; output order is the group
 * order of the semisort (unspecified, fixed for a given seed). */
template <class K, class V, class Op>
ss_status collect_reduce(const K* keys, const V* vals, K* ukeys_out, V* sums_out, uint64_t capacity,
                         uint64_t* d_num_unique, uint64_t n, Op op, V identity, void* ws, size_t ws_bytes,
                         const ss_options* opt, cudaStream_t stream) {
  static_assert(!std::is_same<V, void>::value, "collect_reduce needs a value type");
  if (!d_num_unique || !detail::aligned(d_num_unique, 8)) return SS_ERR_INVALID_ARG;
  if (n == 0) return cudaMemsetAsync(d_num_unique, 0, 8, stream) == cudaSuccess ? SS_OK : SS_ERR_CUDA;
  if (!keys || !vals || !ws || (capacity && (!ukeys_out || !sums_out))) return SS_ERR_INVALID_ARG;
  const size_t semi = workspace_size<K, V>(SS_OP_SEMISORT_EQUAL, n, opt);
  if (!semi) return SS_ERR_UNSUPPORTED;
  const detail::FoldLayout<K, V> L(semi, n);
  if (ws_bytes < L.total) return SS_ERR_WORKSPACE_TOO_SMALL;
  char* b = static_cast<char*>(ws);
  K* sk = reinterpret_cast<K*>(b + L.keys);
  V* sv = reinterpret_cast<V*>(b + L.vals);
  ss_status s = semisort_equal<K, V>(keys, vals, sk, sv, n, b + L.semi, semi, opt, stream);
  if (s != SS_OK) return s;
  uint32_t* starts = reinterpret_cast<uint32_t*>(b + L.starts);
  uint64_t* base = reinterpret_cast<uint64_t*>(b + L.base);
  uint32_t* tflags = reinterpret_cast<uint32_t*>(b + L.flags);
  V* head = reinterpret_cast<V*>(b + L.head);
  V* tail = reinterpret_cast<V*>(b + L.tail);
  ss::k_fold_count<K><<<L.ntiles, ss::kFoldThreads, 0, stream>>>(sk, n, starts);
  ss::k_fold_scan<<<1, 1024, 0, stream>>>(starts, L.ntiles, base, d_num_unique);
  ss::k_fold_tiles<K, V, Op><<<L.ntiles, ss::kFoldThreads, 0, stream>>>(sk, sv, n, base, ukeys_out, sums_out,
                                                                          capacity, head, tail, tflags, op, identity);
  ss::k_fold_join<V, Op><<<(L.ntiles + 255) / 256, 256, 0, stream>>>(L.ntiles, base, starts, tflags, head, tail,
                                                                      sums_out, capacity, op);
  return cudaGetLastError() == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

}  // namespace semisort

#endif  // SEMISORT_HPP_
