// Plain CPU oracle for semisort, collect-reduce and histogram.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
// calls this file; only the tests, the smoke check and the bench's CPU
// baseline leg do.  It shares no code, header, table or helper with the CUDA
// library.
//
// Every routine here is the plain definition of the problem, written out, not
// the paper's algorithm:
//   * semisort_< is the stable sort by key (Sec. 2.1, "stable" definition, and
//     the base case of Sec. 3.3 which asks for a stable comparison sort).
//   * semisort_= accepts any grouping; its canonical form is the stable sort by
//     key.  A second, independent reading is the hash-table group-by in
//     first-occurrence order (the separate-chaining base case of Sec. 3.3,
//     which keeps input order inside each chain).
//   * histogram (Sec. 2.1): (unique key, number of occurrences).
//   * collect-reduce (Sec. 2.1) with the map M(r) = value and the monoid
//     (+ mod 2^64, 0), the operator the paper's experiments use (Sec. 5.2).
// Both the sort path and the hash path exist so that each can be checked
// against the other and against O(n^2) brute force in the tests.
//
// Key types: 0 = uint32, 1 = uint64, 2 = 128-bit (little-endian lo, hi;
// ordered as an unsigned 128-bit integer).  Value types: 0 = uint32,
// 1 = uint64.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <functional>
#include <numeric>
#include <unordered_map>
#include <vector>

namespace {

struct K128 {
  uint64_t lo, hi;
};
inline bool operator==(const K128& a, const K128& b) { return a.lo == b.lo && a.hi == b.hi; }
inline bool operator!=(const K128& a, const K128& b) { return !(a == b); }
inline bool operator<(const K128& a, const K128& b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
struct K128Hash {
  size_t operator()(const K128& k) const {
    return std::hash<uint64_t>()(k.lo) ^ (std::hash<uint64_t>()(k.hi) * 0x100000001b3ull);
  }
};
template <class K>
struct HashOf {
  using type = std::hash<K>;
};
template <>
struct HashOf<K128> {
  using type = K128Hash;
};

// Permutation that stably sorts the records by key.
template <class K>
std::vector<uint64_t> stable_order(uint64_t n, const K* keys) {
  std::vector<uint64_t> p(n);
  std::iota(p.begin(), p.end(), uint64_t(0));
  std::stable_sort(p.begin(), p.end(), [&](uint64_t a, uint64_t b) { return keys[a] < keys[b]; });
  return p;
}

// Group ids in first-occurrence order, and the size of each group.
template <class K>
void first_occurrence_groups(uint64_t n, const K* keys, std::vector<uint64_t>& gid,
                             std::vector<uint64_t>& gsize, std::vector<uint64_t>& gfirst) {
  std::unordered_map<K, uint64_t, typename HashOf<K>::type> table;
  table.reserve(size_t(n) + 1);
  gid.resize(n);
  gsize.clear();
  gfirst.clear();
  for (uint64_t i = 0; i < n; ++i) {
    auto it = table.find(keys[i]);
    if (it == table.end()) {
      uint64_t g = gsize.size();
      table.emplace(keys[i], g);
      gsize.push_back(1);
      gfirst.push_back(i);
      gid[i] = g;
    } else {
      gid[i] = it->second;
      gsize[it->second] += 1;
    }
  }
}

template <class K, class V>
void stable_sort_kv(uint64_t n, const K* keys, const V* vals, K* ko, V* vo) {
  std::vector<uint64_t> p = stable_order(n, keys);
  std::vector<K> kt(n);
  std::vector<V> vt(n);
  for (uint64_t i = 0; i < n; ++i) {
    kt[i] = keys[p[i]];
    if (vals) vt[i] = vals[p[i]];
  }
  if (n) std::memcpy(ko, kt.data(), n * sizeof(K));
  if (vals && vo && n) std::memcpy(vo, vt.data(), n * sizeof(V));
}

template <class K, class V>
void group_by_kv(uint64_t n, const K* keys, const V* vals, K* ko, V* vo) {
  std::vector<uint64_t> gid, gsize, gfirst;
  first_occurrence_groups(n, keys, gid, gsize, gfirst);
  std::vector<uint64_t> cursor(gsize.size());
  uint64_t acc = 0;
  for (size_t g = 0; g < gsize.size(); ++g) {
    cursor[g] = acc;
    acc += gsize[g];
  }
  std::vector<K> kt(n);
  std::vector<V> vt(n);
  for (uint64_t i = 0; i < n; ++i) {  // input order, so each chain stays stable
    uint64_t pos = cursor[gid[i]]++;
    kt[pos] = keys[i];
    if (vals) vt[pos] = vals[i];
  }
  if (n) std::memcpy(ko, kt.data(), n * sizeof(K));
  if (vals && vo && n) std::memcpy(vo, vt.data(), n * sizeof(V));
}

// Sort path of collect-reduce: unique keys in ascending order.
template <class K>
uint64_t reduce_sorted(uint64_t n, const K* keys, const uint64_t* vals, K* uk, uint64_t* sums,
                       uint32_t* counts) {
  std::vector<uint64_t> p = stable_order(n, keys);
  uint64_t u = 0;
  for (uint64_t i = 0; i < n;) {
    uint64_t j = i;
    uint64_t s = 0;
    while (j < n && keys[p[j]] == keys[p[i]]) {
      if (vals) s += vals[p[j]];  // unsigned wraparound = addition mod 2^64
      ++j;
    }
    uk[u] = keys[p[i]];
    if (sums) sums[u] = s;
    if (counts) counts[u] = uint32_t(j - i);
    ++u;
    i = j;
  }
  return u;
}

// Hash path of collect-reduce: unique keys in first-occurrence order.
template <class K>
uint64_t reduce_hash(uint64_t n, const K* keys, const uint64_t* vals, K* uk, uint64_t* sums,
                     uint32_t* counts) {
  std::vector<uint64_t> gid, gsize, gfirst;
  first_occurrence_groups(n, keys, gid, gsize, gfirst);
  uint64_t u = gsize.size();
  for (uint64_t g = 0; g < u; ++g) {
    uk[g] = keys[gfirst[g]];
    if (sums) sums[g] = 0;
    if (counts) counts[g] = uint32_t(gsize[g]);
  }
  if (sums && vals)
    for (uint64_t i = 0; i < n; ++i) sums[gid[i]] += vals[i];
  return u;
}

template <class K>
uint64_t count_runs(uint64_t n, const K* keys) {
  uint64_t r = 0;
  for (uint64_t i = 0; i < n; ++i)
    if (i == 0 || keys[i] != keys[i - 1]) ++r;
  return r;
}

template <class K>
uint64_t count_distinct(uint64_t n, const K* keys) {
  std::unordered_map<K, char, typename HashOf<K>::type> t;
  t.reserve(size_t(n) + 1);
  for (uint64_t i = 0; i < n; ++i) t.emplace(keys[i], 0);
  return t.size();
}

template <class F>
int dispatch_k(int kt, F&& f) {
  switch (kt) {
    case 0: f((const uint32_t*)nullptr); return 0;
    case 1: f((const uint64_t*)nullptr); return 0;
    case 2: f((const K128*)nullptr); return 0;
    default: return -1;
  }
}

template <class F>
int dispatch_kv(int kt, int vt, F&& f) {
  if (vt != 0 && vt != 1) return -1;
  return dispatch_k(kt, [&](auto kp) {
    using K = std::remove_const_t<std::remove_pointer_t<decltype(kp)>>;
    if (vt == 0)
      f((K*)nullptr, (uint32_t*)nullptr);
    else
      f((K*)nullptr, (uint64_t*)nullptr);
  });
}

}  // namespace

extern "C" {

// semisort_< by definition; also the canonical form of semisort_=.
// vals/vals_out may be NULL (keys only).  Returns 0, or -1 on a bad type code.
int ss_oracle_stable_sort(int kt, int vt, uint64_t n, const void* keys, const void* vals,
                          void* keys_out, void* vals_out) {
  return dispatch_kv(kt, vt, [&](auto kp, auto vp) {
    using K = std::remove_pointer_t<decltype(kp)>;
    using V = std::remove_pointer_t<decltype(vp)>;
    stable_sort_kv<K, V>(n, (const K*)keys, (const V*)vals, (K*)keys_out, (V*)vals_out);
  });
}

// semisort_= by the hash-table reading: groups in first-occurrence order,
// input order inside each group.
int ss_oracle_group_by(int kt, int vt, uint64_t n, const void* keys, const void* vals,
                       void* keys_out, void* vals_out) {
  return dispatch_kv(kt, vt, [&](auto kp, auto vp) {
    using K = std::remove_pointer_t<decltype(kp)>;
    using V = std::remove_pointer_t<decltype(vp)>;
    group_by_kv<K, V>(n, (const K*)keys, (const V*)vals, (K*)keys_out, (V*)vals_out);
  });
}

// collect-reduce with (+ mod 2^64, 0); sort path (ascending keys).
// ukeys/sums must hold n entries.  Returns the number of unique keys.
uint64_t ss_oracle_collect_reduce_sorted(int kt, uint64_t n, const void* keys, const uint64_t* vals,
                                         void* ukeys, uint64_t* sums) {
  uint64_t u = 0;
  dispatch_k(kt, [&](auto kp) {
    using K = std::remove_const_t<std::remove_pointer_t<decltype(kp)>>;
    u = reduce_sorted<K>(n, (const K*)keys, vals, (K*)ukeys, sums, nullptr);
  });
  return u;
}

// collect-reduce, hash path (first-occurrence order).
uint64_t ss_oracle_collect_reduce_hash(int kt, uint64_t n, const void* keys, const uint64_t* vals,
                                       void* ukeys, uint64_t* sums) {
  uint64_t u = 0;
  dispatch_k(kt, [&](auto kp) {
    using K = std::remove_const_t<std::remove_pointer_t<decltype(kp)>>;
    u = reduce_hash<K>(n, (const K*)keys, vals, (K*)ukeys, sums, nullptr);
  });
  return u;
}

// histogram; sort path (ascending keys).
uint64_t ss_oracle_histogram_sorted(int kt, uint64_t n, const void* keys, void* ukeys,
                                    uint32_t* counts) {
  uint64_t u = 0;
  dispatch_k(kt, [&](auto kp) {
    using K = std::remove_const_t<std::remove_pointer_t<decltype(kp)>>;
    u = reduce_sorted<K>(n, (const K*)keys, nullptr, (K*)ukeys, nullptr, counts);
  });
  return u;
}

// histogram; hash path (first-occurrence order).
uint64_t ss_oracle_histogram_hash(int kt, uint64_t n, const void* keys, void* ukeys,
                                  uint32_t* counts) {
  uint64_t u = 0;
  dispatch_k(kt, [&](auto kp) {
    using K = std::remove_const_t<std::remove_pointer_t<decltype(kp)>>;
    u = reduce_hash<K>(n, (const K*)keys, nullptr, (K*)ukeys, nullptr, counts);
  });
  return u;
}

// Number of maximal runs of equal adjacent keys.
uint64_t ss_oracle_count_runs(int kt, uint64_t n, const void* keys) {
  uint64_t r = 0;
  dispatch_k(kt, [&](auto kp) {
    using K = std::remove_const_t<std::remove_pointer_t<decltype(kp)>>;
    r = count_runs<K>(n, (const K*)keys);
  });
  return r;
}

// Number of distinct keys.
uint64_t ss_oracle_count_distinct(int kt, uint64_t n, const void* keys) {
  uint64_t r = 0;
  dispatch_k(kt, [&](auto kp) {
    using K = std::remove_const_t<std::remove_pointer_t<decltype(kp)>>;
    r = count_distinct<K>(n, (const K*)keys);
  });
  return r;
}

// The output-mixing function of SplitMix64 (Steele, Lea and Flood, OOPSLA
// 2014), written from its published definition.  The library's built-in key
// hash is specified to be this bijection, so tests compare against it.
uint64_t ss_oracle_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

}  // extern "C"
