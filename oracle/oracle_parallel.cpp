// The oracle's stable sort (semisort_< by definition, Sec. 2.1) on all host
// cores, for the CPU baseline of the benchmark.
//
// TEST INFRASTRUCTURE ONLY, like oracle.cpp: only the tests and the bench's
// CPU legs load it.  It computes the same definition as ss_oracle_stable_sort
// -- the stable order of the records by key -- with libstdc++'s parallel-mode
// stable sort (OpenMP) in place of std::stable_sort; a test checks that both
// give identical outputs.  Built separately (with -fopenmp) so that a host
// without OpenMP still builds the main oracle.
#include <omp.h>

#include <cstdint>
#include <cstring>
#include <numeric>
#include <parallel/algorithm>
#include <vector>

namespace {

template <class K, class V>
void stable_sort_kv_parallel(uint64_t n, const K* keys, const V* vals, K* ko, V* vo) {
  std::vector<uint64_t> p(n);
  std::iota(p.begin(), p.end(), uint64_t(0));
  __gnu_parallel::stable_sort(p.begin(), p.end(), [&](uint64_t a, uint64_t b) { return keys[a] < keys[b]; });
  std::vector<K> kt(n);
  std::vector<V> vt(vals ? n : 0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)n; ++i) {
    kt[i] = keys[p[i]];
    if (vals) vt[i] = vals[p[i]];
  }
  if (n) std::memcpy(ko, kt.data(), n * sizeof(K));
  if (vals && vo && n) std::memcpy(vo, vt.data(), n * sizeof(V));
}

}  // namespace

extern "C" {

// Stable sort of (u32 or u64 key, u32 or u64 value) records by key on
// `threads` OpenMP threads (0 = all).  kt/vt: 0 = uint32, 1 = uint64.  vals
// and vals_out may be NULL.  Returns the thread count used, or -1 on a bad
// type code.
int ss_oracle_stable_sort_parallel(int kt, int vt, uint64_t n, const void* keys, const void* vals,
                                   void* keys_out, void* vals_out, int threads) {
  if ((kt != 0 && kt != 1) || (vt != 0 && vt != 1)) return -1;
  omp_set_num_threads(threads > 0 ? threads : omp_get_num_procs());
  const int used = omp_get_max_threads();
  if (kt == 0 && vt == 0)
    stable_sort_kv_parallel<uint32_t, uint32_t>(n, (const uint32_t*)keys, (const uint32_t*)vals,
                                                (uint32_t*)keys_out, (uint32_t*)vals_out);
  else if (kt == 0)
    stable_sort_kv_parallel<uint32_t, uint64_t>(n, (const uint32_t*)keys, (const uint64_t*)vals,
                                                (uint32_t*)keys_out, (uint64_t*)vals_out);
  else if (vt == 0)
    stable_sort_kv_parallel<uint64_t, uint32_t>(n, (const uint64_t*)keys, (const uint32_t*)vals,
                                                (uint64_t*)keys_out, (uint32_t*)vals_out);
  else
    stable_sort_kv_parallel<uint64_t, uint64_t>(n, (const uint64_t*)keys, (const uint64_t*)vals,
                                                (uint64_t*)keys_out, (uint64_t*)vals_out);
  return used;
}

}  // extern "C"
