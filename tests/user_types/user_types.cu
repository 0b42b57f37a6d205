// Test instantiations of the C++ template entry points (include/semisort.hpp)
// for a user-defined key type and a non-commutative monoid, exported with C
// linkage for the Python tests.
//
// Key12: three 32-bit words, equal when all words are equal, ordered as the
// 96-bit integer (c, b, a) -- the order of a 128-bit key (lo = a | b << 32,
// hi = c), so the oracle's 128-bit sort is the reference.
// Horner: values (h, p) with (h1, p1) op (h2, p2) = (h1 p2 + h2, p1 p2) mod
// 2^64, identity (0, 1): associative, not commutative.  A group of values
// (x_i, M) folds to (x_1 M^(k-1) + ... + x_k, M^k) only in input order.
#include <stdint.h>

#include "semisort.hpp"

struct Key12 {
  uint32_t a, b, c;
};

template <>
struct semisort::key_traits<Key12> {
  __device__ static uint64_t hash(const Key12& k) {
    return ((((uint64_t)k.b << 32) | k.a) * 0x9E3779B97F4A7C15ull) ^ ((uint64_t)k.c * 0xC2B2AE3D27D4EB4Full);
  }
  __device__ static bool equal(const Key12& x, const Key12& y) { return x.a == y.a && x.b == y.b && x.c == y.c; }
  __device__ static bool less(const Key12& x, const Key12& y) {
    if (x.c != y.c) return x.c < y.c;
    if (x.b != y.b) return x.b < y.b;
    return x.a < y.a;
  }
};

struct HornerV {
  uint64_t h, p;
};
struct Horner {
  __device__ HornerV operator()(const HornerV& x, const HornerV& y) const { return {x.h * y.p + y.h, x.p * y.p}; }
};

static ss_options opts(uint64_t seed, uint32_t alpha, uint32_t subarray, uint32_t lbits) {
  ss_options o = {};
  o.seed = seed;
  o.alpha = alpha;
  o.subarray = subarray;
  o.n_light_log2 = lbits;
  return o;
}

extern "C" {

size_t ut_workspace(int op, uint64_t n, uint32_t alpha, uint32_t subarray, uint32_t lbits) {
  const ss_options o = opts(0, alpha, subarray, lbits);
  return semisort::workspace_size<Key12, uint64_t>((ss_op)op, n, &o);
}

int ut_semisort(int op, const void* k, const uint64_t* v, void* ko, uint64_t* vo, uint64_t n, void* ws, size_t wsb,
                uint64_t seed, uint32_t alpha, uint32_t subarray, uint32_t lbits, void* stream) {
  const ss_options o = opts(seed, alpha, subarray, lbits);
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (op == SS_OP_SEMISORT_EQUAL)
    return semisort::semisort_equal<Key12, uint64_t>((const Key12*)k, v, (Key12*)ko, vo, n, ws, wsb, &o, st);
  return semisort::semisort_less<Key12, uint64_t>((const Key12*)k, v, (Key12*)ko, vo, n, ws, wsb, &o, st);
}

size_t ut_fold_workspace(uint64_t n, int key12) {
  const ss_options o = opts(0, 0, 0, 0);
  return key12 ? semisort::collect_reduce_workspace_size<Key12, HornerV>(n, &o)
               : semisort::collect_reduce_workspace_size<uint64_t, HornerV>(n, &o);
}

// collect-reduce with the Horner monoid; key12 = 1: Key12 keys, else u64 keys.
int ut_fold(int key12, const void* k, const void* v, void* uk, void* sums, uint64_t cap, uint64_t* nu, uint64_t n,
            void* ws, size_t wsb, uint64_t seed, void* stream) {
  const ss_options o = opts(seed, 0, 0, 0);
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const HornerV id = {0, 1};
  if (key12)
    return semisort::collect_reduce<Key12, HornerV, Horner>((const Key12*)k, (const HornerV*)v, (Key12*)uk,
                                                            (HornerV*)sums, cap, nu, n, Horner{}, id, ws, wsb, &o, st);
  return semisort::collect_reduce<uint64_t, HornerV, Horner>((const uint64_t*)k, (const HornerV*)v, (uint64_t*)uk,
                                                             (HornerV*)sums, cap, nu, n, Horner{}, id, ws, wsb, &o, st);
}

}  // extern "C"
