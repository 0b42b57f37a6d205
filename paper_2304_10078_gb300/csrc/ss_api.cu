// C ABI of the semisort library: argument checks, the workspace plan and the
// dispatch to the per-key-type pipelines.  See include/semisort.h.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "../../include/semisort.h"
#include "ss_common.cuh"
#include "ss_host.h"
#include "ss_learn.cuh"
#include "ss_plan.h"
#include "ss_plan_host.h"

using namespace ss;

namespace {


int num_sms() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cache[dev]) cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev);
  return cache[dev];
}

int kbytes_of(int t) { return t == SS_U32 ? 4 : t == SS_U64 ? 8 : t == SS_U128 ? 16 : 0; }

// Plan for built-in key and value types (type codes of the C ABI).
ss_status make_plan(int op, int kt, int vt, uint64_t n, const ss_options* opt, int nsm, Plan* P,
                    uint32_t num_inst = 0) {
  const int kbytes = kbytes_of(kt);
  if (!kbytes) return SS_ERR_INVALID_ARG;
  if (op == SS_OP_SEMISORT_EQUAL || op == SS_OP_SEMISORT_LESS)
    if (vt != SS_U32 && vt != SS_U64) return SS_ERR_INVALID_ARG;
  const int vbytes = op == SS_OP_HISTOGRAM ? 0 : op == SS_OP_COLLECT_REDUCE ? 8 : (vt == SS_U32 ? 4 : 8);
  // temporaries hold (key, value) records aligned to 16, 8 or 4 bytes by size
  const size_t ralign = std::max(kbytes == 16 ? 16 : kbytes, vbytes);
  const size_t recbytes = (kbytes + vbytes + ralign - 1) / ralign * ralign;
  return plan_workspace(op, kbytes, vbytes, recbytes, kbytes <= 8, n, opt, nsm, P, num_inst);
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
// Caller arrays are accessed element by element: each needs its element's alignment.
bool aligned_to(const void* p, size_t bytes) { return (reinterpret_cast<uintptr_t>(p) & (bytes - 1)) == 0; }

struct Range {
  uintptr_t a, b;
};
bool overlap(Range x, Range y) { return x.a < y.b && y.a < x.b; }

thread_local int g_launches = 0;

std::mutex g_timer_mu;
PhaseTimer g_timer;
bool g_timer_ready = false;

PhaseTimer* timer_for(const ss_options* opt, cudaStream_t st) {
  if (!opt || !(opt->flags & SS_FLAG_PHASE_TIMING)) return nullptr;
  std::lock_guard<std::mutex> g(g_timer_mu);
  if (!g_timer_ready) {
    for (int i = 0; i <= PhaseTimer::kMax; ++i) cudaEventCreate(&g_timer.ev[i]);
    g_timer_ready = true;
  }
  g_timer.on = true;
  g_timer.start(st);
  return &g_timer;
}

// vt: 0 = u32 values, 1 = u64 values, 2 = keys only.
cudaError_t dispatch(int op, int kt, int vt, const Plan& P, const Work& w, cudaStream_t st, PhaseTimer* tm) {
  g_launches = 0;
  LaunchCfg c{num_sms(), tm, &g_launches};
  switch (kt) {
    case SS_U32: return run_u32(op, vt, P, w, st, c);
    case SS_U64: return run_u64(op, vt, P, w, st, c);
    case SS_U128: return run_u128(op, vt, P, w, st, c);
    default: return cudaErrorNotSupported;
  }
}

ss_status semisort_common(int op, ss_type kt, ss_type vt, const void* keys, const void* vals,
                          void* keys_out, void* vals_out, uint64_t n, void* ws, size_t ws_bytes,
                          const ss_options* opt, ss_stream_t stream, const uint64_t* d_offsets = nullptr,
                          uint32_t num_inst = 0) {
  if (num_inst > 0 && !d_offsets) return SS_ERR_INVALID_ARG;
  // semisort_< on hash buckets (SS_FLAG_HASH_BUCKETS): the semisort_= pipeline
  // with a sorting base case
  const bool hash_less = op == kOpLess && opt && (opt->flags & SS_FLAG_HASH_BUCKETS);
  if (hash_less) op = kOpEqual;
  if (n == 0) return SS_OK;
  if (!keys || !keys_out || !ws) return SS_ERR_INVALID_ARG;
  if ((vals == nullptr) != (vals_out == nullptr)) return SS_ERR_INVALID_ARG;
  {
    const size_t ka = (size_t)kbytes_of(kt), va = vt == SS_U32 ? 4 : 8;
    if (!ka) return SS_ERR_INVALID_ARG;
    if (!aligned_to(keys, ka) || !aligned_to(keys_out, ka) || !aligned16(ws) || (vals && !aligned_to(vals, va)) ||
        (vals_out && !aligned_to(vals_out, va)) || (d_offsets && !aligned_to(d_offsets, 8)))
      return SS_ERR_INVALID_ARG;
  }
  Plan P;
  ss_status s = make_plan(op, kt, vt, n, opt, num_sms(), &P, num_inst);
  if (s != SS_OK) return s;
  if (ws_bytes < P.total) return SS_ERR_WORKSPACE_TOO_SMALL;
  const size_t kb = n * P.kbytes, vb = n * (vt == SS_U32 ? 4 : 8);
  Range rk{(uintptr_t)keys, (uintptr_t)keys + kb}, rko{(uintptr_t)keys_out, (uintptr_t)keys_out + kb};
  Range rw{(uintptr_t)ws, (uintptr_t)ws + P.total};
  if (overlap(rk, rko) && keys != keys_out) return SS_ERR_INVALID_ARG;
  if (overlap(rw, rk) || overlap(rw, rko)) return SS_ERR_INVALID_ARG;
  if (vals) {
    Range rv{(uintptr_t)vals, (uintptr_t)vals + vb}, rvo{(uintptr_t)vals_out, (uintptr_t)vals_out + vb};
    if (overlap(rv, rvo) && vals != vals_out) return SS_ERR_INVALID_ARG;
    if (overlap(rw, rv) || overlap(rw, rvo)) return SS_ERR_INVALID_ARG;
    if (overlap(rk, rv) || overlap(rk, rvo) || overlap(rko, rv) || overlap(rko, rvo)) return SS_ERR_INVALID_ARG;
    if ((keys == keys_out) != (vals == vals_out)) return SS_ERR_INVALID_ARG;
  }
  if (opt && (opt->splitter_mode < 0 || opt->splitter_mode > 1)) return SS_ERR_INVALID_ARG;
  Work w;
  memset(&w, 0, sizeof(w));
  fill_work(P, ws, &w);
  w.seed = opt ? opt->seed : 0;
  w.in_k = keys;
  w.in_v = vals;
  w.out_k = keys_out;
  w.out_v = vals_out;
  w.has_vals = vals != nullptr;
  w.splitter_mode = (op == kOpLess && opt && kt != SS_U128) ? (uint32_t)opt->splitter_mode : 0u;
  w.offsets = d_offsets;
  w.less_base = hash_less ? 1u : 0u;
  w.swap = (opt && (opt->flags & SS_FLAG_SWAP_OUTPUT)) ? 1u : 0u;
  w.auto_nl = (opt && opt->n_light_log2) ? 0u : 1u;
  w.ident = (opt && (opt->flags & SS_FLAG_IDENTITY_HASH) && kt != SS_U128) ? 1u : 0u;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  PhaseTimer* tm = timer_for(opt, st);
  cudaError_t e = dispatch(op, kt, vals ? (int)vt : 2, P, w, st, tm);
  if (e == cudaErrorNotSupported) return SS_ERR_UNSUPPORTED;
  return e == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

// collect-reduce (vals != NULL) and histogram (vals == NULL, counts in sums).
ss_status reduce_common(int op, ss_type kt, const void* keys, const uint64_t* vals, void* ukeys, void* sums,
                        uint64_t capacity, uint64_t* d_num_unique, uint64_t n, void* ws, size_t ws_bytes,
                        const ss_options* opt, ss_stream_t stream, const uint64_t* d_offsets = nullptr,
                        uint32_t num_inst = 0, uint64_t* d_out_offsets = nullptr) {
  if (!d_num_unique || (reinterpret_cast<uintptr_t>(d_num_unique) & 7)) return SS_ERR_INVALID_ARG;
  if (num_inst > 0 && (!d_offsets || !d_out_offsets || (reinterpret_cast<uintptr_t>(d_out_offsets) & 7)))
    return SS_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int kb1 = kbytes_of(kt);
  if (!kb1) return SS_ERR_INVALID_ARG;
  if (n == 0) {
    if (ws && aligned16(ws) && ws_bytes >= sizeof(Ctrl)) {
      if (cudaMemsetAsync(ws, 0, sizeof(Ctrl), st) != cudaSuccess) return SS_ERR_CUDA;
    }
    const size_t cnt = num_inst > 0 ? num_inst : 1;
    if (cudaMemsetAsync(d_num_unique, 0, 8 * cnt, st) != cudaSuccess) return SS_ERR_CUDA;
    if (num_inst > 0 && cudaMemsetAsync(d_out_offsets, 0, 8 * (cnt + 1), st) != cudaSuccess) return SS_ERR_CUDA;
    return SS_OK;
  }
  if (!keys || !ukeys || !sums || !ws) return SS_ERR_INVALID_ARG;
  if (op == kOpReduce && !vals) return SS_ERR_INVALID_ARG;
  if (!aligned_to(keys, kb1) || !aligned_to(ukeys, kb1) || !aligned_to(sums, op == kOpReduce ? 8 : 4) ||
      !aligned16(ws) || (vals && !aligned_to(vals, 8)) || (d_offsets && !aligned_to(d_offsets, 8)))
    return SS_ERR_INVALID_ARG;
  Plan P;
  ss_status s = make_plan(op, kt, SS_U64, n, opt, num_sms(), &P, num_inst);
  if (s != SS_OK) return s;
  if (ws_bytes < P.total) return SS_ERR_WORKSPACE_TOO_SMALL;
  const uint64_t sb = op == kOpReduce ? 8 : 4;
  Range rk{(uintptr_t)keys, (uintptr_t)keys + n * kb1};
  Range rv{(uintptr_t)vals, (uintptr_t)vals + (vals ? n * 8 : 0)};
  Range ru{(uintptr_t)ukeys, (uintptr_t)ukeys + capacity * kb1};
  Range rs{(uintptr_t)sums, (uintptr_t)sums + capacity * sb};
  Range rw{(uintptr_t)ws, (uintptr_t)ws + P.total};
  Range rn{(uintptr_t)d_num_unique, (uintptr_t)d_num_unique + 8 * (num_inst > 0 ? num_inst : 1)};
  const Range outs[3] = {ru, rs, rn};
  for (const Range& o : outs) {
    if (overlap(o, rk) || overlap(o, rw) || (vals && overlap(o, rv))) return SS_ERR_INVALID_ARG;
  }
  if (overlap(ru, rs) || overlap(ru, rn) || overlap(rs, rn)) return SS_ERR_INVALID_ARG;
  if (overlap(rw, rk) || (vals && overlap(rw, rv))) return SS_ERR_INVALID_ARG;
  Work w;
  memset(&w, 0, sizeof(w));
  fill_work(P, ws, &w);
  w.seed = opt ? opt->seed : 0;
  w.in_k = keys;
  w.in_v = vals;
  w.out_k = ukeys;
  w.out_v = nullptr;
  w.has_vals = vals != nullptr;
  w.sums_out = sums;
  w.num_unique = d_num_unique;
  w.out_capacity = capacity;
  w.offsets = d_offsets;
  w.inst_off_out = d_out_offsets;
  w.auto_nl = (opt && opt->n_light_log2) ? 0u : 1u;
  w.ident = (opt && (opt->flags & SS_FLAG_IDENTITY_HASH) && kt != SS_U128) ? 1u : 0u;
  PhaseTimer* tm = timer_for(opt, st);
  cudaError_t e = dispatch(op, kt, op == kOpReduce ? (int)SS_U64 : 2, P, w, st, tm);
  if (e == cudaErrorNotSupported) return SS_ERR_UNSUPPORTED;
  return e == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

__global__ void k_hash_u64(const uint64_t* k, uint64_t* o, uint64_t n, uint64_t salt) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    o[i] = mix64(k[i] ^ salt);
}

}  // namespace

extern "C" {

ss_status ss_workspace_size(int op, ss_type key_type, ss_type val_type, uint64_t n, const ss_options* opt,
                            size_t* bytes) {
  if (!bytes) return SS_ERR_INVALID_ARG;
  if (op < 0 || op > 3) return SS_ERR_INVALID_ARG;
  if (op == SS_OP_SEMISORT_LESS && opt && (opt->flags & SS_FLAG_HASH_BUCKETS)) op = SS_OP_SEMISORT_EQUAL;
  Plan P;
  ss_status s = make_plan(op, key_type, val_type, n, opt, num_sms(), &P);
  if (s != SS_OK) return s;
  *bytes = P.total;
  return SS_OK;
}

ss_status semisort_equal(ss_type key_type, ss_type val_type, const void* keys, const void* vals, void* keys_out,
                         void* vals_out, uint64_t n, void* ws, size_t ws_bytes, const ss_options* opt,
                         ss_stream_t stream) {
  return semisort_common(kOpEqual, key_type, val_type, keys, vals, keys_out, vals_out, n, ws, ws_bytes, opt,
                         stream);
}

ss_status semisort_less(ss_type key_type, ss_type val_type, const void* keys, const void* vals, void* keys_out,
                        void* vals_out, uint64_t n, void* ws, size_t ws_bytes, const ss_options* opt,
                        ss_stream_t stream) {
  return semisort_common(kOpLess, key_type, val_type, keys, vals, keys_out, vals_out, n, ws, ws_bytes, opt,
                         stream);
}

ss_status collect_reduce(ss_type key_type, const void* keys, const uint64_t* vals, void* ukeys_out,
                         uint64_t* sums_out, uint64_t capacity, uint64_t* d_num_unique, uint64_t n, void* ws,
                         size_t ws_bytes, const ss_options* opt, ss_stream_t stream) {
  if (n && !vals) return SS_ERR_INVALID_ARG;
  return reduce_common(kOpReduce, key_type, keys, vals, ukeys_out, sums_out, capacity, d_num_unique, n, ws,
                       ws_bytes, opt, stream);
}

ss_status histogram(ss_type key_type, const void* keys, void* ukeys_out, uint32_t* counts_out, uint64_t capacity,
                    uint64_t* d_num_unique, uint64_t n, void* ws, size_t ws_bytes, const ss_options* opt,
                    ss_stream_t stream) {
  return reduce_common(kOpHist, key_type, keys, nullptr, ukeys_out, counts_out, capacity, d_num_unique, n, ws,
                       ws_bytes, opt, stream);
}

ss_status ss_workspace_size_batched(int op, ss_type key_type, ss_type val_type, uint64_t n, uint32_t num_instances,
                                    const ss_options* opt, size_t* bytes) {
  if (!bytes || op < 0 || op > 3 || num_instances == 0) return SS_ERR_INVALID_ARG;
  if (op == SS_OP_SEMISORT_LESS && opt && (opt->flags & SS_FLAG_HASH_BUCKETS)) op = SS_OP_SEMISORT_EQUAL;
  Plan P;
  ss_status s = make_plan(op, key_type, val_type, n, opt, num_sms(), &P, num_instances);
  if (s != SS_OK) return s;
  *bytes = P.total;
  return SS_OK;
}

ss_status semisort_equal_batched(ss_type key_type, ss_type val_type, const void* keys, const void* vals,
                                 void* keys_out, void* vals_out, const uint64_t* d_offsets, uint32_t num_instances,
                                 uint64_t n, void* ws, size_t ws_bytes, const ss_options* opt, ss_stream_t stream) {
  if (num_instances == 0) return SS_ERR_INVALID_ARG;
  return semisort_common(kOpEqual, key_type, val_type, keys, vals, keys_out, vals_out, n, ws, ws_bytes, opt,
                         stream, d_offsets, num_instances);
}

ss_status semisort_less_batched(ss_type key_type, ss_type val_type, const void* keys, const void* vals,
                                void* keys_out, void* vals_out, const uint64_t* d_offsets, uint32_t num_instances,
                                uint64_t n, void* ws, size_t ws_bytes, const ss_options* opt, ss_stream_t stream) {
  if (num_instances == 0) return SS_ERR_INVALID_ARG;
  return semisort_common(kOpLess, key_type, val_type, keys, vals, keys_out, vals_out, n, ws, ws_bytes, opt,
                         stream, d_offsets, num_instances);
}

ss_status collect_reduce_batched(ss_type key_type, const void* keys, const uint64_t* vals,
                                 const uint64_t* d_offsets, uint32_t num_instances, uint64_t n, void* ukeys_out,
                                 uint64_t* sums_out, uint64_t capacity, uint64_t* d_num_unique,
                                 uint64_t* d_out_offsets, void* ws, size_t ws_bytes, const ss_options* opt,
                                 ss_stream_t stream) {
  if (num_instances == 0 || (n && !vals)) return SS_ERR_INVALID_ARG;
  return reduce_common(kOpReduce, key_type, keys, vals, ukeys_out, sums_out, capacity, d_num_unique, n, ws,
                       ws_bytes, opt, stream, d_offsets, num_instances, d_out_offsets);
}

ss_status histogram_batched(ss_type key_type, const void* keys, const uint64_t* d_offsets, uint32_t num_instances,
                            uint64_t n, void* ukeys_out, uint32_t* counts_out, uint64_t capacity,
                            uint64_t* d_num_unique, uint64_t* d_out_offsets, void* ws, size_t ws_bytes,
                            const ss_options* opt, ss_stream_t stream) {
  if (num_instances == 0) return SS_ERR_INVALID_ARG;
  return reduce_common(kOpHist, key_type, keys, nullptr, ukeys_out, counts_out, capacity, d_num_unique, n, ws,
                       ws_bytes, opt, stream, d_offsets, num_instances, d_out_offsets);
}

ss_status ss_last_device_error(void* ws, ss_stream_t stream, int* code) {
  if (!ws || !code) return SS_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Ctrl* c = reinterpret_cast<Ctrl*>(ws);
  uint32_t v = 0;
  if (cudaMemcpyAsync(&v, &c->error, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return SS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SS_ERR_CUDA;
  if (cudaMemsetAsync(&c->error, 0, 4, st) != cudaSuccess) return SS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SS_ERR_CUDA;
  *code = (int)v;
  return SS_OK;
}

int ss_get_stats(void* ws, ss_stream_t stream, uint64_t* out, int count) {
  if (!ws || !out || count <= 0) return 0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Ctrl h;
  if (cudaMemcpyAsync(&h, ws, sizeof(Ctrl), cudaMemcpyDeviceToHost, st) != cudaSuccess) return 0;
  if (cudaStreamSynchronize(st) != cudaSuccess) return 0;
  const int m = std::min(count, 16);
  for (int i = 0; i < m; ++i) out[i] = h.stats[i];
  return m;
}

int ss_phase_times(float* ms, const char** names, int max) {
  std::lock_guard<std::mutex> g(g_timer_mu);
  if (!g_timer_ready || !g_timer.on) return 0;
  const int m = std::min(max, g_timer.count);
  if (m <= 0) return 0;
  cudaEventSynchronize(g_timer.ev[g_timer.count]);
  for (int i = 0; i < m; ++i) {
    float t = 0;
    cudaEventElapsedTime(&t, g_timer.ev[i], g_timer.ev[i + 1]);
    if (ms) ms[i] = t;
    if (names) names[i] = g_timer.name[i];
  }
  return m;
}

int ss_kernel_launches(void) { return g_launches; }

const char* ss_status_string(ss_status s) {
  switch (s) {
    case SS_OK: return "ok";
    case SS_ERR_INVALID_ARG: return "invalid argument";
    case SS_ERR_UNSUPPORTED: return "unsupported type or size";
    case SS_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case SS_ERR_CAPACITY: return "capacity exceeded";
    case SS_ERR_NOMEM: return "not enough device memory";
    case SS_ERR_TIMEOUT: return "device wait timed out";
    case SS_ERR_CUDA: return "CUDA runtime error";
    case SS_ERR_DEPTH: return "recursion depth limit reached";
  }
  return "unknown status";
}

ss_status ss_hash_u64(const uint64_t* keys, uint64_t* out, uint64_t n, uint64_t salt, ss_stream_t stream) {
  if (n == 0) return SS_OK;
  if (!keys || !out) return SS_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const uint64_t blocks = std::min<uint64_t>((n + 255) / 256, 65535);
  k_hash_u64<<<(unsigned)blocks, 256, 0, st>>>(keys, out, n, salt);
  return cudaGetLastError() == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// semisort_equal_noalloc: semisort_= whose scratch space is a file-scope
// device array of this translation unit instead of a caller workspace.
// ---------------------------------------------------------------------------
namespace {

constexpr uint64_t kNoAllocMaxN = 1ull << 18;      // records per call
constexpr size_t kNoAllocBytes = 24ull << 20;      // every plan of kNoAllocMaxN u32/u64 keys; 128-bit keys need alpha >= 256

static __device__ __align__(256) unsigned char g_noalloc_ws[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};

// Device address of the array on the current device, looked up once per device.
ss_status noalloc_workspace(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SS_ERR_CUDA;
  if (dev < 0 || dev >= 64) return SS_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_ws) != cudaSuccess || p == nullptr) return SS_ERR_CUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return SS_OK;
}

}  // namespace

extern "C" ss_status semisort_equal_noalloc(ss_type key_type, ss_type val_type, const void* keys, const void* vals,
                                            void* keys_out, void* vals_out, uint64_t n, const ss_options* opt,
                                            ss_stream_t stream) {
  if (n > kNoAllocMaxN) return SS_ERR_UNSUPPORTED;
  if (n == 0) return SS_OK;
  void* ws = nullptr;
  const ss_status s = noalloc_workspace(&ws);
  if (s != SS_OK) return s;
  // Phase timing creates CUDA events, so this entry point ignores that flag.
  ss_options o;
  memset(&o, 0, sizeof(o));
  if (opt) o = *opt;
  o.flags &= ~SS_FLAG_PHASE_TIMING;
  // The device error flag lives inside the static array, where a caller of
  // this entry point cannot read it.  Hash bucketing cannot exhaust the
  // recursion levels at these sizes, but identity bucketing can (keys that
  // differ only in bits above those the levels consume), so this entry point
  // always buckets by the hash.
  o.flags &= ~SS_FLAG_IDENTITY_HASH;
  // Nothing in the array has to start at zero: the pipeline's first kernel
  // resets the control block, and every other region is written before it is read.
  return semisort_common(kOpEqual, key_type, val_type, keys, vals, keys_out, vals_out, n, ws, kNoAllocBytes, &o,
                         stream);
}

// ---------------------------------------------------------------------------
// The learned-splitter model on its own (test and inspection entry points).
// ---------------------------------------------------------------------------
extern "C" size_t ss_mlp_workspace_size(void) { return sizeof(LearnState); }

namespace {

// The trainer's dynamic shared memory limit, raised once per device.
bool learn_train_ready() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  std::lock_guard<std::mutex> g(mu);
  if (!done[dev]) {
    if (cudaFuncSetAttribute(k_learn_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem)) !=
        cudaSuccess)
      return false;
    done[dev] = true;
  }
  return true;
}

ss_status mlp_setup(const float* d_params, const float* d_x, const float* d_t, uint32_t m, void* ws, size_t ws_bytes,
                    cudaStream_t st, LearnState** out) {
  if (!ws || !aligned16(ws) || ws_bytes < sizeof(LearnState)) return SS_ERR_WORKSPACE_TOO_SMALL;
  if (m > (uint32_t)(kGradCTAsMax * kGradPts)) return SS_ERR_UNSUPPORTED;
  LearnState* L = reinterpret_cast<LearnState*>(ws);
  if (d_params && cudaMemcpyAsync(L->p, d_params, sizeof(float) * kMlpParams, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return SS_ERR_CUDA;
  if (m && (cudaMemcpyAsync(L->x, d_x, sizeof(float) * m, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(L->t, d_t, sizeof(float) * m, cudaMemcpyDeviceToDevice, st) != cudaSuccess))
    return SS_ERR_CUDA;
  if (cudaMemsetAsync(L->m, 0, sizeof(float) * 2 * kMlpParams, st) != cudaSuccess) return SS_ERR_CUDA;
  *out = L;
  return SS_OK;
}

}  // namespace

extern "C" ss_status ss_mlp_loss_grad(const float* d_params, const float* d_x, const float* d_t, uint32_t m,
                                      float* d_out, void* ws, size_t ws_bytes, ss_stream_t stream) {
  if (!d_params || !d_x || !d_t || !d_out || m == 0) return SS_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  LearnState* L = nullptr;
  ss_status s = mlp_setup(d_params, d_x, d_t, m, ws, ws_bytes, st, &L);
  if (s != SS_OK) return s;
  k_learn_range<<<1, 32, 0, st>>>(L, 0, 1, m);
  k_learn_step<<<(m + kGradPts - 1) / kGradPts, kGradThreads, 0, st>>>(L, 0, 0.0f);
  if (cudaMemcpyAsync(d_out, L->grad, sizeof(float) * (kMlpParams + 1), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return SS_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

extern "C" ss_status ss_mlp_train(const float* d_x, const float* d_t, uint32_t m, const float* d_params0,
                                  uint32_t steps, float lr, float* d_params_out, float* d_loss_out, void* ws,
                                  size_t ws_bytes, ss_stream_t stream) {
  if (!d_x || !d_t || !d_params0 || !d_params_out || m == 0) return SS_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  LearnState* L = nullptr;
  ss_status s = mlp_setup(d_params0, d_x, d_t, m, ws, ws_bytes, st, &L);
  if (s != SS_OK) return s;
  k_learn_range<<<1, 32, 0, st>>>(L, 0, 1, m);
  const uint32_t ctas = (m + kGradPts - 1) / kGradPts;
  if (steps) {
    if (!learn_train_ready()) return SS_ERR_CUDA;
    k_learn_train<<<kTrainCTAs, kTrainThreads, sizeof(TrainSmem), st>>>(L, steps, lr, 0);
  }
  k_learn_step<<<ctas, kGradThreads, 0, st>>>(L, 0, 0.0f);  // loss at the final parameters
  if (cudaMemcpyAsync(d_params_out, L->p, sizeof(float) * kMlpParams, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return SS_ERR_CUDA;
  if (d_loss_out &&
      cudaMemcpyAsync(d_loss_out, &L->grad[kMlpParams], sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return SS_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}

extern "C" ss_status ss_mlp_invert(const float* d_params, ss_type key_type, uint64_t kmin, uint64_t kmax,
                                   uint32_t n_light_log2, void* d_splitters, void* ws, size_t ws_bytes,
                                   ss_stream_t stream) {
  if (!d_params || !d_splitters || kmax < kmin) return SS_ERR_INVALID_ARG;
  if (n_light_log2 < 1 || n_light_log2 > (uint32_t)kLessTopLog2) return SS_ERR_UNSUPPORTED;
  if (key_type != SS_U32 && key_type != SS_U64) return SS_ERR_UNSUPPORTED;
  if (key_type == SS_U32 && kmax > 0xFFFFFFFFull) return SS_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  LearnState* L = nullptr;
  ss_status s = mlp_setup(d_params, nullptr, nullptr, 0, ws, ws_bytes, st, &L);
  if (s != SS_OK) return s;
  k_learn_range<<<1, 32, 0, st>>>(L, kmin, kmax, 0);
  const uint32_t nl = 1u << n_light_log2;
  if (key_type == SS_U32)
    k_learn_invert<uint32_t><<<(nl + 255) / 256, 256, 0, st>>>(L, nullptr, n_light_log2);
  else
    k_learn_invert<uint64_t><<<(nl + 255) / 256, 256, 0, st>>>(L, nullptr, n_light_log2);
  const size_t kb = key_type == SS_U32 ? 4 : 8;
  if (cudaMemcpyAsync(d_splitters, L->splitters, kb * (nl - 1), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return SS_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? SS_OK : SS_ERR_CUDA;
}
