/*
 * semisort.h -- C ABI of the GB300 (sm_103a) semisort library.
 *
 * Implements the problems of Sec. 2.1 of Dong, Wu, Wang, Dhulipala, Gu, Sun,
 * "High-Performance and Flexible Parallel Algorithms for Semisort and Related
 * Problems" (SPAA 2023), with the three-step method of Sec. 3 (Algorithm 1):
 * Sampling and Bucketing, Blocked Distributing, Local Refining.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Records are given as two separate device arrays (structure of arrays):
 *    keys[n] and vals[n].  Key types: SS_U32, SS_U64, SS_U128 (16 bytes,
 *    little-endian lo then hi, ordered as an unsigned 128-bit integer).  Value
 *    types: SS_U32, SS_U64.
 *  - All pointers are DEVICE pointers owned by the caller.  Key, value and
 *    output arrays need the alignment of their element type (4, 8 or 16
 *    bytes); the workspace must be 16-byte aligned.
 *    The library never allocates device memory: scratch space comes from the
 *    caller's workspace `ws` of `ws_bytes` bytes, sized by
 *    ss_workspace_size() for the same (op, types, n, options).
 *  - Calls are asynchronous and stream ordered on `stream` (0 = legacy
 *    default stream).  No call synchronizes with the host; every size that
 *    steers the recursion stays on the device, so a call can be captured in a
 *    CUDA graph.  Workspace and outputs must not be shared by calls that may
 *    run concurrently.
 *  - Return values report argument errors found on the host at enqueue time.
 *    Failures found on the device (an internal capacity limit, the recursion
 *    depth limit of six levels) set a flag in the workspace; ss_last_device_error() reads
 *    and clears it.  Each call resets the flag when it starts, so the flag
 *    describes the most recent call on that workspace.  No kernel traps.
 *  - n = 0 is valid and enqueues nothing.  n must be below 2^32 - 2^20
 *    (SS_ERR_UNSUPPORTED otherwise): offsets inside a subproblem are 32-bit,
 *    which halves the count-matrix traffic; with 16-byte records, input,
 *    output and the two temporaries of 2^32 records would need 256 GB.
 *  - Determinism: for a fixed options.seed every output is bit-identical
 *    across runs (the method is race-free, Sec. 2.2 and Sec. 3).
 */
#ifndef SEMISORT_H_
#define SEMISORT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ss_stream_t; /* same type as cudaStream_t */

typedef enum {
  SS_OK = 0,
  SS_ERR_INVALID_ARG = 1,         /* null/misaligned pointer, bad type, overlap */
  SS_ERR_UNSUPPORTED = 2,         /* type combination or size not supported */
  SS_ERR_WORKSPACE_TOO_SMALL = 3, /* ws_bytes below ss_workspace_size() */
  SS_ERR_CAPACITY = 4,            /* more unique keys than the output capacity */
  SS_ERR_NOMEM = 5,               /* request exceeds free device memory */
  SS_ERR_TIMEOUT = 6,             /* reserved: no kernel of this library waits on another */
  SS_ERR_CUDA = 7,                /* a CUDA runtime call failed */
  SS_ERR_DEPTH = 8                /* recursion deeper than the level limit */
} ss_status;

typedef enum { SS_U32 = 0, SS_U64 = 1, SS_U128 = 2 } ss_type;

/* Operation codes for ss_workspace_size(). */
typedef enum {
  SS_OP_SEMISORT_EQUAL = 0,
  SS_OP_SEMISORT_LESS = 1,
  SS_OP_COLLECT_REDUCE = 2,
  SS_OP_HISTOGRAM = 3
} ss_op;

/* Tunables; a zero field means "choose automatically".
 *   seed          seeds sampling and the per-level hash salts (Sec. 3.1).
 *   subarray      records per subarray l at recursion levels >= 2 (Sec. 3.2).
 *   n_light_log2  log2 of the light-bucket count n_L at the top level.
 *   alpha         base-case threshold: largest bucket one CTA refines (Sec. 3.3).
 *   sample_size   samples per top-level subproblem |S|.
 *   splitter_mode 0 = sampled splitters, 1 = learned splitters (semisort_less).
 *   flags         SS_FLAG_* bits. */
typedef struct {
  uint64_t seed;
  uint32_t subarray;
  uint32_t n_light_log2;
  uint32_t alpha;
  uint32_t sample_size;
  int32_t splitter_mode;
  int32_t flags;
} ss_options;

#define SS_FLAG_PHASE_TIMING 0x1 /* record per-kernel CUDA events (ss_phase_times) */
/* Integer keys (u32, u64) bucketed by their own bits instead of a hash: the
 * lowest bits at the top level, the next ones at each deeper level (the
 * "-i" variants of Sec. 4.1).  Same results; fast for keys whose low bits are
 * spread, slow (deep recursion, SS_ERR_DEPTH) for keys that share them.
 * Ignored for 128-bit keys and by semisort_< with range buckets. */
#define SS_FLAG_IDENTITY_HASH 0x2
/* semisort_less only: the paper's semisort_< -- hash buckets (as
 * semisort_equal) whose base cases are sorted by key -- instead of the range
 * partition.  Equal keys are contiguous and in input order, but groups are not
 * in key order (the semisort_equal contract). */
#define SS_FLAG_HASH_BUCKETS 0x4
/* semisort_equal / semisort_less (and their batched forms): one temporary
 * array instead of two.  The distribution levels alternate between the
 * temporary and the caller's output arrays -- the swap of A and T of Sec. 3.4
 * -- so the workspace is about half as large (17.6 GB instead of 33.6 GB for
 * 10^9 u64/u64 records).  Same results; the levels that write the output
 * arrays write keys and values separately, which costs time. */
#define SS_FLAG_SWAP_OUTPUT 0x8

/* Bytes of workspace needed by `op` on n records with the given types and
 * options (NULL = defaults).  Returns SS_ERR_UNSUPPORTED for unsupported type
 * combinations or sizes. */
ss_status ss_workspace_size(int op, ss_type key_type, ss_type val_type, uint64_t n,
                            const ss_options* opt, size_t* bytes);

/* semisort_= (Sec. 2.1; Algorithm 1 with the hash-table base case of Sec. 3.3).
 * Reorders the n records so that records with equal keys are contiguous;
 * records of one key keep their input order (stable).  The order of the key
 * groups is unspecified but fixed for a given options.seed.
 * keys_out/vals_out may equal keys/vals (in place); partial overlap is an
 * error.  vals may be NULL together with vals_out (keys only). */
ss_status semisort_equal(ss_type key_type, ss_type val_type, const void* keys, const void* vals,
                         void* keys_out, void* vals_out, uint64_t n, void* ws, size_t ws_bytes,
                         const ss_options* opt, ss_stream_t stream);

/* semisort_< as a range-partitioned variant: buckets are key ranges cut by
 * sample splitters (heavy keys get their own equality buckets), and each base
 * case is a stable comparison sort (Sec. 3.3), so the output equals the
 * stable sort of the input by key.  Arguments as semisort_equal. */
ss_status semisort_less(ss_type key_type, ss_type val_type, const void* keys, const void* vals,
                        void* keys_out, void* vals_out, uint64_t n, void* ws, size_t ws_bytes,
                        const ss_options* opt, ss_stream_t stream);

/* collect-reduce (Sec. 2.1, Sec. 3.5) with the map M(r) = value and the monoid
 * (+ mod 2^64, 0).  Writes one (unique key, sum) pair per distinct key into
 * ukeys_out/sums_out (capacity entries each) and the number of distinct keys
 * into *d_num_unique (device pointer).  If that number exceeds capacity, the
 * count is still written, only the first `capacity` outputs are stored and the
 * device flag SS_ERR_CAPACITY is raised.  Output
 * order is unspecified but fixed for a given seed. */
ss_status collect_reduce(ss_type key_type, const void* keys, const uint64_t* vals, void* ukeys_out,
                         uint64_t* sums_out, uint64_t capacity, uint64_t* d_num_unique, uint64_t n,
                         void* ws, size_t ws_bytes, const ss_options* opt, ss_stream_t stream);

/* histogram (Sec. 2.1): collect-reduce with M(r) = 1, counts as uint32. */
ss_status histogram(ss_type key_type, const void* keys, void* ukeys_out, uint32_t* counts_out,
                    uint64_t capacity, uint64_t* d_num_unique, uint64_t n, void* ws,
                    size_t ws_bytes, const ss_options* opt, ss_stream_t stream);

/* semisort_= without a workspace argument and without allocating anything.
 * The paper has no counterpart: this entry point exists for callers that must
 * not allocate device memory at the time of the call and have no workspace to
 * hand over -- for instance code running under a fixed device-memory budget
 * that another framework's caching allocator has already taken, or a loop that
 * cannot afford the device-wide synchronization cudaMalloc may cause.
 * Scratch space is one static device array of 24 MiB inside the library,
 * shared by every call on a device; it keeps whatever the last call left in it.
 * Limits and behaviour:
 *  - n <= 262144 (2^18) records; larger n returns SS_ERR_UNSUPPORTED.  Options
 *    whose plan would not fit the array (ss_workspace_size() above 24 MiB, which
 *    only 128-bit keys with alpha below 256 reach) return
 *    SS_ERR_WORKSPACE_TOO_SMALL.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) and remembers it; make that first call before any
 *    stream capture begins.
 *  - Calls that may overlap in time (different streams or host threads without
 *    ordering between them) race on the shared array and give wrong results;
 *    order them on one stream or synchronize between them.
 *  - SS_FLAG_PHASE_TIMING and SS_FLAG_IDENTITY_HASH are ignored: keys are
 *    always bucketed by the hash, which cannot exhaust the recursion levels at
 *    these sizes (identity bucketing can, on keys that differ only in high
 *    bits).  A device-side failure would set the flag inside the internal
 *    array, where callers cannot read it.
 * Other arguments, output and errors as semisort_equal. */
ss_status semisort_equal_noalloc(ss_type key_type, ss_type val_type, const void* keys,
                                 const void* vals, void* keys_out, void* vals_out, uint64_t n,
                                 const ss_options* opt, ss_stream_t stream);

/* The learned-splitter model on its own.  semisort_less with
 * options.splitter_mode = 1 fits a monotone CDF model to the light (non-heavy)
 * keys of its 2^16-key top-level sample and inverts it into the top level's
 * splitters (a gain in load balance only: bucketing stays exact key
 * comparison).  Heavy keys keep their own equality buckets.  Training runs
 * every Adam step in one launch of a cluster of 8 CTAs and stops on a loss
 * plateau.  The model is a 1-32-32-1
 * perceptron in FP32 with softplus-positive weights and logistic hidden units;
 * SS_MLP_PARAMS parameters laid out v1[32] | c1[32] | v2[32*32] (row j: the
 * weights into hidden unit j of layer 2) | c2[32] | v3[32] | c3, with weights
 * w = softplus(v).  Inputs are keys normalized to [0, 1]; targets are ranks
 * divided by the sample size.  Each entry point needs a device workspace of
 * ss_mlp_workspace_size() bytes (16-byte aligned) and is stream-ordered. */
#define SS_MLP_PARAMS 1153
size_t ss_mlp_workspace_size(void);

/* Mean squared error over m <= 4096 points (x[m], t[m], device floats) and its
 * gradient with respect to the parameters: d_out[0..1153) = gradient,
 * d_out[1153] = loss.  Sums run in a fixed order (deterministic). */
ss_status ss_mlp_loss_grad(const float* d_params, const float* d_x, const float* d_t, uint32_t m,
                           float* d_out, void* ws, size_t ws_bytes, ss_stream_t stream);

/* `steps` full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, learning
 * rate lr) from d_params0; writes the trained parameters and the loss at them. */
ss_status ss_mlp_train(const float* d_x, const float* d_t, uint32_t m, const float* d_params0,
                       uint32_t steps, float lr, float* d_params_out, float* d_loss_out, void* ws,
                       size_t ws_bytes, ss_stream_t stream);

/* Splitter j (1 <= j < 2^n_light_log2, n_light_log2 <= 11): the smallest key k
 * in [kmin, kmax] with f((k - kmin) / (kmax - kmin)) >= j / 2^n_light_log2 (kmax if
 * none), by bisection over the integer keys, f evaluated in FP32.  Keys SS_U32
 * or SS_U64; d_splitters receives 2^n_light_log2 - 1 keys. */
ss_status ss_mlp_invert(const float* d_params, ss_type key_type, uint64_t kmin, uint64_t kmax,
                        uint32_t n_light_log2, void* d_splitters, void* ws, size_t ws_bytes,
                        ss_stream_t stream);

/* Batched forms: num_instances independent problems over one concatenation of
 * records.  d_offsets (device, num_instances + 1 entries) gives instance i the
 * records [d_offsets[i], d_offsets[i+1]); it must start at 0, end at n and not
 * decrease (otherwise the device flag reports SS_ERR_INVALID_ARG and nothing is
 * written).  All instances run in one pipeline: instances of at most alpha
 * records go straight to the base case, larger ones become the top level's
 * segments, so one call enqueues the same fixed kernel sequence whatever the
 * instance sizes (and can be captured in a CUDA graph).  Workspace:
 * ss_workspace_size_batched().  options.subarray also sets the top level's
 * subarray size (default 2^18 records).  options.splitter_mode = 1 with
 * semisort_less_batched and 32- or 64-bit keys: one CDF model is trained on a
 * 2^16-key sample of the whole batch (light keys only) and inverted at 2^8
 * ranges; every instance above alpha judges the model's splitters against
 * those of its own sample (the model's are kept unless their largest range
 * bucket exceeds twice the light keys' share and the sampled splitters'
 * largest); ss_get_stats entry 12 counts the instances that kept them.
 * Results are the same either way. */
ss_status ss_workspace_size_batched(int op, ss_type key_type, ss_type val_type, uint64_t n,
                                    uint32_t num_instances, const ss_options* opt, size_t* bytes);

/* semisort_= of every instance within its own range of keys_out/vals_out. */
ss_status semisort_equal_batched(ss_type key_type, ss_type val_type, const void* keys, const void* vals,
                                 void* keys_out, void* vals_out, const uint64_t* d_offsets,
                                 uint32_t num_instances, uint64_t n, void* ws, size_t ws_bytes,
                                 const ss_options* opt, ss_stream_t stream);

/* semisort_< (stable sort by key) of every instance within its own range. */
ss_status semisort_less_batched(ss_type key_type, ss_type val_type, const void* keys, const void* vals,
                                void* keys_out, void* vals_out, const uint64_t* d_offsets,
                                uint32_t num_instances, uint64_t n, void* ws, size_t ws_bytes,
                                const ss_options* opt, ss_stream_t stream);

/* collect-reduce of every instance: instance i's (unique key, sum) pairs occupy
 * ukeys_out/sums_out[d_out_offsets[i] .. d_out_offsets[i+1]) (device, num_instances
 * + 1 entries) and d_num_unique[i] (device, num_instances entries) is their number.
 * capacity bounds the total; beyond it nothing is stored and the device flag
 * reports SS_ERR_CAPACITY (the counts and offsets are still written). */
ss_status collect_reduce_batched(ss_type key_type, const void* keys, const uint64_t* vals,
                                 const uint64_t* d_offsets, uint32_t num_instances, uint64_t n,
                                 void* ukeys_out, uint64_t* sums_out, uint64_t capacity,
                                 uint64_t* d_num_unique, uint64_t* d_out_offsets, void* ws,
                                 size_t ws_bytes, const ss_options* opt, ss_stream_t stream);

/* histogram of every instance, laid out as collect_reduce_batched. */
ss_status histogram_batched(ss_type key_type, const void* keys, const uint64_t* d_offsets,
                            uint32_t num_instances, uint64_t n, void* ukeys_out, uint32_t* counts_out,
                            uint64_t capacity, uint64_t* d_num_unique, uint64_t* d_out_offsets, void* ws,
                            size_t ws_bytes, const ss_options* opt, ss_stream_t stream);

/* Reads (and clears) the device error flag left in `ws` by earlier calls on
 * `stream`; synchronizes the stream.  *code receives the ss_status of the
 * first device-side failure (SS_OK if none). */
ss_status ss_last_device_error(void* ws, ss_stream_t stream, int* code);

/* Per-call statistics kept in the workspace by the last call (synchronizes the
 * stream).  out[0..count) receives, in order: levels used, records distributed
 * at levels 1, 2, 3 and 4-6 (4 entries), records refined, records copied, heavy keys at
 * level 1, largest refined bucket, refine items, records whose bucket was all
 * distinct keys, splitters of the semisort_< top level (0 sampled, 1 learned,
 * 2 learned but rejected on the sample or not usable), the largest top-level
 * range bucket's count in the 2^16-key sample (batched learned mode: the
 * instances that kept the model's splitters), the largest top-level light
 * bucket in records, the semisort_< top level's n_L, and the Adam steps the
 * learned-splitter training ran (it stops early on a loss plateau).
 * Returns the number of entries written (at most 16). */
int ss_get_stats(void* ws, ss_stream_t stream, uint64_t* out, int count);

/* Per-kernel timings (milliseconds) of the last call made with
 * SS_FLAG_PHASE_TIMING; names[i] receives a static string.  Synchronizes.
 * Returns the number of phases written (at most max). */
int ss_phase_times(float* ms, const char** names, int max);

/* Number of kernels the most recent semisort / collect-reduce / histogram call
 * on this host thread enqueued (0 before any call). */
int ss_kernel_launches(void);

/* Human-readable name of a status code (static storage). */
const char* ss_status_string(ss_status s);

/* The library's fixed 64-bit key hash (the SplitMix64 output mixer applied to
 * key XOR salt), applied on the device to n keys: out[i] = mix(keys[i] ^ salt).
 * Exposed so that tests can compare it with an independent statement of the
 * published function. */
ss_status ss_hash_u64(const uint64_t* keys, uint64_t* out, uint64_t n, uint64_t salt,
                      ss_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SEMISORT_H_ */
