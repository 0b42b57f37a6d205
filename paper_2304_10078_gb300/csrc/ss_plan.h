// Work descriptors and the workspace plan shared by host and device code.
//
// The recursion of Algorithm 1 is run level by level.  Level l holds a list
// of segments (subproblems, the light buckets of level l-1 that exceed the
// base-case threshold alpha); each segment is cut into subarrays ("tiles",
// the blocks of size l in Sec. 3.2).  All lists live in the caller's
// workspace and are built on the device, so the host never waits for them.
#pragma once
#include <stddef.h>
#include <stdint.h>

namespace ss {

constexpr int kMaxLevels = 6;          // recursion levels (Algorithm 1) before the depth error
constexpr int kMaxLightLog2 = 9;       // n_L <= 512 per segment
constexpr uint32_t kMaxHeavy = 512;    // heavy keys per segment
constexpr uint32_t kMaxBuckets = 1024; // n_L + heavy: bucket ids fit two 5-bit rank passes
constexpr uint32_t kCopyChunk = 1u << 16;  // records per copy item
// semisort_< top level: up to 2^12 key ranges (4095 splitters) cut from a
// 2^16-key sample; with up to 512 heavy equality buckets the q < 4608
// boundaries give 2q + 1 < 9217 bucket ids, ranked in three 5-bit passes.
constexpr int kLessTopLog2 = 12;
constexpr uint32_t kBigBounds = (1u << kLessTopLog2) + kMaxHeavy;
constexpr uint32_t kBigBuckets = 2 * kBigBounds + 16;
constexpr uint32_t kBigSample = 1u << 16;
// Batched semisort_< in learned mode: one CDF model for all instances, trained
// on a 2^16-key sample of the whole batch and inverted at 2^8 ranges (the
// largest range count of a narrow level); an instance with 2^l ranges takes
// every 2^(8 - l)-th splitter.
constexpr int kBatchLearnLog2 = 8;

// Operations.
enum Op : int { kOpEqual = 0, kOpLess = 1, kOpReduce = 2, kOpHist = 3 };

// Buffer ids used by work items.
enum Buf : uint32_t { kBufIn = 0, kBufT = 1, kBufOut = 2, kBufT2 = 3 };

// Lookup table of the wide semisort_< top level: boundary search ranges per
// key cell.  Cell c covers the keys kmin + [c, c + 1) * 2^shift (keys below kmin
// fall in cell 0, keys above the last cell in cell kTopCells - 1); boundaries
// cell[c] .. cell[c + 1] - 1 lie inside cell c.
constexpr uint32_t kTopCells = 4096;
struct TopTable {
  uint64_t kmin;
  uint32_t shift;
  uint32_t q;
  uint16_t cell[kTopCells + 1];
};

// Finish items of a batched call's instances of at most alpha records carry
// this level tag (they go straight to the base case).
constexpr uint32_t kDirectLevel = kMaxLevels;
// Item classes of a batched call's output placement: direct items, then one
// per distribution level.
constexpr uint32_t kItemClasses = kMaxLevels + 1;

// Finish-item kinds.
enum ItemKind : uint32_t { kItemRefine = 0, kItemCopy = 1, kItemHeavyOut = 2 };

struct Seg {
  uint64_t start;      // first record of the segment (same index space in every buffer)
  uint32_t len;        // records
  uint32_t ntiles;     // subarrays
  uint32_t first_tile; // index of the first subarray in the level's tile list
  uint32_t bbase;      // base of the segment's bucket rows / heavy table (capacity nbcap)
  uint64_t cbase;      // base of the segment's count matrix (nbcap x ntiles, bucket-major)
  uint32_t lbits;      // log2 n_L
  uint32_t nh;         // heavy keys found by sampling (semisort_<: splitter boundaries)
  uint32_t nbcap;      // bucket-id capacity of the segment
  uint32_t fin_off;    // first finish item emitted by this segment
  uint32_t next_off;   // first next-level segment emitted by this segment
  uint32_t cnt_fin;    // finish items emitted
  uint32_t cnt_next;   // next-level segments emitted
  uint32_t nb;         // bucket ids in use
  uint64_t mult;       // odd multiplier of this segment's bucketing hash
  uint32_t shift;      // identity hashing: first key bit of this segment's light-bucket id
  uint32_t ident;      // bucket ids from the key's own bits (identity hash)
  uint32_t nl;         // light buckets n_L (a power of two, or 768)
  uint32_t cbits;      // semisort_<, integer keys: log2 of the key-cell table's cells (0: no table)
};

struct Tile {
  uint64_t start;  // first record
  uint32_t len;    // records
  uint32_t seg;    // owning segment
  uint32_t idx;    // subarray index within the segment
  uint32_t pad;
};

struct Item {
  uint64_t start;   // first record
  uint32_t len;     // records
  uint32_t kind;    // ItemKind
  uint32_t buf;     // buffer holding the records (Buf)
  uint32_t aux;     // heavy-output: segment; otherwise 0
  uint32_t aux2;    // heavy-output: heavy index; otherwise 0
  uint32_t level;   // level that emitted the item
};

// Control block (device).
struct Ctrl {
  uint32_t nsegs[kMaxLevels];
  uint32_t ntiles[kMaxLevels];
  uint32_t nfin;       // finish items so far
  uint32_t error;      // first device-side ss_status (0 = none)
  uint64_t stats[16];  // see ss_get_stats
};

// Everything a kernel needs: workspace pointers + problem constants.
struct Work {
  // problem
  uint64_t n;
  uint32_t alpha;      // base-case threshold
  uint32_t l1, l2;     // subarray size at level 1 / levels >= 2
  uint32_t lbits1;     // log2 n_L at level 1
  uint32_t s1, s2;     // sample size caps at level 1 / levels >= 2
  uint32_t op;
  uint32_t ident;      // identity hash for integer keys (bucket ids from the key's own bits)
  uint32_t less_base;  // semisort_< with hash buckets: sort each base case
  uint32_t swap;       // semisort: levels alternate between T and the output arrays (no T2)
  uint32_t auto_nl;    // top-level n_L chosen by size (no n_light_log2 option)
  uint32_t out_cap;    // collect-reduce / histogram capacity (clamped)
  uint64_t seed;
  // user buffers
  const void* in_k;
  const void* in_v;
  void* out_k;
  void* out_v;
  int has_vals;
  // workspace buffers
  void* t_k;
  void* t_v;
  void* t2_k;
  void* t2_v;
  Seg* segs[kMaxLevels];
  Tile* tiles[kMaxLevels];
  uint32_t* C[kMaxLevels];
  void* hkeys[kMaxLevels];       // heavy keys (sorted), per segment at bbase
  uint16_t* htab[kMaxLevels];    // heavy hash table: heavy index or 0xFFFF, per segment at 2*bbase (4 hcap slots)
  uint32_t* bsize[kMaxLevels];   // bucket totals
  uint32_t* boff[kMaxLevels];    // bucket offsets within segment
  uint64_t* hpart[kMaxLevels];   // collect-reduce heavy partials (nbcap x ntiles layout, rows >= n_L)
  uint32_t seg_cap[kMaxLevels];
  uint32_t tile_cap[kMaxLevels];
  uint64_t c_cap[kMaxLevels];
  uint32_t bucket_cap[kMaxLevels];
  Item* items;
  uint32_t item_cap;
  uint64_t* item_out;   // per item: outputs produced (collect-reduce / histogram)
  uint64_t* item_pos;   // per item: exclusive prefix of item_out
  uint64_t* block_sums; // scratch for the device-wide scan
  uint64_t* num_unique; // user pointer (collect-reduce / histogram)
  void* sums_out;       // user pointer: u64 sums or u32 counts
  void* splitters[kMaxLevels];  // semisort_<: per-segment sorted boundaries at bbase
  uint16_t* lcell[kMaxLevels];  // semisort_<, integer keys: per-segment key-cell tables at 2*bbase
  void* bigs;           // semisort_<: the sorted top-level sample (kBigSample keys)
  void* bigs_tmp;       // its sorted runs before the merge
  void* learn;          // semisort_<: learned-splitter state (LearnState)
  TopTable* toptab;     // semisort_<: lookup table of the wide top level
  uint32_t splitter_mode;  // 0 sampled, 1 learned (semisort_< top level)
  // batched calls: instance i holds records [offsets[i], offsets[i+1])
  const uint64_t* offsets;  // device, num_inst + 1 entries; null for a single instance
  uint32_t num_inst;
  uint64_t* inst_base;      // collect-reduce / histogram: per (class, instance) output base (kItemClasses x num_inst)
  uint64_t* inst_first;     // per (class, instance) first item position in the item scan
  uint64_t* inst_off_out;   // user: num_inst + 1 output offsets
  uint32_t* scratch32;  // histogram: per-position counts of compacted base cases
  uint64_t* item_aux;   // collect-reduce: heavy totals per item
  uint64_t out_capacity;
  Ctrl* ctrl;
};

// Host-side plan of workspace capacities and offsets.
struct Plan {
  uint64_t n;
  int op, kbytes, vbytes;
  uint32_t alpha, l1, l2, lbits1, s1, s2;
  uint32_t seg_cap[kMaxLevels], tile_cap[kMaxLevels], bucket_cap[kMaxLevels];
  uint64_t c_cap[kMaxLevels];
  uint32_t item_cap;
  size_t off_tk, off_tv, off_t2k, off_t2v;
  size_t off_segs[kMaxLevels], off_tiles[kMaxLevels], off_C[kMaxLevels], off_hkeys[kMaxLevels],
      off_htab[kMaxLevels], off_bsize[kMaxLevels], off_boff[kMaxLevels], off_hpart[kMaxLevels],
      off_split[kMaxLevels], off_lcell[kMaxLevels];
  size_t off_items, off_item_out, off_item_pos, off_block_sums, off_ctrl, off_scratch32, off_item_aux;
  size_t off_bigs, off_bigs_tmp, off_learn, off_inst_base, off_inst_first, off_toptab;
  uint32_t num_inst;
  size_t total;
};

}  // namespace ss
