// Host-side workspace plan of the semisort pipeline: capacities and offsets
// of every device work list inside the caller's workspace, and the Work
// descriptor that points the kernels at them.  Shared by the C ABI and the
// C++ template entry points.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "../../include/semisort.h"
#include "ss_learn.cuh"
#include "ss_plan.h"

namespace ss {

constexpr uint64_t kMaxN = (1ull << 32) - (1ull << 20);
constexpr uint32_t kAlphaMax = 4096;  // records one refine CTA holds (kRefMax)

inline size_t al(size_t x) { return (x + 255) & ~size_t(255); }

inline uint32_t ceil_log2(uint64_t x) {
  uint32_t b = 0;
  while ((1ull << b) < x) ++b;
  return b;
}

// Capacities and offsets of every device work list for n records (see
// ss_plan.h), for keys of kbytes bytes and values of vbytes bytes held in
// temporaries of recbytes-byte records.  `integral`: keys are unsigned
// integers of at most 8 bytes (the semisort_< top level may then use its wide
// bucket space and lookup table).
inline ss_status plan_workspace(int op, int kbytes, int vbytes, size_t recbytes, bool integral, uint64_t n,
                                const ss_options* opt, int nsm, Plan* P, uint32_t num_inst = 0) {
  memset(P, 0, sizeof(*P));
  const bool batched = num_inst > 0;
  P->num_inst = num_inst;
  P->n = n;
  P->op = op;
  P->kbytes = kbytes;
  P->vbytes = vbytes;
  if (kbytes <= 0) return SS_ERR_INVALID_ARG;
  if (n >= kMaxN) return SS_ERR_UNSUPPORTED;
  if (nsm <= 0) nsm = 152;
  uint32_t alpha = (opt && opt->alpha) ? opt->alpha : kAlphaMax;
  alpha = std::min(std::max(alpha, 64u), kAlphaMax);
  P->alpha = alpha;
  // top-level light buckets: n_L ~ 2n / alpha, at most 2^9 hash buckets or 2^11
  // semisort_< key ranges
  // (semisort_< with 16-byte keys keeps the narrow top level: 2^8 ranges)
  const bool wide = op == SS_OP_SEMISORT_LESS && integral && !batched;
  const uint32_t lb_max = wide ? (uint32_t)kLessTopLog2
                               : op == SS_OP_SEMISORT_LESS ? (uint32_t)kMaxLightLog2 - 1 : (uint32_t)kMaxLightLog2;
  uint32_t lb1 = 0;
  if (opt && opt->n_light_log2)
    lb1 = std::min<uint32_t>(std::max<uint32_t>(opt->n_light_log2, 1), lb_max);
  else
    lb1 = std::min<uint32_t>(std::max<uint32_t>(ceil_log2((2 * n + alpha - 1) / alpha), 1), lb_max);
  P->lbits1 = lb1;
  uint64_t l1 = (n + 2 * (uint64_t)nsm - 1) / (2 * (uint64_t)nsm);
  l1 = ((l1 + 4095) / 4096) * 4096;
  l1 = std::max<uint64_t>(l1, 32768);
  P->l1 = (uint32_t)std::min<uint64_t>(l1, 1u << 31);
  uint32_t l2 = (opt && opt->subarray) ? opt->subarray : 32768;
  l2 = std::max<uint32_t>(((l2 + 4095) / 4096) * 4096, 4096);
  P->l2 = l2;
  // batched calls: subarrays of `subarray` records (default 2^18) at level 0 too
  if (batched) P->l1 = (opt && opt->subarray) ? l2 : (1u << 18);
  uint32_t s1 = (opt && opt->sample_size) ? opt->sample_size : 16384;
  uint32_t p2 = 2048;
  while (p2 < s1 && p2 < 16384) p2 <<= 1;
  s1 = p2;
  if (P->kbytes > 8) s1 = std::min<uint32_t>(s1, 8192);
  P->s1 = s1;
  P->s2 = 8192;
  const bool less = op == SS_OP_SEMISORT_LESS;
  const bool red = op == SS_OP_COLLECT_REDUCE || op == SS_OP_HISTOGRAM;
  // level 0: one segment; bucket rows per segment are n_L + n_H,cap (hash
  // buckets) or 4 n_L (semisort_<: 2q + 1 ids for q < 2 n_L boundaries)
  const uint32_t nl0 = 1u << lb1;
  const uint32_t rows0 = less ? 4 * nl0 : nl0 + std::min<uint32_t>(nl0, kMaxHeavy);
  P->seg_cap[0] = 1;
  P->tile_cap[0] = (uint32_t)((n + P->l1 - 1) / P->l1);
  P->bucket_cap[0] = rows0;
  P->c_cap[0] = (uint64_t)rows0 * P->tile_cap[0];
  if (batched) {
    // one segment per instance above alpha; each has n_L < 4m/alpha + 2 and at
    // most 2 n_L (4 n_L for semisort_<) bucket rows, and m/l + 1 subarrays
    P->seg_cap[0] = num_inst;
    P->tile_cap[0] = (uint32_t)((n + P->l1 - 1) / P->l1 + num_inst);
    P->bucket_cap[0] = (uint32_t)((less ? 16 : 8) * n / alpha + 8ull * num_inst + 64);
    P->c_cap[0] = (uint64_t)kMaxBuckets * P->tile_cap[0];
  }
  for (int l = 1; l < kMaxLevels; ++l) {
    const uint64_t segs = n / (alpha + 1) + 1;
    P->seg_cap[l] = (uint32_t)segs;
    P->tile_cap[l] = (uint32_t)((n + l2 - 1) / l2 + segs);
    // a segment of m > alpha records has n_L < 4m/alpha + 2 light buckets, so
    // its rows (at most 2 n_L, or 4 n_L for semisort_<) sum over the segments
    // (fewer than n/alpha of them) to below 12n/alpha (24n/alpha)
    P->bucket_cap[l] = (uint32_t)((less ? 24 : 12) * n / alpha + 64);
    // rows x subarrays: sum over segments of rows * (m/l2 + 1)
    P->c_cap[l] = (uint64_t)kMaxBuckets * ((n + l2 - 1) / l2) + P->bucket_cap[l];
  }
  uint64_t items = n / kCopyChunk + 16 + num_inst;
  for (int l = 0; l < kMaxLevels; ++l) items += P->bucket_cap[l];
  P->item_cap = (uint32_t)std::min<uint64_t>(items, 0xFFFFFFF0ull);
  // layout: control block first, so status calls can find it without a plan
  size_t o = al(sizeof(Ctrl));
  // temporaries T and T2 hold records (key, value) as array of structures;
  // semisort_= / semisort_< with SS_FLAG_SWAP_OUTPUT swap T with the output
  // arrays instead of using T2 (Sec. 3.4); collect-reduce / histogram always
  // need T (compacted base-case outputs)
  const bool multi = n > alpha;  // (batched: some instance may exceed alpha)
  const bool need_t = multi || red;
  const bool swap = !red && opt && (opt->flags & SS_FLAG_SWAP_OUTPUT);
  P->off_tk = o;
  o = al(o + (need_t ? n * recbytes : 0));
  P->off_tv = o;
  P->off_t2k = o;
  o = al(o + (multi && !swap ? n * recbytes : 0));
  P->off_t2v = o;
  for (int l = 0; l < kMaxLevels; ++l) {
    if (!multi) {
      P->seg_cap[l] = P->tile_cap[l] = P->bucket_cap[l] = 0;
      P->c_cap[l] = 0;
    }
    P->off_segs[l] = o;
    o = al(o + (size_t)P->seg_cap[l] * sizeof(Seg));
    P->off_tiles[l] = o;
    o = al(o + (size_t)P->tile_cap[l] * sizeof(Tile));
    P->off_C[l] = o;
    o = al(o + (size_t)P->c_cap[l] * 4);
    P->off_hkeys[l] = o;
    o = al(o + (size_t)P->bucket_cap[l] * P->kbytes);
    P->off_htab[l] = o;
    o = al(o + (size_t)P->bucket_cap[l] * 4);
    P->off_bsize[l] = o;
    o = al(o + (size_t)P->bucket_cap[l] * 4);
    P->off_boff[l] = o;
    o = al(o + (size_t)P->bucket_cap[l] * 4);
    P->off_hpart[l] = o;
    o = al(o + (op == SS_OP_COLLECT_REDUCE ? (size_t)P->c_cap[l] * 8 : 0));
    P->off_split[l] = o;
    o = al(o + (less ? (size_t)P->bucket_cap[l] * P->kbytes : 0));
    // key-cell tables of the narrow semisort_< levels: 2 n_L + 1 cells per
    // segment within its 4 n_L bucket rows (two u16 per row)
    P->off_lcell[l] = o;
    o = al(o + (less && integral ? (size_t)P->bucket_cap[l] * 4 : 0));
  }
  if (!multi) P->item_cap = std::max<uint32_t>(1, num_inst);
  P->off_items = o;
  o = al(o + (size_t)P->item_cap * sizeof(Item));
  P->off_item_out = o;
  o = al(o + (red ? (size_t)P->item_cap * 8 : 0));
  P->off_item_pos = o;
  o = al(o + (red ? (size_t)P->item_cap * 8 : 0));
  P->off_block_sums = o;
  o = al(o + (red ? ((size_t)P->item_cap / 4096 + 2) * 8 : 0));
  P->off_item_aux = o;
  o = al(o + (op == SS_OP_COLLECT_REDUCE ? (size_t)P->item_cap * 8 : 0));
  P->off_scratch32 = o;
  o = al(o + (op == SS_OP_HISTOGRAM ? (size_t)n * 4 : 0));
  // the 2^16-key sample and the learned-splitter state: the wide semisort_<
  // top level, and batched semisort_< of integer keys (learned mode)
  const bool learn_space = less && integral && multi;
  P->off_bigs = o;
  o = al(o + (learn_space ? (size_t)kBigSample * P->kbytes : 0));
  P->off_bigs_tmp = o;
  o = al(o + (learn_space ? (size_t)kBigSample * P->kbytes : 0));
  P->off_learn = o;
  o = al(o + (learn_space ? sizeof(LearnState) : 0));
  P->off_toptab = o;
  o = al(o + (wide && multi ? sizeof(TopTable) : 0));
  P->off_inst_base = o;
  o = al(o + (batched && red ? (size_t)kItemClasses * num_inst * 8 : 0));
  P->off_inst_first = o;
  o = al(o + (batched && red ? (size_t)kItemClasses * num_inst * 8 : 0));
  P->off_ctrl = 0;
  P->total = o;
  return SS_OK;
}

inline void fill_work(const Plan& P, void* ws, Work* w) {
  char* b = static_cast<char*>(ws);
  w->n = P.n;
  w->alpha = P.alpha;
  w->l1 = P.l1;
  w->l2 = P.l2;
  w->lbits1 = P.lbits1;
  w->s1 = P.s1;
  w->s2 = P.s2;
  w->op = P.op;
  w->t_k = b + P.off_tk;
  w->t_v = b + P.off_tv;
  w->t2_k = b + P.off_t2k;
  w->t2_v = b + P.off_t2v;
  for (int l = 0; l < kMaxLevels; ++l) {
    w->segs[l] = reinterpret_cast<Seg*>(b + P.off_segs[l]);
    w->tiles[l] = reinterpret_cast<Tile*>(b + P.off_tiles[l]);
    w->C[l] = reinterpret_cast<uint32_t*>(b + P.off_C[l]);
    w->hkeys[l] = b + P.off_hkeys[l];
    w->htab[l] = reinterpret_cast<uint16_t*>(b + P.off_htab[l]);
    w->bsize[l] = reinterpret_cast<uint32_t*>(b + P.off_bsize[l]);
    w->boff[l] = reinterpret_cast<uint32_t*>(b + P.off_boff[l]);
    w->hpart[l] = reinterpret_cast<uint64_t*>(b + P.off_hpart[l]);
    w->splitters[l] = b + P.off_split[l];
    w->lcell[l] = reinterpret_cast<uint16_t*>(b + P.off_lcell[l]);
    w->seg_cap[l] = P.seg_cap[l];
    w->tile_cap[l] = P.tile_cap[l];
    w->c_cap[l] = P.c_cap[l];
    w->bucket_cap[l] = P.bucket_cap[l];
  }
  w->items = reinterpret_cast<Item*>(b + P.off_items);
  w->item_cap = P.item_cap;
  w->item_out = reinterpret_cast<uint64_t*>(b + P.off_item_out);
  w->item_pos = reinterpret_cast<uint64_t*>(b + P.off_item_pos);
  w->block_sums = reinterpret_cast<uint64_t*>(b + P.off_block_sums);
  w->item_aux = reinterpret_cast<uint64_t*>(b + P.off_item_aux);
  w->scratch32 = reinterpret_cast<uint32_t*>(b + P.off_scratch32);
  w->bigs = b + P.off_bigs;
  w->bigs_tmp = b + P.off_bigs_tmp;
  w->learn = b + P.off_learn;
  w->toptab = reinterpret_cast<TopTable*>(b + P.off_toptab);
  w->inst_base = reinterpret_cast<uint64_t*>(b + P.off_inst_base);
  w->inst_first = reinterpret_cast<uint64_t*>(b + P.off_inst_first);
  w->num_inst = P.num_inst > 0 ? P.num_inst : 1;
  w->ctrl = reinterpret_cast<Ctrl*>(b + P.off_ctrl);
}


}  // namespace ss
