"""Semisort across the ranks of a process group (one rank per GPU).

The records are split into contiguous slices, one per rank.  The sharded
form partitions them with one exchange step, following the three steps of
the method (Sec. 3): Sampling and Bucketing over the union of the slices,
the counting matrix of Blocked Distributing with one row per rank, and the
distribution itself as one all-to-all of records; Local Refining is the
library's single-GPU call on each rank's share.

1. Sample: every rank draws a share of a global sample proportional to its
   slice size (seeded positions); the samples are all-gathered, so every rank
   derives the same plan: heavy keys (sample count >= tau) and, for
   semisort_<, splitters cut from the light sample keys.
2. Bucket: every record gets a bucket id (hash bucket or heavy bucket for
   semisort_=, collect-reduce and histogram; range or equality bucket for
   semisort_<, ids increasing with the key).
3. Count: per-rank bucket counts are all-gathered; every rank computes the
   same owner map -- buckets in id order, cut into G contiguous ranges of
   about n / G records.  A light bucket goes whole to one owner; a heavy
   bucket (one key) may be split at record granularity between consecutive
   owners, so skewed inputs stay balanced.
4. Exchange: each rank orders its records stably by bucket, which groups them
   by owner in owner order, and one all-to-all moves them.  A receiver gets
   the chunks of ranks 0..G-1 in rank order, so records of one key arrive in
   global input order.
5. Refine locally: semisort_< is the stable sort of the received records;
   semisort_= groups them, with the (at most two) heavy keys shared with a
   neighbouring owner placed first or last so that each key stays one run in
   the concatenated output; collect-reduce and histogram pre-reduce heavy keys
   on the sending rank (a (key, partial) pair travels instead of the records)
   and reduce the received records and partials.

Concatenated in rank order, the outputs of all ranks are the single-GPU
results for the concatenated input (same contract: semisort_< equals the
stable sort, semisort_= groups stably, collect-reduce / histogram give each
distinct key once).  Host-side control works on small arrays (samples,
per-bucket counts); the bulk record work is done by `local`, an object with
the single-device operations (`GpuLocal` runs the library's kernels).
"""
from __future__ import annotations

from dataclasses import dataclass

import torch
import torch.distributed as dist

MASK64 = (1 << 64) - 1


def _i64(x: int) -> int:
    """A u64 value as the int64 with the same bits."""
    x &= MASK64
    return x - (1 << 64) if x >= 1 << 63 else x


@dataclass
class Plan:
    """The partition every rank derives from the all-gathered sample."""
    op: str
    heavy: torch.Tensor        # int64 views of the heavy keys, ascending in u64 order
    bounds: torch.Tensor       # semisort_<: boundaries (splitters and heavy keys), ascending in u64 order
    bflags: torch.Tensor       # semisort_<: 1 where the boundary is a heavy key
    light_bits: int            # hash buckets: log2 of the light-bucket count
    nbuckets: int              # bucket ids are 0 .. nbuckets - 1
    salt: int


def _flip(x: torch.Tensor) -> torch.Tensor:
    """int64 views of u64 values mapped so that signed order is u64 order."""
    return x ^ (-(1 << 63))


def _counts(ids: torch.Tensor, nb: int) -> torch.Tensor:
    return torch.bincount(ids, minlength=nb).to(torch.int64) if ids.numel() else torch.zeros(nb, dtype=torch.int64)


def make_plan(op: str, keys: torch.Tensor, group, local, seed: int = 1, samples: int = 1 << 14,
              buckets_per_rank: int = 64) -> Plan:
    """Sampling and Bucketing over the union of the slices (identical result
    on every rank).  keys: this rank's int64 views of u64 keys."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    n_loc = torch.tensor([keys.numel()], dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n_loc, group=group)
    sizes = [int(s.item()) for s in sizes]
    n = sum(sizes)
    # this rank's share of the sample, at seeded positions of its slice
    share = (samples * keys.numel() + n - 1) // n if n else 0
    if keys.numel() and share:
        ctr = torch.arange(share, dtype=torch.int64, device=keys.device) + (rank << 32)
        h = local.hash64(ctr, _i64(seed * 0x9E3779B97F4A7C15 + 1)).to(keys.device)
        pos = (h & 0x7FFFFFFFFFFFFFFF) % keys.numel()
        mine = keys[pos].cpu()
    else:
        mine = torch.zeros(0, dtype=torch.int64)
    got = [None] * world
    dist.all_gather_object(got, mine.tolist(), group=group)
    sample = torch.tensor([v for part in got for v in part], dtype=torch.int64)
    s = sample.numel()
    nl_total = max(2, world * buckets_per_rank)
    light_bits = max(1, (nl_total - 1).bit_length())
    tau = max(2, s // (1 << light_bits)) if s else 2
    # heavy keys: sample count >= tau, ascending in u64 order
    if s:
        order = torch.argsort(_flip(sample), stable=True)
        srt = sample[order]
        uniq, cnt = torch.unique_consecutive(srt, return_counts=True)
        heavy = uniq[cnt >= tau]
        light = srt[torch.repeat_interleave(cnt < tau, cnt)]
    else:
        heavy = torch.zeros(0, dtype=torch.int64)
        light = torch.zeros(0, dtype=torch.int64)
    salt = _i64(seed * 0xD1B54A32D192ED03 + 7)
    if op == "less":
        q = 1 << light_bits
        spl = light[(torch.arange(1, q, dtype=torch.int64) * light.numel()) // q] if light.numel() else \
            torch.zeros(0, dtype=torch.int64)
        allb = torch.cat([spl, heavy])
        ub = torch.unique(_flip(allb))  # ascending, duplicates removed
        bounds = _flip(ub)
        bflags = torch.isin(bounds, heavy).to(torch.int64)
        return Plan(op, heavy, bounds, bflags, light_bits, 2 * bounds.numel() + 1, salt)
    return Plan(op, heavy, torch.zeros(0, dtype=torch.int64), torch.zeros(0, dtype=torch.int64), light_bits,
                (1 << light_bits) + heavy.numel(), salt)


def bucket_ids(keys: torch.Tensor, plan: Plan, local) -> torch.Tensor:
    """Bucket id of every key (int64 views) under the plan."""
    if keys.numel() == 0:
        return torch.zeros(0, dtype=torch.int64)
    if plan.op == "less":
        fk = _flip(keys)
        fb = _flip(plan.bounds)
        u = torch.searchsorted(fb, fk, right=True)
        prev = torch.clamp(u - 1, min=0)
        eq = (u > 0) & (plan.bflags[prev] == 1) & (plan.bounds[prev] == keys) if plan.bounds.numel() else \
            torch.zeros_like(u, dtype=torch.bool)
        return torch.where(eq, 2 * u - 1, 2 * u)
    nl = 1 << plan.light_bits
    h = local.hash64(keys, plan.salt)
    ids = (h >> (64 - plan.light_bits)) & (nl - 1)
    if plan.heavy.numel():
        fh = _flip(plan.heavy)
        j = torch.clamp(torch.searchsorted(fh, _flip(keys)), max=plan.heavy.numel() - 1)
        hit = plan.heavy[j] == keys
        ids = torch.where(hit, nl + j, ids)
    return ids


def is_heavy_bucket(plan: Plan, b: torch.Tensor) -> torch.Tensor:
    if plan.op == "less":
        return (b & 1) == 1
    return b >= (1 << plan.light_bits)


def owner_map(plan: Plan, counts: torch.Tensor, world: int, split_heavy: bool):
    """counts: (world, nbuckets) per-rank bucket counts (identical on every
    rank).  Returns (start, per_rank_off, owner, split): the global first
    position of every bucket, the offset of each rank's records inside it,
    the owner of every unsplit bucket, and a mask of buckets split between
    owners (heavy buckets only, when split_heavy)."""
    tot = counts.sum(dim=0)
    n = int(tot.sum().item())
    start = torch.cumsum(tot, 0) - tot
    per_rank_off = torch.cumsum(counts, 0) - counts
    target = max(1, -(-n // world))
    centre = start + tot // 2
    owner = torch.clamp(centre // target, max=world - 1)
    heavy = is_heavy_bucket(plan, torch.arange(counts.shape[1], dtype=torch.int64))
    first = torch.clamp(start // target, max=world - 1)
    last = torch.clamp((start + torch.clamp(tot - 1, min=0)) // target, max=world - 1)
    split = heavy & (first != last) & (tot > 0) if split_heavy else torch.zeros_like(heavy)
    return start, per_rank_off, owner, split, target


def _exchange(group, world, dest: torch.Tensor, *cols):
    """Records already ordered by destination rank: one all-to-all per column.
    Returns the received columns (chunks of ranks 0..world-1 in rank order)."""
    send = torch.bincount(dest, minlength=world).to(torch.int64) if dest.numel() else \
        torch.zeros(world, dtype=torch.int64)
    recv = torch.zeros(world, dtype=torch.int64)
    dist.all_to_all_single(recv, send, group=group)
    out = []
    for c in cols:
        r = torch.empty(int(recv.sum().item()), dtype=c.dtype)
        dist.all_to_all_single(r, c.contiguous(), output_split_sizes=recv.tolist(),
                               input_split_sizes=send.tolist(), group=group)
        out.append(r)
    return out, recv


def _route(keys, plan, group, local, world, rank, split_heavy):
    """Bucket ids, stable order by bucket and destination rank of every local
    record, from the all-gathered counting matrix."""
    ids = bucket_ids(keys, plan, local)
    cnt = _counts(ids, plan.nbuckets)
    rows = [torch.zeros_like(cnt) for _ in range(world)]
    dist.all_gather(rows, cnt, group=group)
    counts = torch.stack(rows)
    start, off, owner, split, target = owner_map(plan, counts, world, split_heavy)
    order = local.stable_order(ids)
    ids_s = ids[order]
    # position of each record among this rank's records of its bucket
    first_of = torch.cumsum(cnt, 0) - cnt
    j = torch.arange(ids_s.numel(), dtype=torch.int64) - first_of[ids_s]
    gpos = start[ids_s] + off[rank][ids_s] + j
    dest = torch.where(split[ids_s], torch.clamp(gpos // target, max=world - 1), owner[ids_s])
    return ids_s, order, dest, split, owner, start, target


def sharded_semisort(op: str, keys: torch.Tensor, vals: torch.Tensor, group, local, seed: int = 1,
                     samples: int = 1 << 14, buckets_per_rank: int = 64):
    """semisort_= (op 'equal') or semisort_< (op 'less') across the group.
    keys / vals: int64 views of this rank's u64 slice.  Returns this rank's
    share of the output; concatenated in rank order the shares are the
    output for the concatenated input."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    plan = make_plan(op, keys, group, local, seed, samples, buckets_per_rank)
    ids_s, order, dest, split, owner, start, target = _route(keys, plan, group, local, world, rank, True)
    (rk, rv, rb), recv = _exchange(group, world, dest, keys[order], vals[order], ids_s)
    if op == "less":
        return local.semisort_less(rk, rv)
    # semisort_=: a split heavy key shared with the previous owner goes first,
    # one shared with the next owner last
    lo, hi = rank * target, (rank + 1) * target
    head = split[rb] & (start[rb] < lo)
    tail = split[rb] & ~head
    mid = ~(head | tail)
    mk, mv = local.semisort_equal(rk[mid], rv[mid]) if int(mid.sum()) else (rk[mid], rv[mid])
    del hi
    return torch.cat([rk[head], mk, rk[tail]]), torch.cat([rv[head], mv, rv[tail]])


def sharded_reduce(op: str, keys: torch.Tensor, vals: torch.Tensor | None, group, local, seed: int = 1,
                   samples: int = 1 << 14, buckets_per_rank: int = 64):
    """collect-reduce (op 'reduce', u64 wraparound sums) or histogram (op
    'hist', counts) across the group.  Heavy keys are reduced on the sending
    rank; each owner reduces what it receives.  Returns this rank's
    (unique keys, sums or counts); every distinct key appears on exactly one
    rank."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    if vals is None:
        vals = torch.ones(keys.numel(), dtype=torch.int64)
    plan = make_plan("equal", keys, group, local, seed, samples, buckets_per_rank)
    ids = bucket_ids(keys, plan, local)
    nl = 1 << plan.light_bits
    heavy_rec = ids >= nl
    # heavy keys: local partial sums, one (key, partial) pair per heavy key present
    hk, hs = local.collect_reduce(keys[heavy_rec], vals[heavy_rec]) if int(heavy_rec.sum()) else \
        (torch.zeros(0, dtype=torch.int64), torch.zeros(0, dtype=torch.int64))
    k2 = torch.cat([keys[~heavy_rec], hk])
    v2 = torch.cat([vals[~heavy_rec], hs])
    ids_s, order, dest, _, _, _, _ = _route(k2, plan, group, local, world, rank, False)
    (rk, rv), _ = _exchange(group, world, dest, k2[order], v2[order])
    if rk.numel() == 0:
        return rk, rv
    return local.collect_reduce(rk, rv)


class GpuLocal:
    """Single-GPU operations of the sharded form: the library's kernels on
    device tensors (int64 views of u64 data)."""

    def __init__(self, ss=None):
        if ss is None:
            import paper_2304_10078_gb300 as ss
        self.ss = ss

    def hash64(self, x: torch.Tensor, salt: int) -> torch.Tensor:
        return self.ss.hash_u64(x.cuda().view(torch.uint64), salt & MASK64).view(torch.int64)

    def stable_order(self, ids: torch.Tensor) -> torch.Tensor:
        if ids.numel() == 0:
            return ids
        _, v = self.ss.semisort_less(ids.cuda().view(torch.uint64),
                                     torch.arange(ids.numel(), device="cuda", dtype=torch.int64).view(torch.uint64))
        return v.view(torch.int64)

    def semisort_equal(self, k, v):
        ko, vo = self.ss.semisort_equal(k.cuda().view(torch.uint64), v.cuda().view(torch.uint64))
        return ko.view(torch.int64), vo.view(torch.int64)

    def semisort_less(self, k, v):
        ko, vo = self.ss.semisort_less(k.cuda().view(torch.uint64), v.cuda().view(torch.uint64))
        return ko.view(torch.int64), vo.view(torch.int64)

    def collect_reduce(self, k, v):
        uk, s, nu = self.ss.collect_reduce(k.cuda().view(torch.uint64), v.cuda().view(torch.uint64))
        u = int(nu.view(torch.int64)[0].item())
        return uk[:u].view(torch.int64), s[:u].view(torch.int64)
