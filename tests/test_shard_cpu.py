"""The sharded form (paper_2304_10078_gb300/shard.py) on CPU ranks over gloo:
sample all-gather, identical heavy tables and splitters on every rank,
bucket-to-owner mapping from the all-gathered counts, one all-to-all of
records, and the local step.  The local single-device operations are
stand-ins built on the oracle (this is a test of the partitioning logic, not
of the kernels); the concatenated outputs must equal the oracle's result for
the concatenated input."""
import os
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth

PORT = 29613


class CpuLocal:
    """Single-rank operations on int64 views of u64 data, from the oracle."""

    @staticmethod
    def _u(t):
        return t.numpy().view(np.uint64)

    @staticmethod
    def _t(a):
        return torch.from_numpy(np.ascontiguousarray(a).view(np.int64))

    def hash64(self, x, salt):
        return self._t(synth.mix64_np(self._u(x) ^ np.uint64(salt & (2**64 - 1))))

    def stable_order(self, ids):
        _, v = oracle.stable_sort(self._u(ids), np.arange(ids.numel(), dtype=np.uint64))
        return self._t(v)

    def semisort_equal(self, k, v):
        a, b = oracle.group_by(self._u(k), self._u(v))
        return self._t(a), self._t(b)

    def semisort_less(self, k, v):
        a, b = oracle.stable_sort(self._u(k), self._u(v))
        return self._t(a), self._t(b)

    def collect_reduce(self, k, v):
        a, b = oracle.collect_reduce_hash(self._u(k), self._u(v))
        return self._t(a), self._t(b)


def make_input(kind, n):
    if kind == "uniform":
        return synth.uniform_mod(0x5A4D, n, 1000)
    if kind == "zipf":
        return synth.zipf(0x5A4E, n, 1.2, N=10**6)
    if kind == "distinct":
        return synth.splitmix64_outputs(0x5A4F, n)
    return np.full(n, 42, np.uint64)


def _worker(rank, world, kind, n, cuts, op, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(PORT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2304_10078_gb300 import shard
    keys = make_input(kind, n)[cuts[rank]:cuts[rank + 1]]
    vals = np.arange(cuts[rank], cuts[rank + 1], dtype=np.uint64)
    k = torch.from_numpy(keys.view(np.int64).copy())
    v = torch.from_numpy(vals.view(np.int64).copy())
    local = CpuLocal()
    plan = shard.make_plan("less" if op == "less" else "equal", k, None, local)
    if op in ("equal", "less"):
        ko, vo = shard.sharded_semisort(op, k, v, None, local)
    else:
        ko, vo = shard.sharded_reduce(op, k, v if op == "reduce" else None, None, local)
    np.save(os.path.join(outdir, f"k{rank}.npy"), ko.numpy().view(np.uint64))
    np.save(os.path.join(outdir, f"v{rank}.npy"), vo.numpy().view(np.uint64))
    np.save(os.path.join(outdir, f"h{rank}.npy"), plan.heavy.numpy())
    np.save(os.path.join(outdir, f"b{rank}.npy"), plan.bounds.numpy())
    dist.barrier()
    dist.destroy_process_group()


def run_sharded(kind, n, cuts, op):
    global PORT
    PORT += 1
    world = len(cuts) - 1
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_worker, args=(world, kind, n, cuts, op, d), nprocs=world, start_method="spawn")
        ks = [np.load(os.path.join(d, f"k{r}.npy")) for r in range(world)]
        vs = [np.load(os.path.join(d, f"v{r}.npy")) for r in range(world)]
        hs = [np.load(os.path.join(d, f"h{r}.npy")) for r in range(world)]
        bs = [np.load(os.path.join(d, f"b{r}.npy")) for r in range(world)]
    for r in range(1, world):
        assert np.array_equal(hs[r], hs[0]), "heavy tables differ between ranks"
        assert np.array_equal(bs[r], bs[0]), "splitters differ between ranks"
    return ks, vs, hs[0]


CASES = [("uniform", 50_001, [0, 20_000, 50_001]), ("zipf", 60_000, [0, 30_000, 60_000]),
         ("zipf", 40_000, [0, 0, 40_000]), ("equalkeys", 9_000, [0, 4_000, 9_000]),
         ("distinct", 30_000, [0, 7_000, 19_000, 30_000])]


@pytest.mark.parametrize("kind,n,cuts", CASES)
@pytest.mark.parametrize("op", ["less", "equal"])
def test_sharded_semisort_matches_oracle(kind, n, cuts, op):
    ks, vs, heavy = run_sharded(kind, n, cuts, op)
    keys = make_input(kind, n)
    vals = np.arange(n, dtype=np.uint64)
    out_k, out_v = np.concatenate(ks), np.concatenate(vs)
    if op == "less":
        rk, rv = oracle.stable_sort(keys, vals)
        assert np.array_equal(out_k, rk) and np.array_equal(out_v, rv)
    else:
        err = oracle.check_semisort_equal(keys, vals, out_k, out_v)
        assert err is None, err
    if kind == "zipf" and cuts[1] > 0:
        assert len(heavy) > 0
        # heavy keys split between owners keep the shares near n / G
        assert max(len(k) for k in ks) <= 0.75 * n, [len(k) for k in ks]


@pytest.mark.parametrize("kind,n,cuts", CASES)
@pytest.mark.parametrize("op", ["reduce", "hist"])
def test_sharded_reduce_matches_oracle(kind, n, cuts, op):
    ks, vs, _ = run_sharded(kind, n, cuts, op)
    keys = make_input(kind, n)
    out_k, out_v = np.concatenate(ks), np.concatenate(vs)
    assert len(np.unique(out_k)) == len(out_k), "a key reduced on two ranks"
    gk, gv = oracle.stable_sort(out_k, out_v)
    if op == "reduce":
        rk, rs = oracle.collect_reduce_sorted(keys, np.arange(n, dtype=np.uint64))
    else:
        rk, rc = oracle.histogram_sorted(keys)
        rs = rc.astype(np.uint64)
    assert np.array_equal(gk, rk) and np.array_equal(gv, rs)
