"""Parity at the full size of the benchmark (n = 10^9, u64 key, u64 value =
index, default options as bench.py times them), through properties that hold
at any size and that the GPU can check in full:

* semisort_= / semisort_<: the values form a permutation of 0..n-1, every
  output record is an input record (key = input key of its value), records of
  equal keys keep input order (values increase along each run), equal keys
  are contiguous (runs = distinct keys); semisort_< keys do not decrease.
* collect-reduce: the unique count is the number of distinct keys, the keys
  are distinct, and the sums add up to n(n-1)/2 mod 2^64 (value = index).
* histogram: the unique count is the number of distinct keys and the counts
  add up to n.

Collect-reduce and histogram are also compared with the oracle key by key
at the full size (Zipf 1.2 and uniform 10^7 keys): the oracle runs on
contiguous chunks of the input in host threads, and its per-chunk outputs are
combined by the oracle's own collect-reduce (the sum of partial sums is the
sum, by associativity of + mod 2^64).  On all ten benchmark distributions a
grouping-independent checksum sum_k g(k) * sum_k = sum_i g(key_i) * val_i
(mod 2^64, g a hash unrelated to the library's) catches per-key sums that
are wrong in ways the totals hide.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

N = 10**9
DISTS = [("uniform", 10), ("uniform", 10**3), ("uniform", 10**5), ("uniform", 10**7), ("uniform", 10**9),
         ("zipf", 0.6), ("zipf", 0.8), ("zipf", 1.0), ("zipf", 1.2), ("zipf", 1.5)]
SEED = 0x5EED0002


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    if torch.cuda.get_device_properties(0).total_memory < 200 * 2**30:
        pytest.skip("needs a GPU with about 200 GB")
    import paper_2304_10078_gb300 as ss
    import synth.gpu as sg
    ss.build()
    vals = sg.iota(N)
    return ss, sg, vals


def keys_of(sg, kind, p):
    return sg.uniform_exact(SEED, N, p) if kind == "uniform" else sg.zipf(SEED, N, p)


def distinct(torch, k):
    s, _ = torch.sort(k.view(torch.int64))
    return int((s[1:] != s[:-1]).sum().item()) + 1


def check_semisort(torch, keys, vals_out, keys_out, ordered):
    ki, ko, vo = keys.view(torch.int64), keys_out.view(torch.int64), vals_out.view(torch.int64)
    seen = torch.zeros(N, dtype=torch.bool, device="cuda")
    seen[vo] = True
    assert bool(seen.all()), "values are not a permutation"
    del seen
    assert bool((ki[vo] == ko).all()), "a record's key changed"
    same = ko[1:] == ko[:-1]
    assert bool((vo[1:][same] > vo[:-1][same]).all()), "equal keys out of input order"
    runs = int((~same).sum().item()) + 1
    assert runs == distinct(torch, ki), "equal keys not contiguous"
    if ordered:
        flip = ko ^ (-(2**63))  # unsigned order as signed order
        assert bool((flip[1:] >= flip[:-1]).all()), "keys decrease"


@pytest.mark.parametrize("kind,p", [("uniform", 10**7), ("zipf", 0.8), ("uniform", 10**9)])
def test_semisort_equal_full_size(env, kind, p):
    import torch
    ss, sg, vals = env
    keys = keys_of(sg, kind, p)
    o = ss.make_options(seed=1)
    ws = ss.alloc_workspace(ss.OP_EQUAL, keys, vals, o)
    ko, vo = ss.semisort_equal(keys, vals, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    del ws
    check_semisort(torch, keys, vo, ko, ordered=False)


@pytest.mark.parametrize("kind,p", [("uniform", 10**9), ("zipf", 1.2)])
def test_semisort_less_full_size(env, kind, p):
    import torch
    ss, sg, vals = env
    keys = keys_of(sg, kind, p)
    o = ss.make_options(seed=1)
    ws = ss.alloc_workspace(ss.OP_LESS, keys, vals, o)
    ko, vo = ss.semisort_less(keys, vals, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    del ws
    check_semisort(torch, keys, vo, ko, ordered=True)


def test_collect_reduce_and_histogram_full_size(env):
    import torch
    ss, sg, vals = env
    keys = keys_of(sg, "zipf", 1.2)
    d = distinct(torch, keys)
    o = ss.make_options(seed=1)
    ws = ss.alloc_workspace(ss.OP_REDUCE, keys, vals, o)
    uk, sums, nu = ss.collect_reduce(keys, vals, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    u = int(nu.view(torch.int64)[0].item())
    assert u == d
    assert distinct(torch, uk[:u]) == u
    total = int(sums[:u].view(torch.int64).sum().item()) % 2**64  # int64 sums wrap like u64
    assert total == (N * (N - 1) // 2) % 2**64
    del uk, sums, ws
    ws = ss.alloc_workspace(ss.OP_HIST, keys, None, o)
    hk, cnt, nh = ss.histogram(keys, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    h = int(nh.view(torch.int64)[0].item())
    assert h == d
    assert int(cnt[:h].view(torch.int32).to(torch.int64).sum().item()) == N


def test_semisort_less_learned_full_size(env):
    import torch
    ss, sg, vals = env
    keys = keys_of(sg, "uniform", 10**9)
    o = ss.make_options(seed=1, splitter_mode=1)
    ws = ss.alloc_workspace(ss.OP_LESS, keys, vals, o)
    ko, vo = ss.semisort_less(keys, vals, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    assert ss.stats(ws)["l0_splitters"] == 1  # the trained model was used
    del ws
    check_semisort(torch, keys, vo, ko, ordered=True)


def test_batched_semisort_equal_full_size(env):
    """The 4096-instance workload of the benchmark (about 1.7 * 10^9 records):
    every output value stays inside its own instance's range, records are
    intact and stable, and the runs add up to the distinct keys of every
    instance."""
    import torch

    import bench
    ss, sg, _ = env
    off_h, keys, n = bench.batched_workload(sg, torch)
    off = torch.from_numpy(off_h).cuda()
    vals = sg.iota(n)
    o = ss.make_options(seed=1)
    ws = ss.alloc_workspace_batched(ss.OP_EQUAL, keys, off.view(torch.uint64), vals, o)
    ko, vo = ss.semisort_equal_batched(keys, vals, off.view(torch.uint64), workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    del ws
    ki, kk, vv = keys.view(torch.int64), ko.view(torch.int64), vo.view(torch.int64)
    pos_inst = torch.searchsorted(off, torch.arange(n, device="cuda", dtype=torch.int64), right=True) - 1
    val_inst = torch.searchsorted(off, vv, right=True) - 1
    assert bool((pos_inst == val_inst).all()), "a record left its instance"
    del val_inst
    assert bool((ki[vv] == kk).all()), "a record's key changed"
    same = (kk[1:] == kk[:-1]) & (pos_inst[1:] == pos_inst[:-1])
    assert bool((vv[1:][same] > vv[:-1][same]).all()), "equal keys out of input order"
    runs = int((~same).sum().item()) + 1
    # distinct (instance, key) pairs: sort by key, then stably by instance
    order = torch.argsort(ki, stable=True)
    inst_sorted = pos_inst[order]
    o2 = torch.argsort(inst_sorted, stable=True)
    ks, isx = ki[order][o2], inst_sorted[o2]
    pairs = int(((ks[1:] != ks[:-1]) | (isx[1:] != isx[:-1])).sum().item()) + 1
    assert runs == pairs, "equal keys not contiguous within an instance"


def host_u64(t):
    import torch
    return t.view(torch.int64).cpu().numpy().view(np.uint64)


def oracle_reduce_chunked(keys_h, vals_h):
    """The oracle's (unique keys ascending, sums) of the whole input, from
    per-chunk oracle outputs (host threads; the oracle releases the GIL)
    combined by the oracle's sort-based collect-reduce.  vals_h None: counts
    (histogram)."""
    n = len(keys_h)
    parts = max(8, min(16, os.cpu_count() or 8))
    cut = [n * i // parts for i in range(parts + 1)]

    def one(i):
        a, b = cut[i], cut[i + 1]
        if vals_h is None:
            k, c = oracle.histogram_hash(keys_h[a:b])
            return k, c.astype(np.uint64)
        return oracle.collect_reduce_hash(keys_h[a:b], vals_h[a:b])

    with ThreadPoolExecutor(parts) as ex:
        res = list(ex.map(one, range(parts)))
    ks = np.concatenate([r[0] for r in res])
    vs = np.concatenate([r[1] for r in res])
    del res
    return oracle.collect_reduce_sorted(ks, vs)


def host_memory_gb():
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES") / 2**30
    except (ValueError, OSError):
        return 0.0


@pytest.mark.parametrize("kind,p", [("zipf", 1.2), ("uniform", 10**7)])
def test_reduce_and_histogram_full_size_vs_oracle(env, kind, p):
    """Every (key, sum) and (key, count) at n = 10^9 against the oracle."""
    import torch
    if host_memory_gb() < 160:
        pytest.skip("needs about 100 GB of host memory for the oracle")
    ss, sg, vals = env
    keys = keys_of(sg, kind, p)
    o = ss.make_options(seed=1)
    ws = ss.alloc_workspace(ss.OP_REDUCE, keys, vals, o)
    uk, sums, nu = ss.collect_reduce(keys, vals, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    u = int(nu.view(torch.int64)[0].item())
    g_keys, g_sums = host_u64(uk[:u]), host_u64(sums[:u])
    del uk, sums, ws
    ws = ss.alloc_workspace(ss.OP_HIST, keys, None, o)
    hk, cnt, nh = ss.histogram(keys, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    h = int(nh.view(torch.int64)[0].item())
    h_keys = host_u64(hk[:h])
    h_cnt = cnt[:h].view(torch.int32).cpu().numpy().view(np.uint32)
    del hk, cnt, ws
    keys_h, vals_h = host_u64(keys), host_u64(vals)
    del keys
    torch.cuda.empty_cache()

    rk, rs = oracle_reduce_chunked(keys_h, vals_h)
    assert u == len(rk), (u, len(rk))
    gk, gs = oracle.stable_sort(g_keys, g_sums)
    assert np.array_equal(gk, rk), "collect-reduce unique keys differ"
    bad = np.flatnonzero(gs != rs)
    assert len(bad) == 0, f"{len(bad)} sums differ, first at key {rk[bad[0]]}"
    del rs, gk, gs, g_keys, g_sums, vals_h

    rk2, rc = oracle_reduce_chunked(keys_h, None)
    assert h == len(rk2)
    hk_s, hc_s = oracle.stable_sort(h_keys, h_cnt)
    assert np.array_equal(hk_s, rk2), "histogram unique keys differ"
    assert np.array_equal(hc_s.astype(np.uint64), rc), "histogram counts differ"


def gmix(torch, k):
    """A hash of int64 words unrelated to the library's mixers: two rounds of
    multiply and xor-fold, in wrapping int64 arithmetic."""
    x = k * 0x2545F4914F6CDD1D + 0x3C6EF372FE94F82B
    x = x ^ ((x >> 29) & 0x7FFFFFFFF)
    x = x * 0x27BB2EE687B0B0FD
    return x ^ ((x >> 32) & 0xFFFFFFFF)


@pytest.mark.parametrize("kind,p", DISTS)
def test_reduce_weighted_checksum_full_size(env, kind, p):
    """sum_k g(k) * sum_k (output) = sum_i g(key_i) * val_i (input), and the
    same with val = 1 for the histogram, mod 2^64: per-key sums that err by
    +x and -x on two keys change the checksum by x (g(k1) - g(k2))."""
    import torch
    ss, sg, vals = env
    keys = keys_of(sg, kind, p)
    ki, vi = keys.view(torch.int64), vals.view(torch.int64)
    want_r = int((gmix(torch, ki) * vi).sum().item()) % 2**64
    want_h = int(gmix(torch, ki).sum().item()) % 2**64
    o = ss.make_options(seed=1)
    ws = ss.alloc_workspace(ss.OP_REDUCE, keys, vals, o)
    uk, sums, nu = ss.collect_reduce(keys, vals, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    u = int(nu.view(torch.int64)[0].item())
    got_r = int((gmix(torch, uk[:u].view(torch.int64)) * sums[:u].view(torch.int64)).sum().item()) % 2**64
    assert got_r == want_r
    del uk, sums, ws
    ws = ss.alloc_workspace(ss.OP_HIST, keys, None, o)
    hk, cnt, nh = ss.histogram(keys, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    h = int(nh.view(torch.int64)[0].item())
    assert h == u
    c64 = cnt[:h].view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    got_h = int((gmix(torch, hk[:h].view(torch.int64)) * c64).sum().item()) % 2**64
    assert got_h == want_h
