"""Oracle parity on the paths that only very large inputs reach with default
options: three or more distribution levels (Algorithm 1 recursing on light
buckets), keys that become heavy only at a deeper level (Sec. 3.1: a key's
sample count is judged against its own subproblem), and collect-reduce heavy
partial sums spread over many subarrays of one segment (Sec. 3.5).

Small options force those paths at n = 2^22: alpha = 256 (base cases of at
most 256 records), subarrays of 4096 records below the top level, and
n_L = 8 light buckets at the top level, so every top-level bucket holds about
2^19 records and recurses at least twice.  The workload mixes 2000 keys of
about 1000 copies each (light at the top level, where their expected sample
count is below the heavy threshold; heavy once a level-1 or level-2
subproblem holds them) with a uniform background of about 2 copies per key.
Every output is compared with the oracle: semisort_= through the canonical
check, semisort_< bit-exactly with the stable sort, collect-reduce and
histogram bit-exactly after sorting by key."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import to_dev, to_host

pytestmark = pytest.mark.gpu

N = 1 << 22
OPTS = dict(alpha=256, subarray=4096, n_light_log2=3)


@pytest.fixture(scope="module")
def ss():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2304_10078_gb300 as m
    m.build()
    return m


def deep_keys(seed: int, n: int = N) -> np.ndarray:
    """Half the records draw one of 2000 'medium' keys (about 1000 copies
    each), half a background key (about 2 copies each); positions mixed by
    the seeded generator."""
    pick = synth.uniform_mod(seed, n, 2)
    med = synth.key_of_rank(seed + 1, synth.uniform_mod(seed + 2, n, 2000))
    bg = synth.key_of_rank(seed + 3, synth.uniform_mod(seed + 4, n, n // 2) + np.uint64(10**6))
    return np.where(pick == 0, med, bg).astype(np.uint64)


@pytest.fixture(scope="module")
def workload():
    keys = deep_keys(0xDEE9)
    vals = synth.splitmix64_outputs(0xDEEA, N)  # full-range values: sums wrap around
    return keys, vals


def _stats_levels(ss, ws):
    st = ss.stats(ws)
    return st["levels"], st


def test_workload_shape(workload):
    keys, _ = workload
    rk, cnt = oracle.histogram_sorted(keys)
    med = cnt[cnt >= 500]
    assert 1900 <= len(med) <= 2000 and 900 <= np.median(med) <= 1200
    assert np.max(cnt[cnt < 500]) < 20


@pytest.mark.parametrize("seed", [1, 7])
def test_semisort_equal_three_levels(ss, workload, seed):
    import torch
    keys_h, vals_h = workload
    keys, vals = to_dev(keys_h), to_dev(vals_h)
    o = ss.make_options(seed=seed, **OPTS)
    ws = ss.alloc_workspace(ss.OP_EQUAL, keys, vals, o)
    ko, vo = ss.semisort_equal(keys, vals, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    levels, st = _stats_levels(ss, ws)
    assert levels >= 3, st
    assert st["dist_l2"] > 0, st
    err = oracle.check_semisort_equal(keys_h, vals_h, to_host(ko), to_host(vo))
    assert err is None, err


def test_semisort_less_three_levels(ss, workload):
    import torch
    keys_h, vals_h = workload
    keys, vals = to_dev(keys_h), to_dev(vals_h)
    o = ss.make_options(seed=3, **OPTS)
    ws = ss.alloc_workspace(ss.OP_LESS, keys, vals, o)
    ko, vo = ss.semisort_less(keys, vals, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    levels, st = _stats_levels(ss, ws)
    assert levels >= 3, st
    err = oracle.check_sorted_equal(keys_h, vals_h, to_host(ko), to_host(vo))
    assert err is None, err


@pytest.mark.parametrize("op", ["reduce", "hist"])
def test_reduce_three_levels(ss, workload, op):
    import torch
    keys_h, vals_h = workload
    if op == "hist":
        vals_h = None
    keys = to_dev(keys_h)
    o = ss.make_options(seed=5, **OPTS)
    if vals_h is None:
        ws = ss.alloc_workspace(ss.OP_HIST, keys, None, o)
        uk, out, nu = ss.histogram(keys, workspace=ws, options=o)
        rk, rs = oracle.histogram_sorted(keys_h)
    else:
        vals = to_dev(vals_h)
        ws = ss.alloc_workspace(ss.OP_REDUCE, keys, vals, o)
        uk, out, nu = ss.collect_reduce(keys, vals, workspace=ws, options=o)
        rk, rs = oracle.collect_reduce_sorted(keys_h, vals_h)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    levels, st = _stats_levels(ss, ws)
    assert levels >= 3, st
    u = int(to_host(nu)[0])
    assert u == len(rk)
    gk, gs = oracle.stable_sort(to_host(uk)[:u], to_host(out)[:u])
    assert np.array_equal(gk, rk), "unique keys differ"
    assert np.array_equal(gs, rs), "sums/counts differ"


def test_reduce_many_subarray_heavy_partials(ss):
    """One dominant key spread over every subarray of a large segment: its
    sum is assembled from hundreds of per-subarray partials (Sec. 3.5)."""
    import torch
    n = 1 << 23
    keys_h = synth.uniform_mod(0xDEEB, n, 1 << 20)
    keys_h[synth.uniform_mod(0xDEEC, n, 4) == 0] = np.uint64(0xFFFFFFFFFFFFFFFF)
    keys_h[synth.uniform_mod(0xDEED, n, 16) == 0] = np.uint64(0)
    vals_h = synth.splitmix64_outputs(0xDEEE, n)
    keys, vals = to_dev(keys_h), to_dev(vals_h)
    o = ss.make_options(seed=9, subarray=4096, alpha=512)
    ws = ss.alloc_workspace(ss.OP_REDUCE, keys, vals, o)
    uk, out, nu = ss.collect_reduce(keys, vals, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    rk, rs = oracle.collect_reduce_sorted(keys_h, vals_h)
    u = int(to_host(nu)[0])
    assert u == len(rk)
    gk, gs = oracle.stable_sort(to_host(uk)[:u], to_host(out)[:u])
    assert np.array_equal(gk, rk) and np.array_equal(gs, rs)


def test_hash_u64_matches_oracle_mixer(ss):
    """ss_hash_u64 computes mix64(k ^ salt), SplitMix64's output mixer, whose
    oracle statement is pinned against the published output vectors."""
    import torch
    edge = [0, 1, 2, 3, 0xFFFFFFFFFFFFFFFF, 0xFFFFFFFFFFFFFFFE, 1 << 63, (1 << 63) - 1, 0x9E3779B97F4A7C15,
            0xFFFFFFFF, 1 << 32]
    rnd = [int(x) for x in synth.splitmix64_outputs(0xA5A5, 989)]
    ks = np.array(edge + rnd, dtype=np.uint64)
    for salt in (0, 1, 0xFFFFFFFFFFFFFFFF, 0x5EED0002, int(synth.splitmix64_outputs(3, 1)[0])):
        got = to_host(ss.hash_u64(to_dev(ks), salt))
        torch.cuda.synchronize()
        want = np.array([oracle.mix64(int(k) ^ salt) for k in ks], dtype=np.uint64)
        assert np.array_equal(got, want), salt
