"""The paper's variants as flags on the same kernels: identity bucketing of
integer keys (semisort-i, Sec. 4.1) and semisort_< on hash buckets with a
sorting base case (Sec. 3.3).  Results against the CPU oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ss():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2304_10078_gb300 as m
    m.build()
    return m


def keys_for(kind, n):
    if kind == "hashed":
        return synth.uniform_mod(91, n, 10**6) * np.uint64(0x9E3779B97F4A7C15)
    if kind == "small_ints":
        return synth.uniform_mod(92, n, 10**6)
    return synth.zipf(93, n, 1.2, N=10**6)


@pytest.mark.parametrize("kind", ["hashed", "small_ints", "zipf"])
@pytest.mark.parametrize("n", [5000, 1 << 21])
def test_identity_semisort_equal(ss, kind, n):
    import torch
    keys = keys_for(kind, n)
    vals = np.arange(n, dtype=np.uint64)
    o = ss.make_options(seed=1, flags=ss.FLAG_IDENTITY_HASH)
    k, v = to_dev(keys), to_dev(vals)
    ws = ss.alloc_workspace(ss.OP_EQUAL, k, v, o)
    ko, vo = ss.semisort_equal(k, v, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    assert oracle.check_semisort_equal(keys, vals, to_host(ko), to_host(vo)) is None


@pytest.mark.parametrize("kind", ["small_ints", "zipf"])
def test_identity_reduce_hist_u32(ss, kind):
    import torch
    n = 1 << 21
    keys = keys_for(kind, n).astype(np.uint32)
    vals = synth.splitmix64_outputs(94, n)
    o = ss.make_options(seed=1, flags=ss.FLAG_IDENTITY_HASH)
    uk, sums, nu = ss.collect_reduce(to_dev(keys), to_dev(vals), options=o)
    uh, cnt, nh = ss.histogram(to_dev(keys), options=o)
    torch.cuda.synchronize()
    u, h = int(to_host(nu)[0]), int(to_host(nh)[0])
    rk, rs = oracle.collect_reduce_sorted(keys, vals)
    gk, gs = oracle.stable_sort(to_host(uk)[:u], to_host(sums)[:u])
    assert np.array_equal(gk, rk) and np.array_equal(gs, rs)
    hk, hc = oracle.histogram_sorted(keys)
    gk, gc = oracle.stable_sort(to_host(uh)[:h], to_host(cnt)[:h])
    assert np.array_equal(gk, hk) and np.array_equal(gc, hc)


def test_identity_depth_limit_is_reported(ss):
    """Distinct keys that agree in all bits the four levels look at (multiples
    of 2^40) cannot be split by identity bucketing: the call reports the
    recursion-depth error instead of a result."""
    import torch
    n = 1 << 15
    keys = (np.arange(n, dtype=np.uint64) + np.uint64(1)) << np.uint64(40)
    keys = keys[synth.feistel_permute(95, n, np.arange(n, dtype=np.uint64)).astype(np.int64)]
    o = ss.make_options(seed=1, flags=ss.FLAG_IDENTITY_HASH)
    k = to_dev(keys)
    ws = ss.alloc_workspace(ss.OP_EQUAL, k, None, o)
    ss.semisort_equal(k, None, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 8  # SS_ERR_DEPTH
    # the same keys without the flag are hashed and sorted out normally
    o2 = ss.make_options(seed=1)
    ko, _ = ss.semisort_equal(k, None, workspace=ws, options=o2)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    assert oracle.count_runs(to_host(ko)) == n


@pytest.mark.parametrize("kind", ["hashed", "zipf"])
@pytest.mark.parametrize("n", [3000, 1 << 21])
def test_hash_bucket_semisort_less(ss, kind, n):
    """semisort_< on hash buckets: equal keys contiguous and stable (the
    semisort_= contract); every base case is sorted, so a bucket of the top
    level holds its keys in increasing order between group boundaries."""
    import torch
    keys = keys_for(kind, n)
    vals = np.arange(n, dtype=np.uint64)
    o = ss.make_options(seed=1, flags=ss.FLAG_HASH_BUCKETS)
    k, v = to_dev(keys), to_dev(vals)
    ws = ss.alloc_workspace(ss.OP_LESS, k, v, o)
    ko, vo = ss.semisort_less(k, v, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    ko, vo = to_host(ko), to_host(vo)
    assert oracle.check_semisort_equal(keys, vals, ko, vo) is None
    if n <= 4096:  # a single base case: fully sorted
        assert np.array_equal(ko, oracle.stable_sort(keys)[0])


@pytest.mark.parametrize("op", ["equal", "less_hash"])
def test_hash_buckets_keys_with_many_copies(ss, op):
    """floor(Exp(lambda)) with about a thousand copies per key value: such keys
    stay light at shallow levels and must be separated deeper down without
    reaching the recursion-depth limit."""
    import torch
    n = 1 << 24
    keys = synth.exponential(96, n, 6e-5)
    vals = np.arange(n, dtype=np.uint64)
    k, v = to_dev(keys), to_dev(vals)
    if op == "equal":
        o = ss.make_options(seed=1)
        ws = ss.alloc_workspace(ss.OP_EQUAL, k, v, o)
        ko, vo = ss.semisort_equal(k, v, workspace=ws, options=o)
    else:
        o = ss.make_options(seed=1, flags=ss.FLAG_HASH_BUCKETS)
        ws = ss.alloc_workspace(ss.OP_LESS, k, v, o)
        ko, vo = ss.semisort_less(k, v, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    assert oracle.check_semisort_equal(keys, vals, to_host(ko), to_host(vo)) is None
