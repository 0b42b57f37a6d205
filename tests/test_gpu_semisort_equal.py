"""GPU parity of semisort_= against the CPU oracle (bit-exact acceptance:
run count = distinct keys, and the stable sort of the output equals the stable
sort of the input, which proves permutation + contiguity + stability)."""
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


def run_equal(ss, keys_h, vals_h, seed=1, inplace=False, **opt):
    import torch
    keys = to_dev(keys_h)
    vals = None if vals_h is None else to_dev(vals_h)
    o = ss.make_options(seed=seed, **opt)
    ws = ss.alloc_workspace(ss.OP_EQUAL, keys, vals, o)
    if inplace:
        ko, vo = ss.semisort_equal(keys, vals, keys_out=keys, vals_out=vals, workspace=ws, options=o)
    else:
        ko, vo = ss.semisort_equal(keys, vals, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    st = ss.stats(ws)
    return to_host(ko), (None if vo is None else to_host(vo)), st


def check(keys_h, vals_h, ko, vo):
    err = oracle.check_semisort_equal(keys_h, vals_h, ko, vo)
    assert err is None, err


def test_config1_uniform_1e4(ss):
    """n = 2^20, key = splitmix64(seed, i) mod 10^4, value = index."""
    n = 1 << 20
    keys = synth.uniform_mod(0x5EED0001, n, 10**4)
    vals = np.arange(n, dtype=np.uint64)
    ko, vo, st = run_equal(ss, keys, vals)
    check(keys, vals, ko, vo)


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 255, 256, 257, 4095, 4096, 4097, 8191, 32769, 65537, 300001])
def test_edge_sizes(ss, n):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, max(2, n // 7), size=n, dtype=np.uint64)
    vals = np.arange(n, dtype=np.uint64)
    ko, vo, _ = run_equal(ss, keys, vals)
    check(keys, vals, ko, vo)


def test_empty(ss):
    import torch
    k = torch.empty(0, dtype=torch.uint64, device="cuda")
    ko, vo = ss.semisort_equal(k, k.clone())
    assert ko.numel() == 0


@pytest.mark.parametrize("kind", ["all_equal", "all_distinct", "one_heavy", "two_heavy", "zipf15", "zipf08",
                                  "uniform_exact_1e3", "pow2_keys"])
def test_distributions(ss, kind):
    n = 1 << 21
    if kind == "all_equal":
        keys = np.full(n, 0xDEADBEEF, np.uint64)
    elif kind == "all_distinct":
        keys = synth.splitmix64_outputs(3, n)
    elif kind == "one_heavy":
        keys = synth.uniform_mod(4, n, 10**6)
        keys[synth.uniform_mod(5, n, 10) < 6] = 7  # 60% of the records share one key
    elif kind == "two_heavy":
        keys = synth.uniform_mod(4, n, 10**6)
        sel = synth.uniform_mod(6, n, 10)
        keys[sel < 3] = 0
        keys[sel == 3] = 1
    elif kind == "zipf15":
        keys = synth.zipf(7, n, 1.5, N=10**9)
    elif kind == "zipf08":
        keys = synth.zipf(8, n, 0.8, N=10**9)
    elif kind == "uniform_exact_1e3":
        keys = synth.uniform_exact(9, n, 1000)
    else:
        keys = (np.uint64(1) << (synth.uniform_mod(10, n, 64))).astype(np.uint64)
    vals = np.arange(n, dtype=np.uint64)
    ko, vo, st = run_equal(ss, keys, vals)
    check(keys, vals, ko, vo)


def test_recursion_two_levels(ss):
    """2^24 records with 2^22 distinct keys: level-0 buckets exceed the
    base-case threshold, so a second distribution level runs (Sec. 3.3)."""
    n = 1 << 24
    keys = synth.uniform_exact(11, n, 1 << 22)
    vals = np.arange(n, dtype=np.uint64)
    ko, vo, st = run_equal(ss, keys, vals)
    assert st["levels"] >= 2 and st["dist_l1"] > 0
    check(keys, vals, ko, vo)


def test_heavy_records_never_refined(ss):
    """Records of detected heavy keys are final after distribution: they never
    enter a base case (Sec. 3.1, Sec. 3.3)."""
    n = 1 << 22
    keys = synth.uniform_mod(12, n, 10**7)
    sel = synth.uniform_mod(13, n, 100)
    keys[sel < 50] = 99  # one key with half the records
    vals = np.arange(n, dtype=np.uint64)
    ko, vo, st = run_equal(ss, keys, vals)
    check(keys, vals, ko, vo)
    assert st["heavy_l0"] >= 1
    assert st["refined"] <= n - int((sel < 50).sum())


@pytest.mark.parametrize("vdtype", ["u32", "none"])
def test_value_types(ss, vdtype):
    n = 1 << 20
    keys = synth.uniform_mod(14, n, 5000)
    vals = None if vdtype == "none" else np.arange(n, dtype=np.uint32)[::-1].copy()
    ko, vo, _ = run_equal(ss, keys, vals)
    if vals is None:
        assert np.array_equal(oracle.stable_sort(ko)[0], oracle.stable_sort(keys)[0])
        assert oracle.count_runs(ko) == oracle.count_distinct(keys)
    else:
        check(keys, vals, ko, vo)


@pytest.mark.parametrize("n", [3000, 1 << 20, 1 << 23])
def test_in_place(ss, n):
    keys = synth.zipf(15, n, 1.2, N=10**6)
    vals = np.arange(n, dtype=np.uint64)
    ko, vo, _ = run_equal(ss, keys, vals, inplace=True)
    check(keys, vals, ko, vo)


def test_deterministic(ss):
    n = 1 << 22
    keys = synth.zipf(16, n, 1.0, N=10**9)
    vals = np.arange(n, dtype=np.uint64)
    a = run_equal(ss, keys, vals, seed=5)
    b = run_equal(ss, keys, vals, seed=5)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("alpha,subarray,lbits", [(256, 4096, 3), (1024, 8192, 11), (4096, 65536, 1)])
def test_parameters(ss, alpha, subarray, lbits):
    """Any tunable setting gives a correct result (only speed changes)."""
    n = 1 << 21
    keys = synth.zipf(17, n, 1.1, N=10**6)
    vals = np.arange(n, dtype=np.uint64)
    ko, vo, _ = run_equal(ss, keys, vals, alpha=alpha, subarray=subarray, n_light_log2=lbits)
    check(keys, vals, ko, vo)


def test_element_aligned_slices(ss):
    """Arrays need only their element alignment: slices starting at odd
    element offsets (8-byte aligned) work as inputs and outputs."""
    import torch
    n = 300_001
    keys_h = synth.uniform_mod(18, n + 3, 1000)
    vals_h = np.arange(n + 3, dtype=np.uint64)
    k, v = to_dev(keys_h), to_dev(vals_h)
    ko, vo = torch.empty_like(k), torch.empty_like(v)
    ss.semisort_equal(k[1:n + 1], v[1:n + 1], keys_out=ko[3:n + 3], vals_out=vo[3:n + 3])
    torch.cuda.synchronize()
    check(keys_h[1:n + 1], vals_h[1:n + 1], to_host(ko)[3:n + 3], to_host(vo)[3:n + 3])
