"""GPU parity of semisort_< against the CPU oracle: the output must equal the
stable sort of the input by key, bit for bit (keys and values)."""
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


def run_less(ss, keys_h, vals_h, seed=1, inplace=False, **opt):
    import torch
    keys = to_dev(keys_h)
    vals = None if vals_h is None else to_dev(vals_h)
    o = ss.make_options(seed=seed, **opt)
    ws = ss.alloc_workspace(ss.OP_LESS, keys, vals, o)
    if inplace:
        ko, vo = ss.semisort_less(keys, vals, keys_out=keys, vals_out=vals, workspace=ws, options=o)
    else:
        ko, vo = ss.semisort_less(keys, vals, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    st = ss.stats(ws)
    return to_host(ko), (None if vo is None else to_host(vo)), st


def check(keys_h, vals_h, ko, vo):
    err = oracle.check_sorted_equal(keys_h, vals_h, ko, vo)
    assert err is None, err


def test_config1_uniform_1e4(ss):
    n = 1 << 20
    keys = synth.uniform_mod(0x5EED0001, n, 10**4)
    vals = np.arange(n, dtype=np.uint64)
    ko, vo, _ = run_less(ss, keys, vals)
    check(keys, vals, ko, vo)


@pytest.mark.parametrize("n", [1, 2, 3, 31, 255, 256, 257, 4095, 4096, 4097, 8193, 65537, 300001])
def test_edge_sizes(ss, n):
    rng = np.random.default_rng(1000 + n)
    keys = rng.integers(0, max(2, n // 5), size=n, dtype=np.uint64)
    vals = np.arange(n, dtype=np.uint64)
    ko, vo, _ = run_less(ss, keys, vals)
    check(keys, vals, ko, vo)


def test_empty(ss):
    import torch
    k = torch.empty(0, dtype=torch.uint64, device="cuda")
    ko, vo = ss.semisort_less(k, k.clone())
    assert ko.numel() == 0


@pytest.mark.parametrize("kind", ["all_equal", "all_distinct", "one_heavy", "sorted", "reversed", "zipf12",
                                  "exponential", "gaussian_mixture", "uniform_exact_1e5", "extremes"])
def test_distributions(ss, kind):
    n = 1 << 21
    if kind == "all_equal":
        keys = np.full(n, 12345, np.uint64)
    elif kind == "all_distinct":
        keys = synth.splitmix64_outputs(21, n)
    elif kind == "one_heavy":
        keys = synth.uniform_mod(22, n, 10**9)
        keys[synth.uniform_mod(23, n, 10) < 4] = 5
    elif kind == "sorted":
        keys = np.sort(synth.uniform_mod(24, n, 10**6))
    elif kind == "reversed":
        keys = np.sort(synth.uniform_mod(25, n, 10**6))[::-1].copy()
    elif kind == "zipf12":
        keys = synth.zipf(26, n, 1.2, N=10**9)
    elif kind == "exponential":
        keys = synth.exponential(27, n, 1e-6)
    elif kind == "gaussian_mixture":
        keys = synth.gaussian_mixture(28, n)
    elif kind == "uniform_exact_1e5":
        keys = synth.uniform_exact(29, n, 10**5)
    else:
        sel = synth.uniform_mod(30, n, 4)
        keys = np.where(sel == 0, np.uint64(0), np.where(sel == 1, np.uint64(2**64 - 1),
                                                         synth.splitmix64_outputs(31, n)))
    vals = np.arange(n, dtype=np.uint64)
    ko, vo, _ = run_less(ss, keys, vals)
    check(keys, vals, ko, vo)


def test_recursion(ss):
    """2^24 records, 2^23 distinct keys: range buckets recurse (at least two
    distribution levels)."""
    n = 1 << 24
    keys = synth.uniform_exact(32, n, 1 << 23)
    vals = np.arange(n, dtype=np.uint64)
    ko, vo, st = run_less(ss, keys, vals)
    assert st["levels"] >= 2
    check(keys, vals, ko, vo)


@pytest.mark.parametrize("vdtype", ["u32", "none"])
def test_value_types(ss, vdtype):
    n = 1 << 20
    keys = synth.zipf(33, n, 0.9, N=10**7)
    vals = None if vdtype == "none" else np.arange(n, dtype=np.uint32)[::-1].copy()
    ko, vo, _ = run_less(ss, keys, vals)
    if vals is None:
        assert np.array_equal(ko, oracle.stable_sort(keys)[0])
    else:
        check(keys, vals, ko, vo)


@pytest.mark.parametrize("n", [3000, 1 << 20, 1 << 23])
def test_in_place(ss, n):
    keys = synth.zipf(34, n, 1.2, N=10**6)
    vals = np.arange(n, dtype=np.uint64)
    ko, vo, _ = run_less(ss, keys, vals, inplace=True)
    check(keys, vals, ko, vo)


@pytest.mark.parametrize("alpha,subarray,lbits", [(256, 4096, 3), (1024, 8192, 8), (4096, 65536, 1)])
def test_parameters(ss, alpha, subarray, lbits):
    n = 1 << 21
    keys = synth.zipf(35, n, 1.1, N=10**6)
    vals = np.arange(n, dtype=np.uint64)
    ko, vo, _ = run_less(ss, keys, vals, alpha=alpha, subarray=subarray, n_light_log2=lbits)
    check(keys, vals, ko, vo)


@pytest.mark.parametrize("n", [3000, 1 << 20])
def test_clustered_keys(ss, n):
    """Far outliers stretch the key range so that clustered keys share one
    interpolation bucket of their window: the base case must still sort them."""
    rng = np.random.default_rng(n)
    keys = rng.integers(1000, 1000 + 4 * n, size=n, dtype=np.uint64)
    keys[::97] = np.uint64(2**63) + rng.integers(0, 10, size=len(keys[::97]), dtype=np.uint64)
    keys[5] = np.uint64(2**64 - 1)
    vals = np.arange(n, dtype=np.uint64)
    ko, vo, _ = run_less(ss, keys, vals)
    check(keys, vals, ko, vo)


def _window_with_runs(seed, n, runs, dup):
    """One base-case window (n <= alpha) whose keys span [0, 2^40): the
    interpolation bucket of the base case is then 2^25 keys wide, and each
    entry L of `runs` puts L keys into one bucket (its own) in an order with
    inversions -- descending distinct keys, or (dup) three key values
    interleaved, so equal keys also test stability.  The other keys are
    spread over the range."""
    rng = np.random.default_rng(seed)
    parts = [np.array([0, (1 << 40) - 1], dtype=np.uint64)]
    for j, L in enumerate(runs):
        base = np.uint64((8 + 64 * j) << 25)
        if dup:
            k = base + rng.integers(0, 3, size=L, dtype=np.uint64) * np.uint64(1 << 20)
        else:
            k = base + (np.arange(L, 0, -1, dtype=np.uint64) * np.uint64(7))
        parts.append(k)
    rest = n - sum(len(p) for p in parts)
    parts.append(rng.integers(0, 1 << 40, size=rest, dtype=np.uint64))
    # a random order of all keys keeps inversions inside every run
    return np.concatenate(parts)[rng.permutation(n)]


@pytest.mark.parametrize("runs", [[2], [63, 64], [65], [64, 65, 64], [200], [1000, 3]])
@pytest.mark.parametrize("dup", [False, True])
def test_base_case_unordered_runs(ss, runs, dup):
    """Runs of equal interpolation buckets that hold inversions: up to 64
    records they are ordered in parallel, longer ones send the window to the
    bitonic network; either way the output is the stable sort."""
    n = 4096
    keys = _window_with_runs(7 + len(runs) + (100 if dup else 0), n, runs, dup)
    vals = np.arange(n, dtype=np.uint64)
    ko, vo, st = run_less(ss, keys, vals)
    check(keys, vals, ko, vo)
    assert st["refined"] == n
