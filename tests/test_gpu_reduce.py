"""GPU parity of collect-reduce and histogram against the CPU oracle.  The
output order is unspecified, so both sides are compared sorted by key: the
unique keys, the u64 wraparound sums / u32 counts and the unique count must be
bit-exact."""
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


def run_reduce(ss, keys_h, vals_h, seed=1, capacity=None, **opt):
    import torch
    keys = to_dev(keys_h)
    o = ss.make_options(seed=seed, **opt)
    if vals_h is None:
        ws = ss.alloc_workspace(ss.OP_HIST, keys, None, o)
        uk, out, nu = ss.histogram(keys, capacity=capacity, workspace=ws, options=o)
    else:
        vals = to_dev(vals_h)
        ws = ss.alloc_workspace(ss.OP_REDUCE, keys, vals, o)
        uk, out, nu = ss.collect_reduce(keys, vals, capacity=capacity, workspace=ws, options=o)
    torch.cuda.synchronize()
    err = ss.last_device_error(ws)
    u = int(to_host(nu)[0])
    st = ss.stats(ws)
    return to_host(uk), to_host(out), u, err, st


def check(keys_h, vals_h, uk, out, u):
    if vals_h is None:
        rk, rs = oracle.histogram_sorted(keys_h)
    else:
        rk, rs = oracle.collect_reduce_sorted(keys_h, vals_h)
    assert u == len(rk), (u, len(rk))
    gk, gs = oracle.stable_sort(uk[:u], out[:u])
    assert np.array_equal(gk, rk), "unique keys differ"
    assert np.array_equal(gs, rs), "sums/counts differ"


WORKLOADS = ["config1", "all_equal", "all_distinct", "one_heavy", "zipf15", "zipf08", "uniform_exact_1e3",
             "exponential"]


def make_keys(kind, n):
    if kind == "config1":
        return synth.uniform_mod(0x5EED0001, n, 10**4)
    if kind == "all_equal":
        return np.full(n, 77, np.uint64)
    if kind == "all_distinct":
        return synth.splitmix64_outputs(41, n)
    if kind == "one_heavy":
        k = synth.uniform_mod(42, n, 10**6)
        k[synth.uniform_mod(43, n, 10) < 6] = 7
        return k
    if kind == "zipf15":
        return synth.zipf(44, n, 1.5, N=10**9)
    if kind == "zipf08":
        return synth.zipf(45, n, 0.8, N=10**9)
    if kind == "uniform_exact_1e3":
        return synth.uniform_exact(46, n, 1000)
    return synth.exponential(47, n, 1e-4)


@pytest.mark.parametrize("kind", WORKLOADS)
def test_collect_reduce(ss, kind):
    n = 1 << 20
    keys = make_keys(kind, n)
    vals = synth.splitmix64_outputs(48, n)  # full-range values: sums wrap around
    uk, out, u, err, _ = run_reduce(ss, keys, vals)
    assert err == 0
    check(keys, vals, uk, out, u)


@pytest.mark.parametrize("kind", WORKLOADS)
def test_histogram(ss, kind):
    n = 1 << 20
    keys = make_keys(kind, n)
    uk, out, u, err, _ = run_reduce(ss, keys, None)
    assert err == 0
    check(keys, None, uk, out, u)


@pytest.mark.parametrize("n", [1, 2, 63, 64, 4095, 4096, 4097, 8193, 65537, 300001])
@pytest.mark.parametrize("op", ["reduce", "hist"])
def test_edge_sizes(ss, n, op):
    rng = np.random.default_rng(2000 + n)
    keys = rng.integers(0, max(2, n // 3), size=n, dtype=np.uint64)
    vals = None if op == "hist" else np.arange(n, dtype=np.uint64)
    uk, out, u, err, _ = run_reduce(ss, keys, vals)
    assert err == 0
    check(keys, vals, uk, out, u)


def test_empty(ss):
    import torch
    k = torch.empty(0, dtype=torch.uint64, device="cuda")
    _, _, nu = ss.collect_reduce(k, k.clone(), capacity=0)
    _, _, nh = ss.histogram(k, capacity=0)
    torch.cuda.synchronize()
    assert int(to_host(nu)[0]) == 0 and int(to_host(nh)[0]) == 0


def test_recursion(ss):
    n = 1 << 24
    keys = synth.uniform_exact(49, n, 1 << 22)
    vals = np.arange(n, dtype=np.uint64)
    uk, out, u, err, st = run_reduce(ss, keys, vals)
    assert err == 0 and st["levels"] >= 2
    check(keys, vals, uk, out, u)
    # exact multiplicity: every key occurs n / mu = 4 times
    uk, cnt, u, err, _ = run_reduce(ss, keys, None)
    assert err == 0 and u == 1 << 22 and np.all(cnt[:u] == 4)


def test_index_values_closed_form(ss):
    """value = index: the sums add up to n(n-1)/2 (mod 2^64)."""
    n = 3 * (1 << 20) + 5
    keys = synth.zipf(50, n, 1.0, N=10**9)
    vals = np.arange(n, dtype=np.uint64)
    uk, out, u, err, _ = run_reduce(ss, keys, vals)
    assert err == 0
    assert int(out[:u].sum(dtype=np.uint64)) == (n * (n - 1) // 2) % 2**64


def test_capacity_exceeded(ss):
    """Too small an output: the device flag reports SS_ERR_CAPACITY and the
    unique count still tells the caller how much room is needed."""
    n = 1 << 16
    keys = synth.uniform_exact(51, n, 1000)
    uk, out, u, err, _ = run_reduce(ss, keys, None, capacity=100)
    assert err == 4 and u == 1000


def test_deterministic(ss):
    n = 1 << 21
    keys = synth.zipf(52, n, 1.1, N=10**7)
    vals = np.arange(n, dtype=np.uint64)
    a = run_reduce(ss, keys, vals, seed=3)
    b = run_reduce(ss, keys, vals, seed=3)
    assert np.array_equal(a[0][:a[2]], b[0][:b[2]]) and np.array_equal(a[1][:a[2]], b[1][:b[2]])


@pytest.mark.parametrize("alpha,subarray,lbits", [(256, 4096, 3), (4096, 65536, 1)])
def test_parameters(ss, alpha, subarray, lbits):
    n = 1 << 21
    keys = synth.zipf(53, n, 1.1, N=10**6)
    vals = synth.splitmix64_outputs(54, n)
    uk, out, u, err, _ = run_reduce(ss, keys, vals, alpha=alpha, subarray=subarray, n_light_log2=lbits)
    assert err == 0
    check(keys, vals, uk, out, u)


@pytest.mark.parametrize("n", [2, 100, 4096])
@pytest.mark.parametrize("op", ["reduce", "hist"])
def test_single_window_all_distinct(ss, n, op):
    """n <= alpha: the whole input is one base case read from the caller's
    arrays; with all keys distinct the window is its own output and is copied
    to the temporary before the pack (the in-place shortcut applies only to
    windows already in a temporary)."""
    keys = synth.splitmix64_outputs(60 + n, n)
    vals = None if op == "hist" else synth.splitmix64_outputs(61 + n, n)
    uk, out, u, err, st = run_reduce(ss, keys, vals)
    assert err == 0
    assert u == n
    assert st["all_distinct"] == n
    check(keys, vals, uk, out, u)
