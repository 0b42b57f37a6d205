"""GPU parity for the 32-bit and 128-bit key types (Sec. 2.1 allows any key
type with = / < and a hash; the library builds in u32, u64 and u128).  All
four operations are checked against the CPU oracle, bit-exact."""
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


def keys_of(kind, n, seed):
    if kind == "u32":
        return (synth.zipf(seed, n, 1.0, N=10**6) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    # 128-bit: hi carries the key identity, lo a function of it, and a quarter
    # of the keys share hi with a different lo (ordering and equality need both words)
    r = synth.zipf(seed, n, 1.0, N=10**6)
    hi = synth.mix64_np(r) >> np.uint64(40)
    lo = synth.mix64_np(r ^ np.uint64(0x77))
    lo = np.where((r & np.uint64(3)) == 0, lo ^ np.uint64(1), lo)
    return np.stack([lo, hi], axis=1).copy()


def run(ss, op, keys_h, vals_h, **opt):
    import torch
    keys = to_dev(keys_h)
    vals = None if vals_h is None else to_dev(vals_h)
    o = ss.make_options(seed=3, **opt)
    ws = ss.alloc_workspace(op, keys, vals, o)
    if op in (ss.OP_EQUAL, ss.OP_LESS):
        fn = ss.semisort_equal if op == ss.OP_EQUAL else ss.semisort_less
        ko, vo = fn(keys, vals, workspace=ws, options=o)
        res = (to_host(ko), None if vo is None else to_host(vo))
    elif op == ss.OP_REDUCE:
        uk, sums, nu = ss.collect_reduce(keys, vals, workspace=ws, options=o)
        u = int(to_host(nu)[0])
        res = (to_host(uk)[:u], to_host(sums)[:u])
    else:
        uk, cnt, nu = ss.histogram(keys, workspace=ws, options=o)
        u = int(to_host(nu)[0])
        res = (to_host(uk)[:u], to_host(cnt)[:u])
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    return res


@pytest.mark.parametrize("kt", ["u32", "u128"])
@pytest.mark.parametrize("vt", ["u32", "u64", "none"])
@pytest.mark.parametrize("n", [3000, 1 << 20])
def test_semisort_equal(ss, kt, vt, n):
    keys = keys_of(kt, n, 70)
    vals = None if vt == "none" else np.arange(n, dtype=np.uint32 if vt == "u32" else np.uint64)
    ko, vo = run(ss, ss.OP_EQUAL, keys, vals)
    if vals is None:
        assert np.array_equal(oracle.stable_sort(ko)[0], oracle.stable_sort(keys)[0])
        assert oracle.count_runs(ko) == oracle.count_distinct(keys)
    else:
        err = oracle.check_semisort_equal(keys, vals, ko, vo)
        assert err is None, err


@pytest.mark.parametrize("kt", ["u32", "u128"])
@pytest.mark.parametrize("vt", ["u32", "u64", "none"])
@pytest.mark.parametrize("n", [3000, 1 << 20])
def test_semisort_less(ss, kt, vt, n):
    keys = keys_of(kt, n, 71)
    vals = None if vt == "none" else np.arange(n, dtype=np.uint32 if vt == "u32" else np.uint64)
    ko, vo = run(ss, ss.OP_LESS, keys, vals)
    if vals is None:
        assert np.array_equal(ko, oracle.stable_sort(keys)[0])
    else:
        err = oracle.check_sorted_equal(keys, vals, ko, vo)
        assert err is None, err


@pytest.mark.parametrize("kt", ["u32", "u128"])
@pytest.mark.parametrize("n", [3000, 1 << 20])
def test_collect_reduce_and_histogram(ss, kt, n):
    keys = keys_of(kt, n, 72)
    vals = synth.splitmix64_outputs(73, n)
    uk, sums = run(ss, ss.OP_REDUCE, keys, vals)
    rk, rs = oracle.collect_reduce_sorted(keys, vals)
    gk, gs = oracle.stable_sort(uk, sums)
    assert np.array_equal(gk, rk) and np.array_equal(gs, rs)
    uk, cnt = run(ss, ss.OP_HIST, keys, None)
    rk, rc = oracle.histogram_sorted(keys)
    gk, gc = oracle.stable_sort(uk, cnt)
    assert np.array_equal(gk, rk) and np.array_equal(gc, rc)


@pytest.mark.parametrize("kt", ["u32", "u128"])
def test_recursion(ss, kt):
    n = 1 << 23
    if kt == "u32":
        keys = synth.uniform_exact(74, n, 1 << 21).astype(np.uint32)
    else:
        k = synth.uniform_exact(74, n, 1 << 21)
        keys = np.stack([k, k >> np.uint64(7)], axis=1).copy()
    vals = np.arange(n, dtype=np.uint64)
    ko, vo = run(ss, ss.OP_EQUAL, keys, vals)
    assert oracle.check_semisort_equal(keys, vals, ko, vo) is None
    ko, vo = run(ss, ss.OP_LESS, keys, vals)
    assert oracle.check_sorted_equal(keys, vals, ko, vo) is None
