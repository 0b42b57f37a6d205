"""SS_FLAG_SWAP_OUTPUT: semisort_= and semisort_< with one temporary array,
the distribution levels alternating between it and the caller's output
arrays (the swap of A and T, Sec. 3.4).  Same contract as the default path,
checked against the oracle on inputs that reach three and more levels (so
that a level reads the output arrays), in place, keys only, 32- and 128-bit
keys, and the batched form; the workspace is smaller."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import to_dev, to_host
from tests.test_gpu_deep_levels import deep_keys

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ss():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2304_10078_gb300 as m
    m.build()
    return m


def run(ss, op, keys_h, vals_h, in_place=False, **kw):
    import torch
    keys = to_dev(keys_h) if keys_h.ndim == 1 else torch.from_numpy(keys_h.view(np.int64)).cuda().view(torch.uint64)
    vals = None if vals_h is None else to_dev(vals_h)
    o = ss.make_options(seed=4, flags=ss.FLAG_SWAP_OUTPUT, **kw)
    code = ss.OP_EQUAL if op == "equal" else ss.OP_LESS
    ws = ss.alloc_workspace(code, keys, vals, o)
    fn = ss.semisort_equal if op == "equal" else ss.semisort_less
    if in_place:
        ko, vo = fn(keys, vals, keys_out=keys, vals_out=vals, workspace=ws, options=o)
    else:
        ko, vo = fn(keys, vals, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    st = ss.stats(ws)
    kh = to_host(ko) if keys_h.ndim == 1 else ko.view(torch.int64).cpu().numpy().view(np.uint64)
    return kh, None if vo is None else to_host(vo), st


def check(op, keys, vals, ko, vo):
    chk = oracle.check_semisort_equal if op == "equal" else oracle.check_sorted_equal
    err = chk(keys, vals, ko, vo)
    assert err is None, err


@pytest.mark.parametrize("op", ["equal", "less"])
def test_swap_deep_levels(ss, op):
    n = 1 << 22
    keys = deep_keys(0xDEE9, n)
    vals = synth.splitmix64_outputs(0xDEEA, n)
    ko, vo, st = run(ss, op, keys, vals, alpha=256, subarray=4096, n_light_log2=3)
    assert st["levels"] >= 3, st
    check(op, keys, vals, ko, vo)


@pytest.mark.parametrize("op", ["equal", "less"])
@pytest.mark.parametrize("case", ["config1", "in_place", "keys_only", "u32", "u128", "zipf15"])
def test_swap_cases(ss, op, case):
    n = (1 << 20) + 77
    keys = synth.uniform_mod(0x5EED0001, n, 10**4)
    vals = np.arange(n, dtype=np.uint64)
    if case == "keys_only":
        vals = None
    elif case == "u32":
        keys = (keys * np.uint64(2654435761) >> np.uint64(7)).astype(np.uint32)
    elif case == "u128":
        keys = np.stack([keys, synth.key_of_rank(5, keys)], axis=1)
    elif case == "zipf15":
        keys = synth.zipf(0x5EA5, n, 1.5)
    ko, vo, _ = run(ss, op, keys, vals, in_place=case == "in_place", alpha=512)
    if vals is None:
        ref = np.sort(keys, kind="stable") if op == "less" else None
        if op == "less":
            assert np.array_equal(ko, ref)
        else:
            assert oracle.count_runs(ko) == oracle.count_distinct(keys)
            assert np.array_equal(np.sort(ko), np.sort(keys))
    else:
        check(op, keys, vals, ko, vo)


def test_swap_workspace_smaller(ss):
    n = 10**8
    plain = ss.workspace_size(ss.OP_EQUAL, ss.SS_U64, ss.SS_U64, n, ss.make_options(seed=1))
    swap = ss.workspace_size(ss.OP_EQUAL, ss.SS_U64, ss.SS_U64, n, ss.make_options(seed=1, flags=ss.FLAG_SWAP_OUTPUT))
    assert swap < 0.6 * plain and plain - swap >= 16 * n


@pytest.mark.parametrize("op", ["equal", "less"])
def test_swap_batched(ss, op):
    import torch
    from tests.test_gpu_batched import check_semisort, instances
    off, keys = instances(77, 300, 2, 17, 5)
    vals = np.arange(len(keys), dtype=np.uint64)
    k, v, o = to_dev(keys), to_dev(vals), to_dev(off)
    fn = ss.semisort_equal_batched if op == "equal" else ss.semisort_less_batched
    opt = ss.make_options(seed=2, flags=ss.FLAG_SWAP_OUTPUT)
    ws = ss.alloc_workspace_batched(ss.OP_EQUAL if op == "equal" else ss.OP_LESS, k, o, v, opt)
    ko, vo = fn(k, v, o, workspace=ws, options=opt)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    check_semisort(op, off, keys, vals, to_host(ko), to_host(vo))
