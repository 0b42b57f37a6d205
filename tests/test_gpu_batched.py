"""Batched forms on the GPU: every instance's result against the CPU oracle
(bit-exact), instance layouts with empty, tiny and large instances, device-side
rejection of bad offsets, and one call captured in a CUDA graph and replayed."""
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


def instances(seed, ni, lo_log2, hi_log2, empty_every=0):
    """Seeded log-uniform instance sizes; per-instance Zipf keys with its own
    exponent and distinct-key count, keys hashed per instance."""
    u = synth.unit(synth.rand64(seed, 0x1A, np.arange(ni, dtype=np.uint64)))
    sizes = np.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.int64)
    if empty_every:
        sizes[::empty_every] = 0
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    keys = np.empty(int(off[-1]), np.uint64)
    for i in range(ni):
        m = int(sizes[i])
        if m == 0:
            continue
        s = 0.6 + 0.9 * float(synth.unit(synth.rand64(seed, 0x1B, np.array([i], np.uint64)))[0])
        d = max(2, int(np.exp(np.log(10) + (np.log(max(m, 11)) - np.log(10)) *
                              float(synth.unit(synth.rand64(seed, 0x1C, np.array([i], np.uint64)))[0]))))
        keys[int(off[i]):int(off[i + 1])] = synth.zipf(seed * 7919 + i, m, s, N=d)
    return off, keys


def check_semisort(op, off, keys, vals, ko, vo):
    for i in range(len(off) - 1):
        a, b = int(off[i]), int(off[i + 1])
        chk = oracle.check_semisort_equal if op == "equal" else oracle.check_sorted_equal
        err = chk(keys[a:b], vals[a:b], ko[a:b], vo[a:b])
        assert err is None, (i, err)


@pytest.mark.parametrize("op", ["equal", "less"])
@pytest.mark.parametrize("layout", [(300, 2, 16, 5), (4096, 8, 12, 0), (3, 18, 20, 0), (50, 0, 3, 0)])
def test_semisort_batched(ss, op, layout):
    import torch
    ni, lo, hi, empty = layout
    off, keys = instances(11 + ni, ni, lo, hi, empty)
    vals = np.arange(len(keys), dtype=np.uint64)
    k, v, o = to_dev(keys), to_dev(vals), to_dev(off)
    fn = ss.semisort_equal_batched if op == "equal" else ss.semisort_less_batched
    opt = ss.make_options(seed=2)
    ws = ss.alloc_workspace_batched(ss.OP_EQUAL if op == "equal" else ss.OP_LESS, k, o, v, opt)
    ko, vo = fn(k, v, o, workspace=ws, options=opt)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    check_semisort(op, off, keys, vals, to_host(ko), to_host(vo))


@pytest.mark.parametrize("op", ["reduce", "hist"])
@pytest.mark.parametrize("layout", [(300, 2, 16, 5), (4096, 8, 12, 0), (3, 18, 20, 0)])
def test_reduce_batched(ss, op, layout):
    import torch
    ni, lo, hi, empty = layout
    off, keys = instances(21 + ni, ni, lo, hi, empty)
    vals = synth.splitmix64_outputs(22, len(keys))
    k, o = to_dev(keys), to_dev(off)
    opt = ss.make_options(seed=2)
    if op == "reduce":
        ws = ss.alloc_workspace_batched(ss.OP_REDUCE, k, o, to_dev(vals), opt)
        uk, out, nu, oo = ss.collect_reduce_batched(k, to_dev(vals), o, workspace=ws, options=opt)
    else:
        ws = ss.alloc_workspace_batched(ss.OP_HIST, k, o, None, opt)
        uk, out, nu, oo = ss.histogram_batched(k, o, workspace=ws, options=opt)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    uk, out, nu, oo = to_host(uk), to_host(out), to_host(nu), to_host(oo)
    assert oo[0] == 0 and np.all(np.diff(oo.astype(np.int64)) == nu.astype(np.int64))
    for i in range(ni):
        a, b = int(off[i]), int(off[i + 1])
        if op == "reduce":
            rk, rs = oracle.collect_reduce_sorted(keys[a:b], vals[a:b])
        else:
            rk, rs = oracle.histogram_sorted(keys[a:b])
        assert int(nu[i]) == len(rk), i
        gk, gs = oracle.stable_sort(uk[int(oo[i]):int(oo[i + 1])], out[int(oo[i]):int(oo[i + 1])])
        assert np.array_equal(gk, rk) and np.array_equal(gs, rs), i


def test_bad_offsets_rejected_on_device(ss):
    import torch
    keys = to_dev(synth.uniform_mod(31, 10000, 100))
    vals = to_dev(np.arange(10000, dtype=np.uint64))
    off = to_dev(np.array([0, 5000, 4000, 10000], np.uint64))  # decreasing
    ws = ss.alloc_workspace_batched(ss.OP_EQUAL, keys, off, vals)
    ss.semisort_equal_batched(keys, vals, off, workspace=ws)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 1  # SS_ERR_INVALID_ARG
    off2 = to_dev(np.array([0, 5000, 9000], np.uint64))  # does not end at n
    ss.semisort_equal_batched(keys, vals, off2, workspace=ws)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 1


def test_graph_capture_replay(ss):
    """The whole batched call enqueues a fixed kernel sequence with no host
    synchronization, so it can be captured once and replayed; replays give the
    eager call's bits."""
    import torch
    off, keys = instances(41, 512, 6, 14)
    vals = np.arange(len(keys), dtype=np.uint64)
    k, v, o = to_dev(keys), to_dev(vals), to_dev(off)
    opt = ss.make_options(seed=4)
    ws = ss.alloc_workspace_batched(ss.OP_EQUAL, k, o, v, opt)
    ko, vo = torch.empty_like(k), torch.empty_like(v)
    ss.semisort_equal_batched(k, v, o, keys_out=ko, vals_out=vo, workspace=ws, options=opt)
    torch.cuda.synchronize()
    want_k, want_v = to_host(ko), to_host(vo)
    ko.zero_()
    vo.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ss.semisort_equal_batched(k, v, o, keys_out=ko, vals_out=vo, workspace=ws, options=opt, stream=s)
    for _ in range(2):
        ko.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(to_host(ko), want_k) and np.array_equal(to_host(vo), want_v)
    check_semisort("equal", off, keys, vals, want_k, want_v)


@pytest.mark.parametrize("kt", ["u64", "u32"])
def test_semisort_less_batched_learned(ss, kt):
    """Batched semisort_< in learned mode: one model trained on a sample of
    the whole batch, judged per instance; every instance's output is still
    its stable sort, and with smooth light keys the instances keep the model's
    splitters (statistics entry 12)."""
    import torch
    ni = 40
    sizes = np.floor(2.0 ** (14 + 6 * synth.unit(synth.rand64(0x1EA5, 0x1A, np.arange(ni, dtype=np.uint64)))))
    sizes = sizes.astype(np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    n = int(off[-1])
    # a Zipf head (heavy keys, equality buckets) over smooth light keys, same law in every instance
    keys = np.where(synth.uniform_mod(0x1EA6, n, 4) == 0, synth.zipf(0x1EA7, n, 1.2, N=10**6),
                    synth.splitmix64_outputs(0x1EA8, n)).astype(np.uint64)
    if kt == "u32":
        keys = (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    vals = np.arange(n, dtype=np.uint64)
    k, v, o = to_dev(keys), to_dev(vals), to_dev(off)
    res = {}
    for mode in (0, 1):
        opt = ss.make_options(seed=2, splitter_mode=mode)
        ws = ss.alloc_workspace_batched(ss.OP_LESS, k, o, v, opt)
        ko, vo = ss.semisort_less_batched(k, v, o, workspace=ws, options=opt)
        torch.cuda.synchronize()
        assert ss.last_device_error(ws) == 0
        res[mode] = (to_host(ko), to_host(vo), ss.stats(ws))
    check_semisort("less", off, keys, vals, res[1][0], res[1][1])
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert res[1][2]["l0_max_sample_range"] > 0, res[1][2]  # instances that kept the model's splitters
