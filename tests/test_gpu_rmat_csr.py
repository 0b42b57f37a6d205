"""CSR build from an R-MAT edge list (u32 src, u32 dst) over 64 uneven edge
partitions: batched semisort_< on src (dst as value) gives each partition's
edges grouped by source in source order with destinations in input order,
and batched histogram gives the degrees; both bit-exact against the oracle."""
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


def partitions(seed, m, parts=64):
    """Contiguous edge ranges with seeded log-uniform sizes 2^U[0,4], scaled to m."""
    w = 2.0 ** (4.0 * synth.unit(synth.rand64(seed, 0x9A, np.arange(parts, dtype=np.uint64))))
    cut = np.floor(np.cumsum(w) / w.sum() * m).astype(np.int64)
    cut[-1] = m
    return np.concatenate([[0], cut]).astype(np.uint64)


@pytest.mark.parametrize("scale,m", [(16, 1 << 20), (20, 3 << 20)])
def test_rmat_csr_batched(ss, scale, m):
    import torch
    src, dst = synth.rmat_edges(0x5EED0005, m, scale)
    off = partitions(0x5EED0005, m)
    s, d, o = to_dev(src), to_dev(dst), to_dev(off)
    ks, vs = ss.semisort_less_batched(s, d, o)
    uk, cnt, nu, oo = ss.histogram_batched(s, o)
    torch.cuda.synchronize()
    ks, vs, uk, cnt, nu, oo = (to_host(t) for t in (ks, vs, uk, cnt, nu, oo))
    for p in range(len(off) - 1):
        a, b = int(off[p]), int(off[p + 1])
        err = oracle.check_sorted_equal(src[a:b], dst[a:b], ks[a:b], vs[a:b])
        assert err is None, (p, err)
        rk, rc = oracle.histogram_sorted(src[a:b])
        gk, gc = oracle.stable_sort(uk[int(oo[p]):int(oo[p + 1])], cnt[int(oo[p]):int(oo[p + 1])])
        assert int(nu[p]) == len(rk) and np.array_equal(gk, rk) and np.array_equal(gc, rc), p
        # CSR row offsets of the partition agree with the sorted sources
        rows = np.searchsorted(ks[a:b], rk, side="left")
        assert np.array_equal(np.diff(np.append(rows, b - a)), rc.astype(np.int64))


def test_rmat_single_partition_learned(ss):
    """A single partition with learned splitters: the same exact CSR order."""
    import torch
    m = 1 << 21
    src, dst = synth.rmat_edges(0x5EED0006, m, 20)
    o = ss.make_options(seed=1, splitter_mode=1)
    ks, vs = ss.semisort_less(to_dev(src), to_dev(dst), options=o)
    torch.cuda.synchronize()
    assert oracle.check_sorted_equal(src, dst, to_host(ks), to_host(vs)) is None
