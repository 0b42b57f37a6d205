"""semisort_equal_noalloc: the static-scratch entry point gives the same output
as semisort_equal with a caller workspace, on consecutive calls that share the
library's scratch array.  Collected last so that it also runs after every
other GPU test in the same process."""
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


def reference(ss, keys, vals, opts):
    ws = ss.alloc_workspace(ss.OP_EQUAL, keys, vals, opts)
    ko, vo = ss.semisort_equal(keys, vals, workspace=ws, options=opts)
    return to_host(ko), to_host(vo)


def test_two_calls_match_workspace_entry_point(ss):
    import torch
    opts = ss.make_options(seed=7)
    cases = [(synth.uniform_mod(61, 1 << 18, 3000), np.arange(1 << 18, dtype=np.uint64)),
             (synth.zipf(62, 100003, 1.2, N=10**6), np.arange(100003, dtype=np.uint64)[::-1].copy())]
    for keys_h, vals_h in cases:
        keys, vals = to_dev(keys_h), to_dev(vals_h)
        ko = torch.empty_like(keys)
        vo = torch.empty_like(vals)
        ss.semisort_equal_noalloc(keys, vals, ko, vo, options=opts)
        got_k, got_v = to_host(ko), to_host(vo)
        want_k, want_v = reference(ss, keys, vals, opts)
        torch.cuda.synchronize()
        assert np.array_equal(got_k, want_k) and np.array_equal(got_v, want_v)
        assert oracle.check_semisort_equal(keys_h, vals_h, got_k, got_v) is None


def test_size_limit(ss):
    import torch
    n = (1 << 18) + 1
    keys = torch.zeros(n, dtype=torch.uint64, device="cuda")
    with pytest.raises(ss.SemisortError) as e:
        ss.semisort_equal_noalloc(keys, None, torch.empty_like(keys), None)
    assert e.value.code == 2  # SS_ERR_UNSUPPORTED
