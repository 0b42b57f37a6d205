"""The C++ template entry points (include/semisort.hpp) with a user-defined
key type and a non-commutative monoid, through the test instantiations in
tests/user_types/user_types.cu:

* Key12 (three 32-bit words, a 96-bit order) with semisort_= and semisort_<,
  compared with the oracle on the equivalent 128-bit keys, at sizes that span
  several levels and tiles, with a ragged tail, and with forced deep levels;
* collect-reduce with the Horner monoid (h1, p1) op (h2, p2) =
  (h1 p2 + h2, p1 p2) mod 2^64 -- associative, not commutative, so each
  key's result depends on its values being combined in input order (Sec. 3.5)
  -- compared with the oracle's ordered fold, for Key12 and u64 keys,
  including one key whose records span hundreds of fold tiles."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "user_types", "user_types.cu")
LIB = os.path.join(HERE, "_lib", "libusertypes.so")
M = 0x9E3779B97F4A7C15 | 1
MASK = 2**64 - 1


def build_lib():
    deps = [SRC, os.path.join(ROOT, "include", "semisort.hpp")] + [
        os.path.join(ROOT, "paper_2304_10078_gb300", "csrc", f)
        for f in os.listdir(os.path.join(ROOT, "paper_2304_10078_gb300", "csrc"))]
    if os.path.exists(LIB) and all(os.path.getmtime(d) <= os.path.getmtime(LIB) for d in deps):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    subprocess.check_call(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                           "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-I",
                           os.path.join(ROOT, "include"), "-shared", "-o", LIB + ".tmp", SRC])
    os.replace(LIB + ".tmp", LIB)
    return LIB


@pytest.fixture(scope="module")
def ut():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    L = ctypes.CDLL(build_lib())
    vp, u64, u32, i32, sz = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_size_t
    L.ut_workspace.argtypes = [i32, u64, u32, u32, u32]
    L.ut_workspace.restype = sz
    L.ut_semisort.argtypes = [i32, vp, vp, vp, vp, u64, vp, sz, u64, u32, u32, u32, vp]
    L.ut_semisort.restype = i32
    L.ut_fold_workspace.argtypes = [u64, i32]
    L.ut_fold_workspace.restype = sz
    L.ut_fold.argtypes = [i32, vp, vp, vp, vp, u64, vp, u64, vp, sz, u64, vp]
    L.ut_fold.restype = i32
    return L


def key12(seed, n, distinct):
    """(n, 3) uint32 words (a, b, c) of `distinct` seeded key values."""
    r = synth.uniform_mod(seed, n, distinct)
    w = synth.key_of_rank(seed + 1, r)
    c = (synth.key_of_rank(seed + 2, r) & np.uint64(0xF)).astype(np.uint32)
    return np.stack([(w & np.uint64(0xFFFFFFFF)).astype(np.uint32), (w >> np.uint64(32)).astype(np.uint32), c],
                    axis=1)


def as128(k3):
    """The 128-bit key (lo = a | b << 32, hi = c) with the same order."""
    lo = k3[:, 0].astype(np.uint64) | (k3[:, 1].astype(np.uint64) << np.uint64(32))
    return np.stack([lo, k3[:, 2].astype(np.uint64)], axis=1)


def dev(a):
    import torch
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(np.uint8).reshape(-1).copy()).cuda()


def host(t, dtype, shape):
    return t.cpu().numpy().view(dtype).reshape(shape)


def run_semisort(ut, op, k3, vals, seed=1, alpha=0, subarray=0, lbits=0):
    import torch
    n = len(vals)
    ws = torch.empty(max(256, ut.ut_workspace(op, n, alpha, subarray, lbits)), dtype=torch.uint8, device="cuda")
    dk, dv = dev(k3), dev(vals)
    ko, vo = torch.empty_like(dk), torch.empty_like(dv)
    st = torch.cuda.current_stream().cuda_stream
    rc = ut.ut_semisort(op, dk.data_ptr(), dv.data_ptr(), ko.data_ptr(), vo.data_ptr(), n, ws.data_ptr(),
                        ws.numel(), seed, alpha, subarray, lbits, st)
    torch.cuda.synchronize()
    assert rc == 0
    return host(ko, np.uint32, (n, 3)), host(vo, np.uint64, (n,))


@pytest.mark.parametrize("n,distinct", [(1, 1), (4097, 300), (300_001, 5000), (1 << 21, 1 << 19),
                                        (1 << 20, 3)])
@pytest.mark.parametrize("op", [0, 1])
def test_key12_semisort_matches_oracle(ut, n, distinct, op):
    k3 = key12(0x7E57 + n, n, distinct)
    vals = np.arange(n, dtype=np.uint64)
    ko, vo = run_semisort(ut, op, k3, vals)
    if op == 0:
        err = oracle.check_semisort_equal(as128(k3), vals, as128(ko), vo)
    else:
        err = oracle.check_sorted_equal(as128(k3), vals, as128(ko), vo)
    assert err is None, err


@pytest.mark.parametrize("op", [0, 1])
def test_key12_semisort_deep_levels(ut, op):
    n = 1 << 21
    k3 = key12(0x7E58, n, 1 << 18)
    vals = np.arange(n, dtype=np.uint64)
    ko, vo = run_semisort(ut, op, k3, vals, seed=3, alpha=256, subarray=4096, lbits=3)
    check = oracle.check_semisort_equal if op == 0 else oracle.check_sorted_equal
    err = check(as128(k3), vals, as128(ko), vo)
    assert err is None, err


def horner(x, y):
    return ((x[0] * y[1] + y[0]) & MASK, (x[1] * y[1]) & MASK)


def run_fold(ut, key12_mode, keys, xs, seed=1):
    import torch
    n = len(xs)
    vals = np.stack([xs, np.full(n, M, np.uint64)], axis=1)
    ws = torch.empty(max(256, ut.ut_fold_workspace(n, key12_mode)), dtype=torch.uint8, device="cuda")
    dk, dv = dev(keys), dev(vals)
    uk, sums = torch.empty_like(dk), torch.empty_like(dv)
    nu = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = ut.ut_fold(key12_mode, dk.data_ptr(), dv.data_ptr(), uk.data_ptr(), sums.data_ptr(), n, nu.data_ptr(), n,
                    ws.data_ptr(), ws.numel(), seed, st)
    torch.cuda.synchronize()
    assert rc == 0
    u = int(nu.item())
    shape = (n, 3) if key12_mode else (n,)
    return host(uk, np.uint32 if key12_mode else np.uint64, shape)[:u], host(sums, np.uint64, (n, 2))[:u], vals


def canon(keys, sums):
    order = np.lexsort(tuple(keys.T)) if keys.ndim == 2 else np.argsort(keys, kind="stable")
    return keys[order], [tuple(int(x) for x in sums[i]) for i in order]


@pytest.mark.parametrize("case", ["key12", "u64", "u64_one_dominant_key", "key12_tiny"])
def test_noncommutative_collect_reduce_matches_oracle(ut, case):
    if case == "key12":
        n = 200_003
        keys = key12(0xF01D, n, 4000)
    elif case == "key12_tiny":
        n = 37
        keys = key12(0xF01E, n, 5)
    elif case == "u64":
        n = 250_000
        keys = synth.zipf(0xF01F, n, 1.1, N=10**5)
    else:
        n = 1 << 20  # one key holds ~60% of the records: its run spans ~150 fold tiles
        keys = synth.uniform_mod(0xF020, n, 10**4)
        keys[synth.uniform_mod(0xF021, n, 10) < 6] = np.uint64(12345)
    xs = synth.splitmix64_outputs(0xF022, n)
    gk, gs, vals = run_fold(ut, 1 if case.startswith("key12") else 0, keys, xs)
    okeys = as128(keys) if case.startswith("key12") else keys
    ok, ov = oracle.collect_reduce_fold(okeys, [(int(a), int(b)) for a, b in vals], horner, (0, 1))
    assert len(gk) == len(ok)
    gk_c, gs_c = canon(as128(gk) if case.startswith("key12") else gk, gs)
    ok_c, os_c = canon(ok, [list(v) for v in ov])
    assert np.array_equal(gk_c, ok_c), "unique keys differ"
    assert gs_c == os_c, "folded values differ"
