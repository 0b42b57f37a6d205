"""Plain CPU oracle for semisort_=, semisort_<, collect-reduce and histogram.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product library never
imports this package, and this package never imports the product library.

Every function is the plain definition of the problem (Sec. 2.1 of the paper):

* ``stable_sort``       -- semisort_< and the canonical form of semisort_=.
* ``group_by``          -- semisort_= as a first-occurrence hash group-by
                           (the chained hash table base case of Sec. 3.3).
* ``collect_reduce_*``  -- (unique key, sum of values mod 2^64), Sec. 2.1 with
                           the (+, 0) monoid used in Sec. 5.2.
* ``histogram_*``       -- (unique key, count), Sec. 2.1.
* ``check_semisort_equal`` -- acceptance test for any semisort_= output.

Parity status: every function here is pinned in ``tests/test_oracle_pins.py``
against O(n^2) brute force, closed forms and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.cpp")
_lock = threading.Lock()
_lib = None

KT = {np.dtype(np.uint32): 0, np.dtype(np.uint64): 1}
VT = {np.dtype(np.uint32): 0, np.dtype(np.uint64): 1}


_LIB_PAR = os.path.join(_LIBDIR, "liboracle_par.so")
_SRC_PAR = os.path.join(_HERE, "oracle_parallel.cpp")
_lib_par = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (no CUDA involved); the
    all-core stable sort is a separate OpenMP library (build_parallel)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def build_parallel(force: bool = False) -> str:
    """Compile the all-core stable sort (libstdc++ parallel mode, OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PAR) or os.path.getmtime(_LIB_PAR) < os.path.getmtime(_SRC_PAR):
        tmp = _LIB_PAR + ".tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", _SRC_PAR, "-o", tmp])
        os.replace(tmp, _LIB_PAR)
    return _LIB_PAR


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, vp, i32 = ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
            for name in ("ss_oracle_stable_sort", "ss_oracle_group_by"):
                f = getattr(lib, name)
                f.argtypes = [i32, i32, u64, vp, vp, vp, vp]
                f.restype = i32
            for name in ("ss_oracle_collect_reduce_sorted", "ss_oracle_collect_reduce_hash",
                         "ss_oracle_histogram_sorted", "ss_oracle_histogram_hash"):
                f = getattr(lib, name)
                f.argtypes = [i32, u64, vp, vp, vp, vp] if "collect" in name else [i32, u64, vp, vp, vp]
                f.restype = u64
            for name in ("ss_oracle_count_runs", "ss_oracle_count_distinct"):
                f = getattr(lib, name)
                f.argtypes = [i32, u64, vp]
                f.restype = u64
            lib.ss_oracle_mix64.argtypes = [u64]
            lib.ss_oracle_mix64.restype = u64
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _key_code(keys: np.ndarray) -> int:
    """uint32 -> 0, uint64 -> 1, 128-bit keys (shape (n, 2) uint64: lo, hi) -> 2."""
    if keys.ndim == 2:
        assert keys.dtype == np.uint64 and keys.shape[1] == 2
        return 2
    return KT[keys.dtype]


def _c(a):
    return None if a is None else np.ascontiguousarray(a)


def stable_sort(keys, vals=None):
    """Records stably sorted by key: the definition of semisort_<."""
    keys, vals = _c(keys), _c(vals)
    n = keys.shape[0]
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(vals)
    vt = 1 if vals is None else VT[vals.dtype]
    rc = _load().ss_oracle_stable_sort(_key_code(keys), vt, n, _ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo))
    assert rc == 0
    return ko, vo


def stable_sort_parallel(keys, vals=None, threads: int = 0):
    """The same stable sort on `threads` host threads (0 = all) with
    libstdc++'s parallel-mode stable_sort; u32/u64 keys and values.  Returns
    (keys, vals, threads used)."""
    global _lib_par
    with _lock:
        if _lib_par is None:
            lib = ctypes.CDLL(build_parallel())
            f = lib.ss_oracle_stable_sort_parallel
            f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64] + [ctypes.c_void_p] * 4 + [ctypes.c_int]
            f.restype = ctypes.c_int
            _lib_par = lib
    keys, vals = _c(keys), _c(vals)
    n = keys.shape[0]
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(vals)
    vt = 1 if vals is None else VT[vals.dtype]
    used = _lib_par.ss_oracle_stable_sort_parallel(KT[keys.dtype], vt, n, _ptr(keys), _ptr(vals), _ptr(ko),
                                                    _ptr(vo), int(threads))
    assert used > 0
    return ko, vo, used


def group_by(keys, vals=None):
    """semisort_= by first-occurrence hash grouping, stable within groups."""
    keys, vals = _c(keys), _c(vals)
    n = keys.shape[0]
    ko = np.empty_like(keys)
    vo = None if vals is None else np.empty_like(vals)
    vt = 1 if vals is None else VT[vals.dtype]
    rc = _load().ss_oracle_group_by(_key_code(keys), vt, n, _ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo))
    assert rc == 0
    return ko, vo


def _reduce(fn, keys, vals):
    keys = _c(keys)
    n = keys.shape[0]
    uk = np.empty_like(keys)
    if vals is not None:
        vals = _c(vals).astype(np.uint64, copy=False)
        out = np.empty(n, np.uint64)
        u = fn(_key_code(keys), n, _ptr(keys), _ptr(vals), _ptr(uk), _ptr(out))
    else:
        out = np.empty(n, np.uint32)
        u = fn(_key_code(keys), n, _ptr(keys), _ptr(uk), _ptr(out))
    return uk[:u].copy(), out[:u].copy()


def collect_reduce_sorted(keys, vals):
    """(unique keys ascending, u64 wraparound sums)."""
    return _reduce(_load().ss_oracle_collect_reduce_sorted, keys, vals)


def collect_reduce_hash(keys, vals):
    """(unique keys in first-occurrence order, u64 wraparound sums)."""
    return _reduce(_load().ss_oracle_collect_reduce_hash, keys, vals)


def histogram_sorted(keys):
    """(unique keys ascending, u32 counts)."""
    return _reduce(_load().ss_oracle_histogram_sorted, keys, None)


def histogram_hash(keys):
    """(unique keys in first-occurrence order, u32 counts)."""
    return _reduce(_load().ss_oracle_histogram_hash, keys, None)


def collect_reduce_fold(keys, vals, op, identity):
    """collect-reduce with a general monoid (op, identity) (Sec. 2.1): for
    every distinct key, in first-occurrence order, op folded left to right
    over the key's values in input order -- the order a stable grouping keeps
    (Sec. 3.5), so op need not be commutative.  keys: as for group_by; vals:
    a sequence of Python values; op: a Python function.  Returns (unique
    keys, list of folded values).  Plain Python over the records: small n."""
    keys = _c(keys)
    n = keys.shape[0]
    gk, gi = group_by(keys, np.arange(n, dtype=np.uint64))
    flat = gk.reshape(n, -1)
    uk, out = [], []
    i = 0
    while i < n:
        j = i
        acc = identity
        while j < n and np.array_equal(flat[j], flat[i]):
            acc = op(acc, vals[int(gi[j])])
            j += 1
        uk.append(gk[i])
        out.append(acc)
        i = j
    return (np.array(uk, dtype=keys.dtype).reshape((-1,) + keys.shape[1:]) if uk else keys[:0].copy()), out


def count_runs(keys) -> int:
    keys = _c(keys)
    return int(_load().ss_oracle_count_runs(_key_code(keys), keys.shape[0], _ptr(keys)))


def count_distinct(keys) -> int:
    keys = _c(keys)
    return int(_load().ss_oracle_count_distinct(_key_code(keys), keys.shape[0], _ptr(keys)))


def mix64(x: int) -> int:
    """SplitMix64's output mixer (the library's fixed key hash for 64-bit keys)."""
    return int(_load().ss_oracle_mix64(int(x) & 0xFFFFFFFFFFFFFFFF))


def check_semisort_equal(in_keys, in_vals, out_keys, out_vals) -> str | None:
    """Accept a semisort_= output iff (i) its number of maximal equal-key runs
    equals the number of distinct input keys and (ii) its stable sort by key is
    bit-identical to the stable sort of the input.  Together these prove the
    output is a permutation, each key is one contiguous run, and each run keeps
    input order (stability, Sec. 2.2).  Returns None when accepted, else a reason.
    """
    if out_keys.shape != in_keys.shape:
        return "shape mismatch"
    d = count_distinct(in_keys)
    r = count_runs(out_keys)
    if r != d:
        return f"runs {r} != distinct keys {d}"
    ck, cv = stable_sort(in_keys, in_vals)
    ok, ov = stable_sort(out_keys, out_vals)
    if not np.array_equal(ck, ok):
        return "key multiset differs"
    if in_vals is not None and not np.array_equal(cv, ov):
        bad = int(np.flatnonzero(cv != ov)[0])
        return f"value order differs at canonical position {bad}"
    return None


def check_sorted_equal(in_keys, in_vals, out_keys, out_vals) -> str | None:
    """Accept a semisort_< output iff it equals the stable sort of the input."""
    ck, cv = stable_sort(in_keys, in_vals)
    if not np.array_equal(ck, out_keys):
        bad = int(np.flatnonzero(np.any((ck != out_keys).reshape(len(ck), -1), axis=1))[0])
        return f"keys differ at {bad}"
    if in_vals is not None and not np.array_equal(cv, out_vals):
        bad = int(np.flatnonzero(cv != out_vals)[0])
        return f"values differ at {bad}"
    return None
