"""Pins for the CPU oracle: brute force, closed forms, invariants, library
special cases and published test vectors.  CPU only.

Each pin is chosen so that a plausible slip in the oracle (a dropped record, an
unstable tie, a wrong index, keys and values swapped, a sum that is not taken
mod 2^64) fails at least one test.  Mistakes are planted in oracle outputs on
the CPU to show the acceptance checks reject them.
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1


def _keys(rng, n, distinct, kind):
    base = rng.integers(0, distinct, size=n, dtype=np.uint64)
    if kind == "u32":
        return (base * np.uint64(2654435761) % np.uint64(1 << 32)).astype(np.uint32)
    if kind == "u64":
        with np.errstate(over="ignore"):
            return base * np.uint64(0x9E3779B97F4A7C15)
    # 128-bit keys: (lo, hi) where hi carries most of the identity so that the
    # 128-bit order differs from the order of lo alone.
    hi = base * np.uint64(7919)
    lo = (base % np.uint64(3)).astype(np.uint64)
    return np.stack([lo, hi], axis=1)


def _as_tuples(keys):
    if keys.ndim == 2:
        return [(int(r[1]), int(r[0])) for r in keys]  # (hi, lo) orders as u128
    return [int(k) for k in keys]


def brute_stable_sort(keys, vals):
    """Position of record i = #{j : k_j < k_i} + #{j < i : k_j = k_i}."""
    kt = _as_tuples(keys)
    n = len(kt)
    out_pos = [0] * n
    for i in range(n):
        out_pos[i] = sum(1 for j in range(n) if kt[j] < kt[i]) + sum(1 for j in range(i) if kt[j] == kt[i])
    ko = np.empty_like(keys)
    vo = np.empty_like(vals)
    for i in range(n):
        ko[out_pos[i]] = keys[i]
        vo[out_pos[i]] = vals[i]
    return ko, vo


def brute_group_by(keys, vals):
    """Groups ordered by first occurrence, input order inside each group."""
    kt = _as_tuples(keys)
    n = len(kt)
    first = {}
    for i, k in enumerate(kt):
        first.setdefault(k, i)
    pos = []
    for i in range(n):
        before = sum(1 for j in range(n) if first[kt[j]] < first[kt[i]])
        pos.append(before + sum(1 for j in range(i) if kt[j] == kt[i]))
    ko = np.empty_like(keys)
    vo = np.empty_like(vals)
    for i in range(n):
        ko[pos[i]] = keys[i]
        vo[pos[i]] = vals[i]
    return ko, vo


@pytest.mark.parametrize("kind", ["u32", "u64", "u128"])
@pytest.mark.parametrize("distinct", [1, 7, 300])
def test_stable_sort_matches_brute_force(kind, distinct):
    rng = np.random.default_rng(distinct + len(kind))
    n = 400
    keys = _keys(rng, n, distinct, kind)
    vals = np.arange(n, dtype=np.uint64)[::-1].copy()
    ko, vo = oracle.stable_sort(keys, vals)
    bk, bv = brute_stable_sort(keys, vals)
    assert np.array_equal(ko, bk)
    assert np.array_equal(vo, bv)


@pytest.mark.parametrize("kind", ["u32", "u64", "u128"])
@pytest.mark.parametrize("distinct", [1, 7, 300])
def test_group_by_matches_brute_force(kind, distinct):
    rng = np.random.default_rng(100 + distinct)
    n = 400
    keys = _keys(rng, n, distinct, kind)
    vals = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
    ko, vo = oracle.group_by(keys, vals)
    bk, bv = brute_group_by(keys, vals)
    assert np.array_equal(ko, bk)
    assert np.array_equal(vo, bv)


def test_stable_sort_equals_library_stable_argsort():
    """Special case that reduces to a library routine: numpy's stable argsort."""
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 1000, size=200_000, dtype=np.uint64)
    vals = np.arange(keys.size, dtype=np.uint64)
    ko, vo = oracle.stable_sort(keys, vals)
    p = np.argsort(keys, kind="stable")
    assert np.array_equal(ko, keys[p])
    assert np.array_equal(vo, vals[p])


@pytest.mark.parametrize("kind", ["u32", "u64", "u128"])
def test_collect_reduce_and_histogram_brute_force(kind):
    rng = np.random.default_rng(11)
    n = 3000
    keys = _keys(rng, n, 50, kind)
    # values near 2^64 so that every sum wraps: a sum not taken mod 2^64 fails
    vals = (np.uint64(M64) - rng.integers(0, 1000, size=n, dtype=np.uint64))
    kt = _as_tuples(keys)
    want = {}
    cnt = {}
    first = {}
    for i, k in enumerate(kt):
        want[k] = (want.get(k, 0) + int(vals[i])) & M64
        cnt[k] = cnt.get(k, 0) + 1
        first.setdefault(k, i)
    order_sorted = sorted(want)
    order_first = sorted(want, key=lambda k: first[k])

    uk, s = oracle.collect_reduce_sorted(keys, vals)
    assert _as_tuples(uk) == order_sorted
    assert [int(x) for x in s] == [want[k] for k in order_sorted]
    uk, s = oracle.collect_reduce_hash(keys, vals)
    assert _as_tuples(uk) == order_first
    assert [int(x) for x in s] == [want[k] for k in order_first]
    uk, c = oracle.histogram_sorted(keys)
    assert _as_tuples(uk) == order_sorted and c.dtype == np.uint32
    assert [int(x) for x in c] == [cnt[k] for k in order_sorted]
    uk, c = oracle.histogram_hash(keys)
    assert _as_tuples(uk) == order_first
    assert [int(x) for x in c] == [cnt[k] for k in order_first]


def test_sort_and_hash_paths_agree_large():
    """The two independent oracle paths agree on a 2^20-record Zipf input."""
    keys = synth.zipf(7, 1 << 20, 1.2, N=10**6)
    vals = np.arange(keys.size, dtype=np.uint64)
    a_k, a_s = oracle.collect_reduce_sorted(keys, vals)
    b_k, b_s = oracle.collect_reduce_hash(keys, vals)
    p = np.argsort(b_k, kind="stable")
    assert np.array_equal(a_k, b_k[p]) and np.array_equal(a_s, b_s[p])
    gk, gv = oracle.group_by(keys, vals)
    assert oracle.check_semisort_equal(keys, vals, gk, gv) is None


def test_closed_forms_value_is_index():
    """value = index: all sums add to n(n-1)/2 mod 2^64; counts add to n."""
    n = 1 << 18
    keys = synth.uniform_mod(3, n, 10_000)
    vals = np.arange(n, dtype=np.uint64)
    _, s = oracle.collect_reduce_sorted(keys, vals)
    assert int(np.sum(s, dtype=np.uint64)) == (n * (n - 1) // 2) & M64
    _, c = oracle.histogram_sorted(keys)
    assert int(c.sum()) == n


@pytest.mark.parametrize("mu", [1, 10, 1000, 3200])
def test_closed_form_exact_multiplicity(mu):
    """uniform_exact with mu | n: every count is exactly n/mu (Table 2's
    uniform rows print max frequency n/mu and mu distinct keys)."""
    n = 64_000
    keys = synth.uniform_exact(9, n, mu)
    uk, c = oracle.histogram_hash(keys)
    assert uk.size == mu
    assert np.all(c == n // mu)


def test_special_cases():
    n = 1000
    vals = np.arange(n, dtype=np.uint64)
    # all keys equal: every semisort output equals the input
    keys = np.full(n, 42, np.uint64)
    for f in (oracle.stable_sort, oracle.group_by):
        ko, vo = f(keys, vals)
        assert np.array_equal(ko, keys) and np.array_equal(vo, vals)
    # all keys distinct: group_by is the identity
    keys = synth.splitmix64_outputs(1, n)
    ko, vo = oracle.group_by(keys, vals)
    assert np.array_equal(ko, keys) and np.array_equal(vo, vals)
    # empty input
    e = np.empty(0, np.uint64)
    assert oracle.stable_sort(e, e)[0].size == 0
    assert oracle.collect_reduce_sorted(e, e)[0].size == 0
    assert oracle.count_runs(e) == 0 and oracle.count_distinct(e) == 0


def test_checker_accepts_every_valid_grouping():
    rng = np.random.default_rng(2)
    n = 5000
    keys = rng.integers(0, 300, size=n, dtype=np.uint64)
    vals = np.arange(n, dtype=np.uint64)
    for f in (oracle.stable_sort, oracle.group_by):
        ko, vo = f(keys, vals)
        assert oracle.check_semisort_equal(keys, vals, ko, vo) is None
    # an arbitrary permutation of whole groups is still a valid semisort_=
    ko, vo = oracle.stable_sort(keys, vals)
    starts = np.flatnonzero(np.r_[True, ko[1:] != ko[:-1]])
    bounds = list(zip(starts, np.r_[starts[1:], n]))
    rng.shuffle(bounds)
    pk = np.concatenate([ko[a:b] for a, b in bounds])
    pv = np.concatenate([vo[a:b] for a, b in bounds])
    assert oracle.check_semisort_equal(keys, vals, pk, pv) is None


def test_checker_rejects_planted_mistakes():
    """Mistakes planted in an oracle output on the CPU must be rejected."""
    rng = np.random.default_rng(3)
    n = 4000
    keys = rng.integers(0, 100, size=n, dtype=np.uint64)
    vals = np.arange(n, dtype=np.uint64)
    ko, vo = oracle.group_by(keys, vals)
    # unstable: swap two values inside one group
    g = np.flatnonzero(ko == ko[0])
    bad_v = vo.copy()
    bad_v[g[0]], bad_v[g[1]] = bad_v[g[1]], bad_v[g[0]]
    assert oracle.check_semisort_equal(keys, vals, ko, bad_v) is not None
    # a split group: move the last record of the first group to the end
    idx = np.r_[np.arange(g[-1]), np.arange(g[-1] + 1, n), g[-1]]
    assert oracle.check_semisort_equal(keys, vals, ko[idx], vo[idx]) is not None
    # a duplicated record in place of another one
    dk, dv = ko.copy(), vo.copy()
    dk[-1], dv[-1] = dk[-2], dv[-2]
    assert oracle.check_semisort_equal(keys, vals, dk, dv) is not None
    # keys and values exchanged
    assert oracle.check_semisort_equal(keys, vals, vo, ko) is not None
    # semisort_< acceptance rejects a valid grouping that is not key ordered
    sk, sv = oracle.stable_sort(keys, vals)
    assert oracle.check_sorted_equal(keys, vals, sk, sv) is None
    if not np.array_equal(ko, sk):
        assert oracle.check_sorted_equal(keys, vals, ko, vo) is not None


def test_mix64_published_vectors_and_bijectivity():
    """The oracle's mix64 reproduces SplitMix64's published outputs and is a
    bijection (checked with its inverse, derived independently here)."""
    lines = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
             if l.strip() and not l.startswith("#")]
    seed = int(lines[0][1])
    want = [int(l[0]) for l in lines[1:]]
    got = [oracle.mix64(seed + (i + 1) * 0x9E3779B97F4A7C15) for i in range(len(want))]
    assert got == want

    def unxorshift(y, s):
        x = y
        for _ in range(64 // s + 1):
            x = y ^ (x >> s)
        return x

    inv1 = pow(0xBF58476D1CE4E5B9, -1, 1 << 64)
    inv2 = pow(0x94D049BB133111EB, -1, 1 << 64)
    rng = np.random.default_rng(0)
    for x in [0, 1, M64, *map(int, rng.integers(0, 1 << 63, size=200, dtype=np.uint64))]:
        z = oracle.mix64(x)
        z = unxorshift(z, 31)
        z = (z * inv2) & M64
        z = unxorshift(z, 27)
        z = (z * inv1) & M64
        z = unxorshift(z, 30)
        assert z == x


@pytest.mark.parametrize("kt,vt,threads", [(np.uint64, np.uint64, 0), (np.uint32, np.uint64, 3),
                                           (np.uint64, np.uint32, 2), (np.uint32, np.uint32, 0)])
def test_parallel_stable_sort_equals_serial_and_numpy(kt, vt, threads):
    """The all-core oracle sort (the CPU baseline's) gives exactly the
    serial oracle's output, and numpy's stable argsort agrees with both."""
    rng = np.random.default_rng(77)
    n = 300_007
    keys = rng.integers(0, 5000, size=n).astype(kt)
    vals = rng.integers(0, 2**31, size=n).astype(vt)
    pk, pv, used = oracle.stable_sort_parallel(keys, vals, threads)
    assert used >= 1 and (threads == 0 or used == threads)
    sk, sv = oracle.stable_sort(keys, vals)
    assert np.array_equal(pk, sk) and np.array_equal(pv, sv)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(pk, keys[order]) and np.array_equal(pv, vals[order])


def test_collect_reduce_fold_pins():
    """The general-monoid oracle: with (+ mod 2^64, 0) it equals the hash
    collect-reduce; with a non-commutative op (tuple concatenation) every
    key's fold is its values in input order, checked by brute force."""
    rng = np.random.default_rng(33)
    keys = rng.integers(0, 50, size=3000).astype(np.uint64)
    vals = [int(x) for x in rng.integers(0, 2**63, size=3000)]
    uk, out = oracle.collect_reduce_fold(keys, vals, lambda a, b: (a + b) % 2**64, 0)
    hk, hs = oracle.collect_reduce_hash(keys, np.array(vals, dtype=np.uint64))
    assert np.array_equal(uk, hk) and [int(x) for x in hs] == out
    uk, out = oracle.collect_reduce_fold(keys, list(range(3000)), lambda a, b: a + (b,), ())
    first = {}
    for i, k in enumerate(keys.tolist()):
        first.setdefault(k, []).append(i)
    assert [int(k) for k in uk] == list(first.keys())
    assert out == [tuple(v) for v in first.values()]
    k2 = np.stack([keys, keys * 3], axis=1).astype(np.uint64)  # 128-bit keys
    uk2, out2 = oracle.collect_reduce_fold(k2, list(range(3000)), lambda a, b: a + (b,), ())
    assert np.array_equal(uk2[:, 0], uk) and out2 == out
