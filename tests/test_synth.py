"""CPU checks of the seeded input generators against the workload statistics
the paper prints (Table 2) and against closed forms."""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
N_PAPER = 10**9
HEAVY_CUT = 500 * math.log(N_PAPER)  # "more than 500 log n" occurrences, natural log


def _parse(v: str) -> float:
    mult = {"K": 1e3, "M": 1e6, "B": 1e9}
    return float(v[:-1]) * mult[v[-1]] if v[-1] in mult else float(v)


def table2():
    rows = []
    for line in open(os.path.join(GOLDEN, "table2_workload_stats.txt")):
        if line.strip() and not line.startswith("#"):
            d, p, dist, mx, hv = line.split()
            rows.append((d, float(p), _parse(dist), _parse(mx), float(hv)))
    return rows


def _zipf_H(s, lo, hi):
    """sum_{r=lo}^{hi} r^-s, exact head plus Euler-Maclaurin tail."""
    m = min(hi, lo + 2_000_000)
    head = float(np.sum(np.arange(lo, m + 1, dtype=np.float64) ** (-s)))
    if hi <= m:
        return head
    a, b = m + 0.5, hi + 0.5
    return head + (math.log(b / a) if s == 1 else (b ** (1 - s) - a ** (1 - s)) / (1 - s))


@pytest.mark.parametrize("row", [r for r in table2() if r[0] == "zipf"], ids=lambda r: f"s={r[1]}")
def test_zipf_closed_form_matches_table2(row):
    """Zipf over N = 10^9 ranks: max frequency n/H_{N,s} and the heavy share
    (records of ranks whose expected count exceeds 500 ln n) match Table 2.
    This pins the Zipf reading and the natural log in the heavy threshold."""
    _, s, _, maxfreq, heavy = row
    H = _zipf_H(s, 1, N_PAPER)
    assert abs(N_PAPER / H - maxfreq) / maxfreq < 0.01
    r_star = int((N_PAPER / (H * HEAVY_CUT)) ** (1 / s))
    share = 100 * _zipf_H(s, 1, r_star) / H
    assert abs(share - heavy) <= max(0.05 * heavy, 0.05)


@pytest.mark.parametrize("row", [r for r in table2() if r[0] == "exponential"], ids=lambda r: f"l={r[1]}")
def test_exponential_closed_form_matches_table2(row):
    """floor(Exp(lambda)): max frequency n(1-e^-lambda) and heavy share
    1 - 500 ln(n) / (n lambda) match Table 2 (distinct counts are not pinned)."""
    _, lam, _, maxfreq, heavy = row
    assert abs(N_PAPER * (1 - math.exp(-lam)) - maxfreq) / maxfreq < 0.01
    share = max(0.0, 100 * (1 - HEAVY_CUT / (N_PAPER * lam)))
    assert abs(share - heavy) < 0.5


@pytest.mark.parametrize("s", [0.6, 1.0, 1.5])
def test_zipf_sampler_empirical(s):
    """Empirical rank frequencies of the rejection-inversion sampler follow
    r^-s / H_{N,s} for the top ranks (n = 2^20, N = 10^6)."""
    n, N = 1 << 20, 10**6
    r = synth.zipf_ranks(5, n, s, N)
    assert r.min() >= 1 and r.max() <= N
    H = _zipf_H(s, 1, N)
    cnt = np.bincount(r.astype(np.int64), minlength=6)
    for k in (1, 2, 5):
        p = k ** (-s) / H
        sd = math.sqrt(n * p * (1 - p))
        assert abs(cnt[k] - n * p) < 5 * sd + 1


def test_feistel_is_a_bijection():
    for n in (1, 2, 1000, 1 << 16, 999_983):
        p = synth.feistel_permute(4, n, np.arange(n, dtype=np.uint64))
        assert np.array_equal(np.sort(p), np.arange(n, dtype=np.uint64))


def test_uniform_mod_is_config1_definition():
    """key_i = splitmix64(seed, i) mod 10^4; checked against the published
    generator outputs (golden) for the first indices."""
    lines = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
             if l.strip() and not l.startswith("#")]
    seed = int(lines[0][1])
    want = np.array([int(l[0]) for l in lines[1:]], dtype=np.uint64)
    assert np.array_equal(synth.splitmix64_outputs(seed, 5), want)
    assert np.array_equal(synth.uniform_mod(seed, 5, 10**4), want % np.uint64(10**4))
    k = synth.uniform_mod(0x5EED0001, 1 << 20, 10**4)
    assert oracle.count_distinct(k) == 10**4


def test_generators_are_chunkable():
    """Generating [start, start+count) equals slicing the whole array, so big
    inputs can be produced piecewise."""
    n = 10_000
    for f in (lambda st, c: synth.uniform_exact(1, n, 77, st, c),
              lambda st, c: synth.zipf(1, c, 1.2, 10**6, st),
              lambda st, c: synth.exponential(1, c, 1e-3, st),
              lambda st, c: synth.gaussian_mixture(1, c, 8, st)):
        whole = f(0, n)
        part = f(3000, 2000)
        assert np.array_equal(whole[3000:5000], part)


def test_rmat_quadrant_shares():
    src, dst = synth.rmat_edges(3, 1 << 18, 10)
    assert src.max() < 1024 and dst.max() < 1024
    # top bit of src is 1 with probability c + d = 0.24; of dst with b + d = 0.24
    assert abs((src >> 9).mean() - 0.24) < 0.01
    assert abs((dst >> 9).mean() - 0.24) < 0.01


def test_gaussian_mixture_range():
    k = synth.gaussian_mixture(8, 1 << 16)
    means, sigmas, w = synth.gaussian_mixture_params(8)
    assert abs(w.sum() - 1) < 1e-12 and np.all(sigmas >= 2.0**34)
    assert k.min() > 0 and k.max() < np.uint64(1 << 63)
