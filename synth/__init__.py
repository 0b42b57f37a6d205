"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 5, Table 2).

This module holds only input generation: no step of the semisort method is
computed here.  Both the CUDA path (through the GPU twins in ``synth.cu``) and
the CPU oracle consume what it produces.  All randomness is counter based, so
every record is a pure function of (seed, stream, record index, attempt).

Generators
----------
* ``uniform_mod``   -- key_i = SplitMix64 output i (seeded) mod mu (i.i.d.).
* ``uniform_exact`` -- exactly mu distinct keys, each n/mu times: key_i =
                       H(pi(i) mod mu), pi a seeded Feistel permutation of
                       [0, n) (cycle walking), H a seeded bijective mixer.
                       Table 2 prints mu distinct keys with max frequency n/mu,
                       which this reproduces exactly.
* ``zipf``          -- ranks in [1, N] with P(r) ~ r^-s drawn by the
                       rejection-inversion method of Hormann and Derflinger
                       (ACM TOMACS 1996), key = H(rank).
* ``exponential``   -- key = floor(Exp(lambda)).
* ``gaussian_mixture`` -- 8 seeded components, quantized to uint64.
* ``rmat``          -- R-MAT edges (Chakrabarti, Zhan, Faloutsos 2004).
"""
from __future__ import annotations

import math

import numpy as np

M64 = 0xFFFFFFFFFFFFFFFF
GOLDEN = 0x9E3779B97F4A7C15
STREAM_MUL = 0xD1B54A32D192ED03


def _u64(x) -> np.ndarray:
    return np.asarray(x, dtype=np.uint64)


def mix64_np(z: np.ndarray) -> np.ndarray:
    """SplitMix64's output mixer on a uint64 array (wraps mod 2^64)."""
    z = _u64(z)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def mix64_int(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def stream_base(seed: int, stream: int) -> int:
    """Start state of an independent counter stream."""
    return mix64_int((seed ^ ((stream * STREAM_MUL) & M64)) & M64)


def rand64(seed: int, stream: int, ctr: np.ndarray) -> np.ndarray:
    """Counter-based 64-bit random words: mix64(base + (ctr+1) * golden)."""
    base = np.uint64(stream_base(seed, stream))
    with np.errstate(over="ignore"):
        return mix64_np(base + (_u64(ctr) + np.uint64(1)) * np.uint64(GOLDEN))


def unit(x: np.ndarray) -> np.ndarray:
    """Top 53 bits of a random word as a double in [0, 1)."""
    return (_u64(x) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def splitmix64_outputs(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs start..start+n-1 of a SplitMix64 generator seeded with `seed`."""
    i = np.arange(start, start + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64_np(np.uint64(seed & M64) + (i + np.uint64(1)) * np.uint64(GOLDEN))


def key_of_rank(seed: int, rank: np.ndarray) -> np.ndarray:
    """Seeded bijective map from ranks to spread-out 64-bit keys."""
    c = np.uint64(stream_base(seed, 0x4B4559))
    with np.errstate(over="ignore"):
        return mix64_np(_u64(rank) + c)


def uniform_mod(seed: int, n: int, mu: int, start: int = 0) -> np.ndarray:
    """key_i = splitmix64(seed, i) mod mu (i.i.d. uniform over mu values)."""
    return splitmix64_outputs(seed, n, start) % np.uint64(mu)


def _feistel_params(n: int):
    bits = max(2, int(math.ceil(math.log2(max(n, 2)))))
    if bits % 2:
        bits += 1
    half = bits // 2
    return half, (1 << half) - 1


def feistel_permute(seed: int, n: int, i: np.ndarray) -> np.ndarray:
    """Seeded bijection of [0, n): a 4-round balanced Feistel network on
    [0, 2^(2h)) applied repeatedly (cycle walking) until the value is < n."""
    half, mask = _feistel_params(n)
    rk = [np.uint64(stream_base(seed, 0xFE15 + r)) for r in range(4)]
    m = np.uint64(mask)
    h = np.uint64(half)

    def enc(x):
        left, right = x >> h, x & m
        for r in range(4):
            with np.errstate(over="ignore"):
                f = mix64_np(right ^ rk[r]) & m
            left, right = right, left ^ f
        return (left << h) | right

    y = enc(_u64(i))
    bad = y >= np.uint64(n)
    while bad.any():
        y[bad] = enc(y[bad])
        bad = y >= np.uint64(n)
    return y


def uniform_exact(seed: int, n: int, mu: int, start: int = 0, count: int | None = None) -> np.ndarray:
    """Exactly min(mu, n) distinct keys; key r appears ceil((n - r)/mu) times."""
    count = n - start if count is None else count
    i = np.arange(start, start + count, dtype=np.uint64)
    return key_of_rank(seed, feistel_permute(seed, n, i) % np.uint64(mu))


class _ZipfRI:
    """Rejection-inversion sampler for P(k) ~ k^-s on k = 1..N (Hormann and
    Derflinger 1996): invert the integral H of the hat h(x) = x^-s, then accept
    k = round(x) if x falls under the histogram of h around k.  The helper
    functions log1p(x)/x and expm1(x)/x with their series guards, the
    constants H(1.5) - 1 and 2 - H^-1(H(2.5) - h(2)) and the acceptance test
    follow the shape of the Apache Commons RNG RejectionInversionZipfSampler
    (Apache-2.0), a widely used statement of the same published method."""

    def __init__(self, s: float, N: int):
        self.s, self.N = float(s), int(N)
        self.h_x1 = self.H(1.5) - 1.0
        self.h_n = self.H(self.N + 0.5)
        self.sq = 2.0 - self.Hinv(self.H(2.5) - self.h(2.0))

    @staticmethod
    def _helper1(x):  # log1p(x)/x, continuous at 0
        x = np.asarray(x, dtype=np.float64)
        small = np.abs(x) < 1e-8
        return np.where(small, 1.0 - x * (0.5 - x * (1.0 / 3.0 - 0.25 * x)),
                        np.log1p(np.where(small, 1.0, x)) / np.where(small, 1.0, x))

    @staticmethod
    def _helper2(x):  # expm1(x)/x, continuous at 0
        x = np.asarray(x, dtype=np.float64)
        small = np.abs(x) < 1e-8
        return np.where(small, 1.0 + x * 0.5 * (1.0 + x * (1.0 / 3.0) * (1.0 + 0.25 * x)),
                        np.expm1(np.where(small, 1.0, x)) / np.where(small, 1.0, x))

    def h(self, x):
        return np.exp(-self.s * np.log(x))

    def H(self, x):
        lx = np.log(x)
        return self._helper2((1.0 - self.s) * lx) * lx

    def Hinv(self, x):
        t = np.maximum(x * (1.0 - self.s), -1.0)
        return np.exp(self._helper1(t) * x)

    def sample(self, u: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
        """One attempt per uniform; returns (k, accepted)."""
        v = self.h_n + u * (self.h_x1 - self.h_n)
        x = self.Hinv(v)
        k = np.clip(np.floor(x + 0.5), 1, self.N)
        acc = (k - x <= self.sq) | (v >= self.H(k + 0.5) - self.h(k))
        return k.astype(np.uint64), acc


def zipf_ranks(seed: int, n: int, s: float, N: int = 10**9, start: int = 0) -> np.ndarray:
    z = _ZipfRI(s, N)
    idx = np.arange(start, start + n, dtype=np.uint64)
    out = np.zeros(n, np.uint64)
    todo = np.arange(n)
    attempt = 0
    while todo.size:
        ctr = (idx[todo] << np.uint64(6)) | np.uint64(attempt & 63)
        k, acc = z.sample(unit(rand64(seed, 0x21FF + (attempt >> 6), ctr)))
        out[todo[acc]] = k[acc]
        todo = todo[~acc]
        attempt += 1
    return out


def zipf(seed: int, n: int, s: float, N: int = 10**9, start: int = 0) -> np.ndarray:
    """Zipf(s) over N ranks mapped through a seeded bijection to 64-bit keys."""
    return key_of_rank(seed, zipf_ranks(seed, n, s, N, start))


def exponential(seed: int, n: int, lam: float, start: int = 0) -> np.ndarray:
    """key = floor(Exp(lambda))."""
    u = unit(rand64(seed, 0xE4, np.arange(start, start + n, dtype=np.uint64)))
    return np.floor(-np.log1p(-u) / lam).astype(np.uint64)


def gaussian_mixture_params(seed: int, k: int = 8):
    """Component means uniform in [2^40, 2^62], sigma = 2^34 * U[1, 16],
    weights Dirichlet(1) (normalized Exp(1) draws)."""
    r = unit(rand64(seed, 0x6A, np.arange(3 * k, dtype=np.uint64)))
    means = 2.0 ** 40 + r[:k] * (2.0 ** 62 - 2.0 ** 40)
    sigmas = 2.0 ** 34 * (1.0 + 15.0 * r[k:2 * k])
    w = -np.log1p(-r[2 * k:])
    return means, sigmas, w / w.sum()


def gaussian_mixture(seed: int, n: int, k: int = 8, start: int = 0) -> np.ndarray:
    means, sigmas, w = gaussian_mixture_params(seed, k)
    idx = np.arange(start, start + n, dtype=np.uint64)
    u0 = unit(rand64(seed, 0x6B, idx))
    comp = np.minimum(np.searchsorted(np.cumsum(w), u0, side="right"), k - 1)
    u1 = unit(rand64(seed, 0x6C, idx))
    u2 = unit(rand64(seed, 0x6D, idx))
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)  # Box-Muller
    x = means[comp] + sigmas[comp] * z
    x = np.clip(x, 0.0, 18446744073709549568.0)  # largest double below 2^64
    return np.floor(x).astype(np.uint64)


def rmat_edges(seed: int, m: int, scale: int, abcd=(0.57, 0.19, 0.19, 0.05), start: int = 0):
    """R-MAT: each edge picks a quadrant per level with probabilities a, b, c, d;
    src takes the row bits and dst the column bits (no noise, no relabeling)."""
    a, b, c, _ = abcd
    idx = np.arange(start, start + m, dtype=np.uint64)
    src = np.zeros(m, np.uint64)
    dst = np.zeros(m, np.uint64)
    for lvl in range(scale):
        u = unit(rand64(seed, 0x7000 + lvl, idx))
        row = u >= a + b
        col = ((u >= a) & (u < a + b)) | (u >= a + b + c)
        src = (src << np.uint64(1)) | row.astype(np.uint64)
        dst = (dst << np.uint64(1)) | col.astype(np.uint64)
    return src.astype(np.uint32), dst.astype(np.uint32)


def zipf_max_frequency(n: int, s: float, N: int) -> float:
    """Expected count of rank 1: n / H_{N,s} (Euler-Maclaurin tail for large N)."""
    m = min(N, 10**6)
    head = float(np.sum(np.arange(1, m + 1, dtype=np.float64) ** (-s)))
    if N > m:
        a, b = m + 0.5, N + 0.5
        tail = math.log(b / a) if s == 1.0 else (b ** (1 - s) - a ** (1 - s)) / (1 - s)
    else:
        tail = 0.0
    return n / (head + tail)
