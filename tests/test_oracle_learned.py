"""Pins of the learned-splitter oracle (oracle/learned.py) against things
that do not depend on it: central finite differences, a one-unit special
case with a closed form, monotonicity, Adam's first step, and brute-force
inversion."""
import numpy as np
import pytest

from oracle import learned as L


def rand_params(seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 1.0, L.N_PARAMS)


def test_layout():
    assert L.N_PARAMS == 1153
    covered = sorted(L.SLICES.values())
    assert covered[0][0] == 0 and covered[-1][1] == L.N_PARAMS
    for (a, b), (c, d) in zip(covered, covered[1:]):
        assert b == c


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_central_differences(seed):
    p = rand_params(seed)
    rng = np.random.default_rng(100 + seed)
    x = rng.random(37)
    t = np.sort(rng.random(37))
    _, g = L.loss_grad(p, x, t)
    h = 1e-6
    idx = np.concatenate([np.arange(0, L.N_PARAMS, 7), [L.N_PARAMS - 1]])
    for i in idx:
        e = np.zeros(L.N_PARAMS)
        e[i] = h
        num = (L.loss(p + e, x, t) - L.loss(p - e, x, t)) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num)), (i, num, g[i])


def test_single_path_closed_form():
    """Only h1_0 -> h2_0 -> y carries weight: f(x) = s3 * sig(s2 * sig(s1 x + c1) + c2) + c3."""
    p = np.zeros(L.N_PARAMS)
    q = L.unpack(p)  # views into p
    q["v1"][:] = -50.0
    q["v2"][:] = -50.0
    q["v3"][:] = -50.0
    q["v1"][0], q["c1"][0], q["v2"][0, 0], q["c2"][0], q["v3"][0], q["c3"][0] = 1.3, -0.4, 0.7, 0.2, 2.0, -1.0
    p = np.concatenate([q["v1"], q["c1"], q["v2"].ravel(), q["c2"], q["v3"], q["c3"]])
    x = np.linspace(0, 1, 11)
    sp = lambda v: np.log(1 + np.exp(v))
    sg = lambda z: 1 / (1 + np.exp(-z))
    h2_rest = sg(0.0 + 31 * sp(-50.0) * 0.5)  # negligible cross terms
    want = sp(2.0) * sg(sp(0.7) * sg(sp(1.3) * x - 0.4) + 0.2) - 1.0
    got = L.forward(p, x)[0]
    assert np.allclose(got, want, atol=1e-12 + 31 * sp(-50.0) * 2)
    assert h2_rest > 0


@pytest.mark.parametrize("seed", [3, 4])
def test_monotone(seed):
    p = rand_params(seed)
    x = np.linspace(0, 1, 2001)
    y = L.forward(p, x)[0]
    assert np.all(np.diff(y) >= -1e-12)


def test_adam_first_step_moves_each_parameter_by_lr():
    """With zero moments, Adam's bias-corrected first step is lr * g / (|g| + eps)."""
    p = np.zeros(5)
    g = np.array([0.5, -2.0, 1e-3, 0.0, 3.0])
    p1, m, v = L.adam(p, g, np.zeros(5), np.zeros(5), 1, 0.01)
    want = -0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(p1, want, rtol=1e-9, atol=1e-15)


def test_training_reduces_loss_on_a_linear_cdf():
    rng = np.random.default_rng(7)
    x = np.sort(rng.random(256))
    t = (np.arange(256) + 0.5) / 256
    p0 = rand_params(8) * 0.1
    l0 = L.loss(p0, x, t)
    p1, l1 = L.train(p0, x, t, steps=200, lr=0.01)
    assert l1 < 0.05 * l0


def test_invert_matches_brute_force():
    p = rand_params(9)
    kmin, kmax, nl = 1000, 1400, 16
    y_all = L.forward(p, (np.arange(kmin, kmax + 1) - kmin) / (kmax - kmin))[0]
    got = L.invert(p, kmin, kmax, nl)
    for j in range(1, nl):
        hits = np.nonzero(y_all >= j / nl)[0]
        brute = kmin + (hits[0] if hits.size else kmax - kmin)
        assert got[j - 1] >= brute  # made non-decreasing: never below the first crossing
    assert np.all(np.diff(got.astype(np.int64)) >= 0)
    first = []
    for j in range(1, nl):
        hits = np.nonzero(y_all >= j / nl)[0]
        first.append(kmin + (hits[0] if hits.size else kmax - kmin))
    assert np.array_equal(got, np.maximum.accumulate(np.array(first, dtype=np.uint64)))
