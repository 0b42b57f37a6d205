"""Learned splitters on the GPU: the model's gradient against the fp64 oracle,
training against the oracle's training, inversion against the oracle's
forward pass, exact semisort_< results in learned mode, and what the trained
model gains in top-level load balance over sampled splitters."""
import numpy as np
import pytest

import oracle
import synth
from oracle import learned as OL
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


def fdev(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


@pytest.mark.parametrize("m,seed", [(1024, 0), (37, 1), (4096, 2)])
def test_gradient_matches_oracle(ss, m, seed):
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, 0.5, OL.N_PARAMS).astype(np.float32)
    x = rng.random(m).astype(np.float32)
    t = np.sort(rng.random(m)).astype(np.float32)
    loss, g = ss.mlp_loss_grad(fdev(p), fdev(x), fdev(t))
    g = g.cpu().numpy().astype(np.float64)
    want_loss, want = OL.loss_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert abs(float(loss) - want_loss) <= 1e-4 * want_loss
    rel = np.linalg.norm(g - want) / np.linalg.norm(want)
    assert rel <= 1e-3, rel
    assert np.max(np.abs(g - want)) <= 1e-3 * np.max(np.abs(want))


def test_gradient_deterministic(ss):
    rng = np.random.default_rng(5)
    p, x, t = fdev(rng.normal(0, 0.5, OL.N_PARAMS)), fdev(rng.random(2000)), fdev(np.sort(rng.random(2000)))
    a = ss.mlp_loss_grad(p, x, t)[1].cpu().numpy()
    b = ss.mlp_loss_grad(p, x, t)[1].cpu().numpy()
    assert np.array_equal(a, b)


def test_training_tracks_oracle(ss):
    """200 Adam steps from the same start: the FP32 GPU run and the fp64
    oracle reach losses within a factor of three, both far below the start."""
    rng = np.random.default_rng(6)
    keys = np.sort(rng.beta(2.0, 5.0, 1024))
    x = (keys - keys[0]) / (keys[-1] - keys[0])
    t = (np.arange(1024) + 0.5) / 1024
    p0 = rng.normal(0.0, 0.3, OL.N_PARAMS)
    l0 = OL.loss(p0, x, t)
    _, want = OL.train(p0, x, t, steps=200, lr=0.01)
    p, loss = ss.mlp_train(fdev(x), fdev(t), fdev(p0), 200, 0.01)
    got = float(loss.cpu()[0])
    assert got < 0.05 * l0 and want < 0.05 * l0
    assert got < 3 * want + 1e-7 and want < 3 * got + 1e-7, (got, want)
    assert abs(OL.loss(p.cpu().numpy().astype(np.float64), x, t) - got) <= 1e-3 * got + 1e-8


@pytest.mark.parametrize("steps", [1, 2, 5])
def test_adam_steps_match_oracle(ss, steps):
    """Parameters after 1, 2 and 5 full-batch Adam steps, element by element,
    against the fp64 oracle's Adam from the same start.  Adam normalizes each
    element's step by its own gradient history, so an element's FP32 error
    depends on how well its own gradient is resolved:
    * elements whose gradient stays at least 1e-4 of the largest one at every
      step (the oracle's gradients decide) must agree within 1e-3 lr per step;
    * at least 90% of all elements must agree within 0.1 lr per step, and
      every element within 2.5 lr per step (a sign flip costs 2 lr).
    In step 1 every update is lr g/(|g| + eps), about lr in size whatever the
    gradient's scale, so a wrong bias correction or moment update moves
    nearly every element by a large multiple of lr and fails the 90% bound."""
    rng = np.random.default_rng(11)
    keys = np.sort(rng.beta(2.0, 5.0, 1024))
    x = (keys - keys[0]) / (keys[-1] - keys[0])
    t = (np.arange(1024) + 0.5) / 1024
    p0 = rng.normal(0.0, 0.3, OL.N_PARAMS).astype(np.float32).astype(np.float64)
    x32, t32 = x.astype(np.float32), t.astype(np.float32)
    lr = 0.01
    p = p0.copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    resolved = np.ones(OL.N_PARAMS, dtype=bool)
    for s in range(1, steps + 1):
        _, g = OL.loss_grad(p, x32.astype(np.float64), t32.astype(np.float64))
        resolved &= np.abs(g) >= 1e-4 * np.max(np.abs(g))
        p, m, v = OL.adam(p, g, m, v, s, lr)
    got, _ = ss.mlp_train(fdev(x32), fdev(t32), fdev(p0), steps, lr)
    d = np.abs(got.cpu().numpy().astype(np.float64) - p)
    tol = lr * steps
    assert np.max(d[resolved]) <= 1e-3 * tol, (np.max(d[resolved]) / tol, int(resolved.sum()))
    assert np.mean(d <= 0.1 * tol) >= 0.9, np.mean(d <= 0.1 * tol)
    assert np.max(d) <= 2.5 * tol, np.max(d) / tol


@pytest.mark.parametrize("kt", ["u64", "u32"])
def test_invert_against_oracle_forward(ss, kt):
    rng = np.random.default_rng(7)
    x = np.sort(rng.random(1024))
    t = (np.arange(1024) + 0.5) / 1024
    p, _ = ss.mlp_train(fdev(x), fdev(t), fdev(rng.normal(0, 0.3, OL.N_PARAMS)), 300, 0.01)
    pn = p.cpu().numpy().astype(np.float64)
    kmin, kmax = (10**12, 10**12 + 10**9) if kt == "u64" else (1000, 4_000_000_000)
    lb = 8
    spl = to_host(ss.mlp_invert(p, ss.SS_U64 if kt == "u64" else ss.SS_U32, kmin, kmax, lb)).astype(np.int64)
    nl = 1 << lb
    span = kmax - kmin
    f = lambda k: OL.forward(pn, (np.asarray(k, dtype=np.float64) - kmin) / span)[0]
    assert np.all(spl >= kmin) and np.all(spl <= kmax)
    tol = 2e-5  # the GPU evaluates the model in FP32
    for j in range(1, nl):
        s = spl[j - 1]
        tau = j / nl
        if s < kmax:
            assert f(s) >= tau - tol, (j, f(s), tau)
        if s > kmin:
            assert f(s - 1) < tau + tol, (j, f(s - 1), tau)


def run_less(ss, keys_h, vals_h, mode):
    import torch
    keys, vals = to_dev(keys_h), to_dev(vals_h)
    o = ss.make_options(seed=1, splitter_mode=mode)
    ws = ss.alloc_workspace(ss.OP_LESS, keys, vals, o)
    ko, vo = ss.semisort_less(keys, vals, workspace=ws, options=o)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    return to_host(ko), to_host(vo), ss.stats(ws)


@pytest.mark.parametrize("kind", ["uniform", "zipf12", "exponential", "gaussian_mixture"])
def test_learned_mode_results_exact(ss, kind):
    n = 1 << 22
    keys = {"uniform": lambda: synth.uniform_exact(81, n, n),
            "zipf12": lambda: synth.zipf(82, n, 1.2),
            "exponential": lambda: synth.exponential(83, n, 1e-6),
            "gaussian_mixture": lambda: synth.gaussian_mixture(84, n)}[kind]()
    vals = np.arange(n, dtype=np.uint64)
    ko, vo, st = run_less(ss, keys, vals, 1)
    err = oracle.check_sorted_equal(keys, vals, ko, vo)
    assert err is None, err
    assert st["l0_splitters"] in (1, 2)


def test_learned_gain_in_top_level_balance(ss):
    """Hashed (near-uniform) keys: the smooth CDF fit splits the top level more
    evenly than the quantiles of the same 2^16-key sample."""
    n = 1 << 24
    keys = synth.uniform_exact(85, n, n)
    vals = np.arange(n, dtype=np.uint64)
    _, _, st_s = run_less(ss, keys, vals, 0)
    _, _, st_l = run_less(ss, keys, vals, 1)
    assert st_s["l0_splitters"] == 0 and st_l["l0_splitters"] == 1
    mean = n / st_s["l0_light_buckets"]
    ratio_s, ratio_l = st_s["l0_max_light_bucket"] / mean, st_l["l0_max_light_bucket"] / mean
    assert ratio_l < ratio_s, (ratio_l, ratio_s)


@pytest.mark.parametrize("kind", ["uniform", "zipf12", "exponential", "gaussian_mixture"])
def test_learned_judged_against_sampled(ss, kind):
    """The sampled splitters judge the model on the 2^16-key sample: the
    learned splitters are kept unless their largest range bucket exceeds twice
    a range's share of the light keys (plus four standard deviations of
    counting noise) and also the sampled splitters' largest one; a rejected
    model leaves exactly the sampled partition.  Either way the
    output is the stable sort; the training stops within its step budget."""
    n = 1 << 24
    keys = {"uniform": lambda: synth.uniform_exact(94, n, n),
            "zipf12": lambda: synth.zipf(91, n, 1.2),
            "exponential": lambda: synth.exponential(92, n, 1e-6),
            "gaussian_mixture": lambda: synth.gaussian_mixture(93, n)}[kind]()
    vals = np.arange(n, dtype=np.uint64)
    _, _, st_s = run_less(ss, keys, vals, 0)
    ko, vo, st_l = run_less(ss, keys, vals, 1)
    assert st_s["l0_splitters"] == 0 and st_l["l0_splitters"] in (1, 2)
    assert 0 < st_l["learn_steps"] <= 400
    share_max = -(-65536 // st_s["l0_light_buckets"])
    limit = int(2 * share_max + 4 * np.sqrt(2 * share_max))  # twice the share plus counting noise
    if st_l["l0_splitters"] == 1:
        assert st_l["l0_max_sample_range"] <= max(limit, st_s["l0_max_sample_range"]), (st_l, st_s)
    else:
        assert st_l["l0_max_sample_range"] == st_s["l0_max_sample_range"]
        assert st_l["l0_max_light_bucket"] == st_s["l0_max_light_bucket"]
    if kind == "uniform":
        assert st_l["l0_splitters"] == 1  # smooth keys: the model beats the sample's quantile noise
    err = oracle.check_sorted_equal(keys, vals, ko, vo)
    assert err is None, err
