"""Oracle for the learned splitters of semisort_< (test infrastructure only:
used by tests/, never by the library).

A monotone CDF model f: [0, 1] -> R, a 1-32-32-1 perceptron whose weights are
kept positive through softplus and whose hidden units are logistic sigmoids,
so f is non-decreasing in its input:

    w1 = softplus(v1), w2 = softplus(v2), w3 = softplus(v3)
    h1 = sigmoid(w1 * x + c1)                 (32 units)
    h2 = sigmoid(w2 @ h1 + c2)                (32 units; w2[j, i] joins h1_i to h2_j)
    f(x) = w3 . h2 + c3

Trained by mean squared error on (x_m, t_m) pairs -- normalized sample keys
and their ranks -- with Adam (Kingma and Ba, 2015), then inverted by bisection
over the integer key domain to give splitter keys.  Everything here is plain
numpy in float64, written from the definitions: forward pass, analytic
backward pass, Adam, bisection.

Parameter vector layout (1153 floats): v1[32] | c1[32] | v2[32*32] (row j
holds the weights into h2_j) | c2[32] | v3[32] | c3.
"""
from __future__ import annotations

import numpy as np

H = 32
N_PARAMS = H + H + H * H + H + H + 1
SLICES = {"v1": (0, H), "c1": (H, 2 * H), "v2": (2 * H, 2 * H + H * H), "c2": (2 * H + H * H, 3 * H + H * H),
          "v3": (3 * H + H * H, 4 * H + H * H), "c3": (4 * H + H * H, 4 * H + H * H + 1)}


def unpack(p: np.ndarray) -> dict:
    p = np.asarray(p, dtype=np.float64)
    d = {k: p[a:b] for k, (a, b) in SLICES.items()}
    d["v2"] = d["v2"].reshape(H, H)
    return d


def softplus(v):
    return np.log1p(np.exp(-np.abs(v))) + np.maximum(v, 0.0)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(p, x):
    """f(x) for an array of inputs; also the hidden activations."""
    q = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    w1, w2, w3 = softplus(q["v1"]), softplus(q["v2"]), softplus(q["v3"])
    h1 = sigmoid(np.outer(x, w1) + q["c1"])
    h2 = sigmoid(h1 @ w2.T + q["c2"])
    return h2 @ w3 + q["c3"][0], h1, h2


def loss(p, x, t) -> float:
    y, _, _ = forward(p, x)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def loss_grad(p, x, t):
    """(loss, gradient w.r.t. the parameter vector) by the chain rule."""
    q = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    w1, w2, w3 = softplus(q["v1"]), softplus(q["v2"]), softplus(q["v3"])
    y, h1, h2 = forward(p, x)
    m = x.shape[0]
    e = 2.0 * (y - t) / m                          # dL/dy per point
    g = np.zeros(N_PARAMS)
    d2 = e[:, None] * w3[None, :] * h2 * (1.0 - h2)   # dL/dz2
    d1 = (d2 @ w2) * h1 * (1.0 - h1)                  # dL/dz1
    gw3 = h2.T @ e
    gw2 = d2.T @ h1
    gw1 = d1.T @ x
    a, b = SLICES["v1"]; g[a:b] = gw1 * sigmoid(q["v1"])       # softplus' = sigmoid
    a, b = SLICES["c1"]; g[a:b] = d1.sum(axis=0)
    a, b = SLICES["v2"]; g[a:b] = (gw2 * sigmoid(q["v2"])).ravel()
    a, b = SLICES["c2"]; g[a:b] = d2.sum(axis=0)
    a, b = SLICES["v3"]; g[a:b] = gw3 * sigmoid(q["v3"])
    a, b = SLICES["c3"]; g[a:b] = e.sum()
    return float(np.mean((y - t) ** 2)), g


def adam(p, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def train(p0, x, t, steps: int, lr: float):
    """Full-batch Adam from p0; returns (params, final loss)."""
    p = np.array(p0, dtype=np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for s in range(1, steps + 1):
        _, g = loss_grad(p, x, t)
        p, m, v = adam(p, g, m, v, s, lr)
    return p, loss(p, x, t)


def invert(p, kmin: int, kmax: int, nl: int, f=None):
    """Splitter j (1 <= j < nl): the smallest integer key k in [kmin, kmax]
    with f((k - kmin) / (kmax - kmin)) >= j / nl (kmax if none), by bisection;
    then made non-decreasing.  `f` overrides the model evaluation (a callable
    on an array of normalized inputs)."""
    f = f or (lambda xs: forward(p, xs)[0])
    span = float(kmax - kmin) if kmax > kmin else 1.0
    out = []
    for j in range(1, nl):
        tau = j / nl
        lo, hi = kmin, kmax
        while lo < hi:
            mid = lo + (hi - lo) // 2
            if f(np.array([(mid - kmin) / span]))[0] < tau:
                lo = mid + 1
            else:
                hi = mid
        out.append(lo)
    return np.maximum.accumulate(np.array(out, dtype=np.uint64)) if out else np.zeros(0, np.uint64)
