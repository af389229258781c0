"""Learned step-size proposer: the small MLP of the build's learned part
(test infrastructure; the paper has no learned component).

Network: x (6) -> tanh(W1 x + b1) (32) -> tanh(W2 h1 + b2) (32) -> W3 h2 + b3 (1),
1313 parameters, flattened in the order W1 (32x6, row-major), b1, W2 (32x32),
b2, W3 (32), b3.  Inputs are standardised with fixed (mean, std) pairs.

Features of an accepted step n (from the solver's step history):
  [log r_{n-3}, log r_{n-2}, log r_{n-1}, log r_n, log h_n, log Rel],
  r = clamp(E / Rel, 1e-8, 1e8) over the accepted steps (earlier entries repeat
  the first one).  Output: d = log(h_{n+1} / h_n), applied as
  h_{n+1} = h_n exp(clamp(d, log 0.2, log 5)).

Training target, from the next accepted step (n+1, taken at h_{n+1} with error
E_{n+1}): the step that would have produced E = THETA Rel under the local model
E ~ h^3, h* = h_{n+1} (THETA Rel / E_{n+1})^(1/3); target d* = log(h* / h_n).

Pinned in tests/test_oracle_mlp.py: forward and gradients against torch's own
linear/tanh and autograd, Adam against a convex problem's minimum.
"""

from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np

N_IN, N_H = 6, 32
N_PARAMS = N_H * N_IN + N_H + N_H * N_H + N_H + N_H + 1   # 1313
THETA = 0.75
R_CLAMP = 1e-8
D_MIN, D_MAX = math.log(0.2), math.log(5.0)


def unpack(p):
    p = np.asarray(p)
    o = 0
    W1 = p[o:o + N_H * N_IN].reshape(N_H, N_IN); o += N_H * N_IN
    b1 = p[o:o + N_H]; o += N_H
    W2 = p[o:o + N_H * N_H].reshape(N_H, N_H); o += N_H * N_H
    b2 = p[o:o + N_H]; o += N_H
    W3 = p[o:o + N_H]; o += N_H
    b3 = p[o]
    return W1, b1, W2, b2, W3, b3


def init_params(seed: int) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    p = np.zeros(N_PARAMS)
    o = 0
    for fan_in, fan_out in ((N_IN, N_H), (N_H, N_H), (N_H, 1)):
        a = 1.0 / math.sqrt(fan_in)
        p[o:o + fan_in * fan_out] = rng.uniform(-a, a, fan_in * fan_out)
        o += fan_in * fan_out + fan_out
    return p


def forward(p, X):
    """X [n, 6] (already standardised) -> y [n]."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ W3 + b3


def loss_and_grad(p, X, y):
    """Mean squared error 0.5 mean((f(x) - y)^2) and its gradient (backprop)."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    n = X.shape[0]
    a1 = X @ W1.T + b1
    h1 = np.tanh(a1)
    a2 = h1 @ W2.T + b2
    h2 = np.tanh(a2)
    out = h2 @ W3 + b3
    r = out - y
    loss = 0.5 * np.mean(r * r)
    g_out = r / n
    gW3 = h2.T @ g_out
    gb3 = g_out.sum()
    g_h2 = np.outer(g_out, W3)
    g_a2 = g_h2 * (1.0 - h2 * h2)
    gW2 = g_a2.T @ h1
    gb2 = g_a2.sum(axis=0)
    g_h1 = g_a2 @ W2
    g_a1 = g_h1 * (1.0 - h1 * h1)
    gW1 = g_a1.T @ X
    gb1 = g_a1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return loss, g


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), t = 1, 2, ...; returns (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def features(err_hist: Sequence[float], h: float, rtol: float) -> np.ndarray:
    r = [min(max(e / rtol, R_CLAMP), 1.0 / R_CLAMP) for e in err_hist[-4:]]
    while len(r) < 4:
        r.insert(0, r[0])
    return np.array([math.log(x) for x in r] + [math.log(h), math.log(rtol)])


def dataset_from_history(hist: np.ndarray, rtol: float):
    """Rows (t, h, E, accepted, ...) of one solve -> (X raw features, y targets)."""
    acc = hist[hist[:, 3] > 0.5]
    X, y = [], []
    errs: List[float] = []
    for n in range(len(acc) - 1):
        errs.append(acc[n, 2])
        h_n, h_next, e_next = acc[n, 1], acc[n + 1, 1], acc[n + 1, 2]
        r_next = min(max(e_next / rtol, R_CLAMP), 1.0 / R_CLAMP)
        h_star = h_next * (THETA / r_next) ** (1.0 / 3.0)
        X.append(features(errs, h_n, rtol))
        y.append(math.log(h_star / h_n))
    return np.array(X).reshape(-1, N_IN), np.array(y)


def bf16(x):
    """Round binary32 values to bfloat16 (nearest even), returned as binary32."""
    from .formats import round_bf16
    return round_bf16(np.asarray(x, dtype=np.float32))


class Proposer:
    """The proposer as the solver applies it: bfloat16 weights and biases,
    binary32 arithmetic, standardised inputs, clamped output."""

    def __init__(self, params, mean, std):
        self.p = bf16(params).astype(np.float32)
        self.mean = np.asarray(mean, dtype=np.float32)
        self.std = np.asarray(std, dtype=np.float32)

    def __call__(self, err_hist, h, rtol, h_ctrl):
        x = ((features(err_hist, h, rtol).astype(np.float32) - self.mean) / self.std).astype(np.float32)
        W1, b1, W2, b2, W3, b3 = unpack(self.p)
        h1 = np.tanh((W1 @ x + b1).astype(np.float32)).astype(np.float32)
        h2 = np.tanh((W2 @ h1 + b2).astype(np.float32)).astype(np.float32)
        d = float(np.float32(np.dot(W3, h2) + b3))
        return h * math.exp(min(max(d, D_MIN), D_MAX))
