"""Pins of the oracle's MLP proposer against torch's own layers and autograd,
Adam against a convex minimum, and the target against the h^3 error model."""

import math

import numpy as np
import torch

from oracle import mlp


def _torch_forward(p, X):
    W1, b1, W2, b2, W3, b3 = (torch.tensor(a, dtype=torch.float64, requires_grad=True) for a in mlp.unpack(p))
    x = torch.tensor(X, dtype=torch.float64)
    h1 = torch.tanh(torch.nn.functional.linear(x, W1, b1))
    h2 = torch.tanh(torch.nn.functional.linear(h1, W2, b2))
    out = torch.nn.functional.linear(h2, W3.reshape(1, -1), b3.reshape(1)).reshape(-1)
    return out, (W1, b1, W2, b2, W3, b3)


def test_parameter_count():
    assert mlp.N_PARAMS == 1313


def test_forward_and_gradient_match_torch():
    rng = np.random.default_rng(0)
    p = mlp.init_params(1) + 0.1 * rng.standard_normal(mlp.N_PARAMS)
    X = rng.standard_normal((50, 6))
    y = rng.standard_normal(50)
    out, ts = _torch_forward(p, X)
    np.testing.assert_allclose(mlp.forward(p, X), out.detach().numpy(), rtol=1e-12, atol=1e-12)
    loss_t = 0.5 * torch.mean((out - torch.tensor(y)) ** 2)
    loss_t.backward()
    g_t = np.concatenate([t.grad.numpy().ravel() for t in ts])
    loss, g = mlp.loss_and_grad(p, X, y)
    assert abs(loss - loss_t.item()) < 1e-12
    np.testing.assert_allclose(g, g_t, rtol=1e-10, atol=1e-12)


def test_adam_reaches_convex_minimum():
    A = np.diag([1.0, 10.0, 0.1])
    b = np.array([1.0, -2.0, 3.0])
    x = np.zeros(3)
    m = np.zeros(3); v = np.zeros(3)
    for t in range(1, 20001):
        g = A @ x - b
        x, m, v = mlp.adam_step(x, g, m, v, t, 0.01)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-3, atol=1e-3)


def test_target_inverts_the_local_error_model():
    """E = C h^3 exactly: the target step gives E = THETA Rel."""
    C, rtol = 7.0, 1e-6
    hs = 0.01 * np.exp(0.1 * np.arange(8))
    hist = np.zeros((8, 8))
    hist[:, 1] = hs
    hist[:, 2] = C * hs ** 3
    hist[:, 3] = 1.0
    X, y = mlp.dataset_from_history(hist, rtol)
    h_star = hs[:-1] * np.exp(y)
    np.testing.assert_allclose(C * h_star ** 3, mlp.THETA * rtol, rtol=1e-10)
    np.testing.assert_allclose(X[:, 4], np.log(hs[:-1]))
    np.testing.assert_allclose(X[3, :4], np.log(hist[:4, 2] / rtol))
    np.testing.assert_allclose(X[0, :4], np.log(hist[0, 2] / rtol))


def test_proposer_with_constant_output():
    p = np.zeros(mlp.N_PARAMS)
    p[-1] = math.log(1.25)
    prop = mlp.Proposer(p, np.zeros(6), np.ones(6))
    b3 = float(mlp.bf16(np.array([math.log(1.25)], dtype=np.float32))[0])
    h = prop([1e-7, 2e-7], 0.1, 1e-6, 0.2)
    assert abs(h - 0.1 * math.exp(b3)) < 1e-12
    p[-1] = 10.0
    assert abs(mlp.Proposer(p, np.zeros(6), np.ones(6))([1e-7], 0.1, 1e-6, 0.2) - 0.5) < 1e-12
