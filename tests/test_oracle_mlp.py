"""Pins of the oracle's learned-radius network (CPU): the backward pass against
central finite differences of the forward pass, and the forward pass against a
closed form."""
import math

import numpy as np

from oracle import mlp as O


def test_forward_closed_form_with_zero_matrices():
    d = 3
    rng = np.random.default_rng(0)
    theta = np.zeros(O.param_count(d))
    W1, b1, W2, b2, w3, b3 = O.unpack(theta, d)
    b1[:] = rng.standard_normal(64)
    b2[:] = rng.standard_normal(64)
    w3[:] = rng.standard_normal(64)
    theta[-1] = 0.7
    X = rng.standard_normal((5, d))
    # W1 = W2 = 0: every sample gives b3 + sum_j w3_j GELU(b2_j)
    g = lambda z: 0.5 * z * (1 + math.erf(z / math.sqrt(2)))
    expect = 0.7 + sum(w3[j] * g(b2[j]) for j in range(64))
    np.testing.assert_allclose(O.forward(theta, X), expect, rtol=1e-14)


def test_gelu_values():
    # GELU(0) = 0, GELU(z) - GELU(-z) = z, GELU'(0) = 1/2
    z = np.linspace(-3, 3, 13)
    np.testing.assert_allclose(O.gelu(z) - O.gelu(-z), z, atol=1e-15)
    assert O.gelu(np.array(0.0)) == 0.0 and O.gelu_prime(np.array(0.0)) == 0.5


def test_gradient_matches_central_differences():
    d = 4
    rng = np.random.default_rng(1)
    theta = 0.3 * rng.standard_normal(O.param_count(d))
    X = rng.standard_normal((40, d))
    Y = rng.standard_normal(40)
    _, g = O.loss_and_grad(theta, X, Y)
    h = 1e-6
    idx = np.concatenate([rng.choice(O.param_count(d), 60, replace=False), [O.param_count(d) - 1]])
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (np.mean((O.forward(tp, X) - Y) ** 2) - np.mean((O.forward(tm, X) - Y) ** 2)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])
