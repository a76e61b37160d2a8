"""FP64 reference of the learned-radius network (TEST INFRASTRUCTURE ONLY; see
oracle/__init__.py).

The network the kNN search uses to guess each point's k-th neighbour distance:
in -> 64 -> 64 -> 1 with GELU in its erf form, GELU(z) = z (1 + erf(z / sqrt 2)) / 2,
fitted by mean squared error on standardised log radii.  Parameter layout:
W1 [64][in], b1 [64], W2 [64][64], b2 [64], w3 [64], b3.  `loss_and_grad`
is the plain chain rule in FP64; the tests pin it to central finite
differences of `forward` and `forward` to a closed-form case.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

H = 64


def unpack(theta: np.ndarray, d: int):
    o = 0
    W1 = theta[o:o + H * d].reshape(H, d); o += H * d
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    w3 = theta[o:o + H]; o += H
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def param_count(d: int) -> int:
    return H * d + H + H * H + H + H + 1


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_prime(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(theta: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Network output for standardised inputs X [n, d]."""
    W1, b1, W2, b2, w3, b3 = unpack(theta, X.shape[1])
    h1 = gelu(X @ W1.T + b1)
    h2 = gelu(h1 @ W2.T + b2)
    return h2 @ w3 + b3


def loss_and_grad(theta: np.ndarray, X: np.ndarray, Y: np.ndarray):
    """Mean squared error of forward(X) against Y and its gradient (chain rule, FP64)."""
    n, d = X.shape
    W1, b1, W2, b2, w3, b3 = unpack(theta, d)
    z1 = X @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    out = h2 @ w3 + b3
    e = out - Y
    loss = float(np.mean(e * e))
    dout = 2.0 * e / n
    g_w3 = h2.T @ dout
    g_b3 = dout.sum()
    dz2 = (dout[:, None] * w3[None, :]) * gelu_prime(z2)
    g_W2 = dz2.T @ h1
    g_b2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * gelu_prime(z1)
    g_W1 = dz1.T @ X
    g_b1 = dz1.sum(0)
    grad = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, grad
