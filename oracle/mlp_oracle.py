"""FP64 reference of the surrogate network (test infrastructure: only tests, the smoke check
and the benchmark's CPU baseline may use this module; the product path never does).

The paper has no surrogate; the network is the learned part of the build (a small MLP of
log pi~(theta|y) trained on exact evaluations).  This module states its definition plainly,
in FP64 numpy, for the gradient checks of the GPU kernels:

    a1 = tanh(W1 x + b1),  a2 = tanh(W2 a1 + b2),  f(x) = w3 . a2 + b3,
    loss = (1/N) sum_n (f(x_n) - y_n)^2,

with parameters packed in the order W1 (H x D, row-major), b1 (H), W2 (H x H), b2 (H),
w3 (H), b3 (1).  Gradients by the chain rule written out (backpropagation); the tests pin
them against central finite differences.  Adam: Kingma & Ba, "Adam: a method for stochastic
optimization", ICLR 2015 (bias-corrected first and second moments).
"""
from __future__ import annotations

import numpy as np


def n_params(D: int, H: int) -> int:
    return H * D + H + H * H + H + H + 1


def unpack(p: np.ndarray, D: int, H: int):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * D].reshape(H, D); o += H * D
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p, X, D, H):
    """Network output f (N) and the activations (a1, a2), each N x H."""
    W1, b1, W2, b2, w3, b3 = unpack(p, D, H)
    X = np.asarray(X, dtype=np.float64)
    a1 = np.tanh(X @ W1.T + b1)
    a2 = np.tanh(a1 @ W2.T + b2)
    return a2 @ w3 + b3, a1, a2


def loss_and_grad(p, X, y, D, H):
    """Mean squared error over the N samples and its gradient with respect to p."""
    W1, b1, W2, b2, w3, b3 = unpack(p, D, H)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    N = X.shape[0]
    f, a1, a2 = forward(p, X, D, H)
    r = f - y
    loss = float(np.mean(r * r))
    d3 = 2.0 * r / N                      # dloss/df, N
    g_w3 = a2.T @ d3
    g_b3 = d3.sum()
    d2 = np.outer(d3, w3) * (1.0 - a2 * a2)   # N x H
    g_W2 = d2.T @ a1
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (1.0 - a1 * a1)          # N x H
    g_W1 = d1.T @ X
    g_b1 = d1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, g


def input_grad(p, X, D, H):
    """df/dx for each sample (N x D)."""
    W1, b1, W2, b2, w3, b3 = unpack(p, D, H)
    f, a1, a2 = forward(p, X, D, H)
    d2 = w3[None, :] * (1.0 - a2 * a2)
    d1 = (d2 @ W2) * (1.0 - a1 * a1)
    return d1 @ W1


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns the new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
