"""Pins of the FP64 surrogate-network reference: gradients against central finite
differences, the input gradient likewise, a one-unit network against its closed form, and
Adam's first step against its definition (the first bias-corrected step is lr * sign(g))."""
import numpy as np

from oracle import mlp_oracle as M


def _setup(D=4, H=8, N=13, seed=3):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(M.n_params(D, H)) * 0.5
    X = rng.standard_normal((N, D))
    y = rng.standard_normal(N)
    return p, X, y


def test_parameter_gradient_matches_central_differences():
    D, H = 4, 8
    p, X, y = _setup(D, H)
    _, g = M.loss_and_grad(p, X, y, D, H)
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(len(p)):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (M.loss_and_grad(p + e, X, y, D, H)[0] - M.loss_and_grad(p - e, X, y, D, H)[0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-8)


def test_input_gradient_matches_central_differences():
    D, H = 4, 8
    p, X, _ = _setup(D, H)
    g = M.input_grad(p, X, D, H)
    h = 1e-6
    for d in range(D):
        e = np.zeros(D)
        e[d] = h
        fd = (M.forward(p, X + e, D, H)[0] - M.forward(p, X - e, D, H)[0]) / (2 * h)
        np.testing.assert_allclose(g[:, d], fd, rtol=1e-6, atol=1e-9)


def test_single_unit_network_closed_form():
    # H = 1, D = 1: f(x) = w3 tanh(W2 tanh(W1 x + b1) + b2) + b3
    p = np.array([0.7, -0.2, 1.3, 0.1, -0.8, 0.25])
    x = np.array([[0.4], [-1.1]])
    f = M.forward(p, x, 1, 1)[0]
    ref = -0.8 * np.tanh(1.3 * np.tanh(0.7 * x[:, 0] - 0.2) + 0.1) + 0.25
    np.testing.assert_allclose(f, ref, rtol=1e-15)


def test_adam_first_step_is_lr_times_sign():
    g = np.array([3.0, -1e-3, 0.5])
    p1, m, v = M.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(p1, -0.01 * np.sign(g), rtol=1e-12)
