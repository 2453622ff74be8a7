"""Pins of the oracle's warm-start network (plain loops in oracle/mlp_oracle.c):
closed forms for the linear layer and a one-unit network, finite differences
of the loss for the backpropagated gradient, and the special cases of Adam
that its definition fixes exactly (first step, constant gradient)."""
import math

import numpy as np
import pytest

import oracle

WIDTHS_WARM_START = [9, 128, 128, 128, 128, 1]


def test_parameter_count_of_the_warm_start_network():
    # 9*128+128 + 3*(128*128+128) + 128+1
    assert oracle.mlp_nparams(WIDTHS_WARM_START) == 50945


def test_one_hidden_unit_by_hand():
    # y = w2 tanh(w1 x + b1) + b2
    w1, b1, w2, b2 = 2.0, -0.5, 3.0, 0.25
    theta = np.array([w1, b1, w2, b2])
    x = 0.5
    y = oracle.mlp_forward([1, 1, 1], theta, np.array([[x]]))[0]
    assert y == pytest.approx(w2 * math.tanh(w1 * x + b1) + b2, rel=1e-15)
    # its gradient, differentiated by hand
    t = 0.7
    loss, g = oracle.mlp_grad([1, 1, 1], theta, np.array([[x]]), np.array([t]))
    h = math.tanh(w1 * x + b1)
    e = 2.0 * (w2 * h + b2 - t)
    assert loss == pytest.approx((w2 * h + b2 - t) ** 2, rel=1e-14)
    dz = e * w2 * (1 - h * h)
    assert g == pytest.approx([dz * x, dz, e * h, e], rel=1e-13)


def test_linear_layer_gradient_closed_form():
    # no hidden layer: y = W x + b, grad W = (2/B) sum (y - t) x^T, grad b = (2/B) sum (y - t)
    rng = np.random.default_rng(1)
    B, n = 11, 4
    W, b = rng.standard_normal(n), rng.standard_normal()
    X, T = rng.standard_normal((B, n)), rng.standard_normal(B)
    theta = np.concatenate([W, [b]])
    loss, g = oracle.mlp_grad([n, 1], theta, X, T)
    r = X @ W + b - T
    assert loss == pytest.approx(np.mean(r ** 2), rel=1e-13)
    assert g[:n] == pytest.approx(2.0 / B * (X.T @ r), rel=1e-12, abs=1e-14)
    assert g[n] == pytest.approx(2.0 / B * r.sum(), rel=1e-12)


@pytest.mark.parametrize("widths", [[5, 6, 7, 1], [3, 16, 16, 16, 1], [9, 12, 12, 12, 12, 1]])
def test_gradient_matches_central_differences(widths):
    rng = np.random.default_rng(len(widths))
    n = oracle.mlp_nparams(widths)
    theta = rng.standard_normal(n) * 0.4
    X = rng.standard_normal((13, widths[0]))
    T = rng.standard_normal(13)
    _, g = oracle.mlp_grad(widths, theta, X, T)
    idx = rng.choice(n, size=min(n, 60), replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(n)
        e[i] = h
        fd = (oracle.mlp_grad(widths, theta + e, X, T)[0] - oracle.mlp_grad(widths, theta - e, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, np.abs(g).max()), (i, fd, g[i])


def test_forward_is_the_loss_minimiser_output():
    # loss = mean((forward - T)^2) for the same parameters
    rng = np.random.default_rng(3)
    w = [4, 8, 8, 1]
    theta = rng.standard_normal(oracle.mlp_nparams(w)) * 0.5
    X, T = rng.standard_normal((17, 4)), rng.standard_normal(17)
    loss, _ = oracle.mlp_grad(w, theta, X, T)
    y = oracle.mlp_forward(w, theta, X)
    assert loss == pytest.approx(np.mean((y - T) ** 2), rel=1e-14)


def test_adam_first_step_and_constant_gradient():
    # with zero moments, the bias-corrected moments equal g and g^2 at every
    # step of a constant gradient, so each step moves by lr * g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-9, 0.0])
    theta = np.array([1.0, 2.0, 3.0, 4.0])
    m, v = np.zeros(4), np.zeros(4)
    lr, eps = 1e-2, 1e-8
    expect = theta.copy()
    for t in range(1, 6):
        oracle.adam_step(theta, m, v, g, t, lr=lr, eps=eps)
        expect = expect - lr * g / (np.abs(g) + eps)
        assert theta == pytest.approx(expect, rel=1e-12, abs=1e-15)


def test_adam_moments_follow_their_recursions():
    rng = np.random.default_rng(5)
    theta, m, v = np.zeros(6), np.zeros(6), np.zeros(6)
    gs = [rng.standard_normal(6) for _ in range(3)]
    for t, g in enumerate(gs, 1):
        oracle.adam_step(theta, m, v, g, t, lr=0.1, b1=0.5, b2=0.25)
    # closed forms of the exponential averages after three steps
    m3 = 0.5 * (0.5 * (0.5 * gs[0]) + 0.5 * gs[1]) + 0.5 * gs[2]
    v3 = 0.25 * (0.25 * (0.75 * gs[0] ** 2) + 0.75 * gs[1] ** 2) + 0.75 * gs[2] ** 2
    assert m == pytest.approx(m3, rel=1e-14)
    assert v == pytest.approx(v3, rel=1e-14)


def test_training_fits_a_teacher_network():
    # a student of the same shape trained by Adam on a teacher's outputs
    rng = np.random.default_rng(7)
    w = [2, 8, 8, 1]
    n = oracle.mlp_nparams(w)
    teacher = rng.standard_normal(n)
    X = rng.uniform(-1, 1, (64, 2))
    T = oracle.mlp_forward(w, teacher, X)
    theta = rng.standard_normal(n) * 0.3
    m, v = np.zeros(n), np.zeros(n)
    l0, _ = oracle.mlp_grad(w, theta, X, T)
    for t in range(1, 401):
        _, g = oracle.mlp_grad(w, theta, X, T)
        oracle.adam_step(theta, m, v, g, t, lr=1e-2)
    l1, _ = oracle.mlp_grad(w, theta, X, T)
    assert l1 < 0.02 * l0
