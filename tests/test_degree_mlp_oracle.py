"""Pins of the learned-degree oracle (oracle/degree_mlp.py) against what calculus and the
definition of Adam fix, independently of its own code: central finite differences of the
loss, a network small enough to differentiate by hand with the scalar chain rule, the
closed form of Adam's first step, and a planted mistake in the back-propagation that the
finite-difference check catches."""
import math

import numpy as np
import pytest

from oracle import degree_mlp as D


def _random_params(sizes, seed, scale=0.6):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, D.param_count(sizes))


def _fd_gradient(params, sizes, mean, scale, X, z, h=1e-6):
    g = np.empty_like(params)
    for k in range(params.size):
        p1, p2 = params.copy(), params.copy()
        p1[k] += h
        p2[k] -= h
        l1, _ = D.loss_and_gradient(p1, sizes, mean, scale, X, z)
        l2, _ = D.loss_and_gradient(p2, sizes, mean, scale, X, z)
        g[k] = (l1 - l2) / (2 * h)
    return g


def test_param_count_of_the_library_network():
    # 8 -> 64 -> 64 -> 64 -> 1: 8*64+64 + 2*(64*64+64) + 64+1
    assert D.param_count(D.LIBRARY_SIZES) == 576 + 2 * 4160 + 65 == 8961


@pytest.mark.parametrize("sizes", [(3, 4, 4, 4, 1), (2, 5, 1), (8, 6, 6, 6, 1)])
def test_gradient_matches_central_finite_differences(sizes):
    rng = np.random.default_rng(sum(sizes))
    params = _random_params(sizes, 1 + len(sizes))
    X = rng.normal(size=(17, sizes[0]))
    z = rng.normal(size=17)
    mean = rng.normal(0, 0.3, sizes[0])
    scale = rng.uniform(0.5, 2.0, sizes[0])
    _, g = D.loss_and_gradient(params, sizes, mean, scale, X, z)
    g_fd = _fd_gradient(params, sizes, mean, scale, X, z)
    assert np.max(np.abs(g - g_fd)) <= 1e-7 * np.max(np.abs(g_fd))


def test_one_input_two_hidden_units_worked_by_hand():
    # y = v1 tanh(w1 x + b1) + v2 tanh(w2 x + b2) + c, L = (y - z)^2 / 2 (one sample)
    w1, w2, b1, b2, v1, v2, c = 0.3, -0.2, 0.1, 0.0, 0.7, -0.4, 0.05
    x, z = 0.5, 0.2
    h1, h2 = math.tanh(w1 * x + b1), math.tanh(w2 * x + b2)
    y = v1 * h1 + v2 * h2 + c
    r = y - z
    expect = {
        "w1": r * v1 * (1 - h1 * h1) * x, "w2": r * v2 * (1 - h2 * h2) * x,
        "b1": r * v1 * (1 - h1 * h1), "b2": r * v2 * (1 - h2 * h2),
        "v1": r * h1, "v2": r * h2, "c": r,
    }
    # flat order: W1 (2 x 1) row by row, b1, W2 (1 x 2), b2
    params = np.array([w1, w2, b1, b2, v1, v2, c])
    loss, g = D.loss_and_gradient(params, (1, 2, 1), [0.0], [1.0], [[x]], [z])
    assert abs(loss - 0.5 * r * r) < 1e-15
    got = dict(zip(["w1", "w2", "b1", "b2", "v1", "v2", "c"], g))
    for k, v in expect.items():
        assert abs(got[k] - v) < 1e-15, k
    # the same values by hand: y = 0.7 tanh(0.25) - 0.4 tanh(-0.1) + 0.05
    assert abs(y - (0.7 * 0.24491866240370913 + 0.4 * 0.09966799462495582 + 0.05)) < 1e-15


def test_three_hidden_layers_of_one_unit_worked_by_hand():
    # chain y = u4 tanh(u3 tanh(u2 tanh(u1 x' + c1) + c2) + c3) + c4, x' = (x - mu) s
    u1, c1, u2, c2, u3, c3, u4, c4 = 0.8, -0.1, -1.1, 0.2, 0.6, 0.05, 1.3, -0.3
    mu, s, x, z = 0.4, 2.0, 0.9, 0.25
    xp = (x - mu) * s
    a1 = math.tanh(u1 * xp + c1)
    a2 = math.tanh(u2 * a1 + c2)
    a3 = math.tanh(u3 * a2 + c3)
    y = u4 * a3 + c4
    r = y - z
    d3 = r * u4 * (1 - a3 * a3)
    d2 = d3 * u3 * (1 - a2 * a2)
    d1 = d2 * u2 * (1 - a1 * a1)
    expect = [d1 * xp, d1, d2 * a1, d2, d3 * a2, d3, r * a3, r]
    params = np.array([u1, c1, u2, c2, u3, c3, u4, c4])
    yv, _ = D.forward(params, (1, 1, 1, 1, 1), [mu], [s], [[x]])
    assert abs(yv[0] - y) < 1e-15
    _, g = D.loss_and_gradient(params, (1, 1, 1, 1, 1), [mu], [s], [[x]], [z])
    assert np.max(np.abs(g - np.array(expect))) < 1e-15


def test_normalisation_is_applied_before_the_first_layer():
    sizes = (3, 4, 4, 4, 1)
    params = _random_params(sizes, 5)
    rng = np.random.default_rng(6)
    X = rng.normal(size=(9, 3))
    mean, scale = D.normalisation(X)
    y1, _ = D.forward(params, sizes, mean, scale, X)
    y2, _ = D.forward(params, sizes, np.zeros(3), np.ones(3), (X - X.mean(0)) / X.std(0))
    assert np.max(np.abs(y1 - y2)) < 1e-13
    # a constant feature keeps scale 1
    Xc = X.copy()
    Xc[:, 1] = 2.5
    _, sc = D.normalisation(Xc)
    assert sc[1] == 1.0


def test_first_adam_step_is_lr_times_the_gradient_sign():
    # from zero moments the bias-corrected estimates are g and g^2: the step is
    # lr g / (|g| + eps), i.e. lr sign(g) for |g| >> eps
    sizes = (2, 3, 3, 3, 1)
    p0 = _random_params(sizes, 7)
    rng = np.random.default_rng(8)
    X, z = rng.normal(size=(5, 2)), rng.normal(size=5)
    _, g = D.loss_and_gradient(p0, sizes, [0, 0], [1, 1], X, z)
    lr = 1e-3
    p1, m1, m2, step, _ = D.adam_epoch(p0, np.zeros_like(p0), np.zeros_like(p0), 0, sizes, [0, 0],
                                       [1, 1], X, z, np.arange(5), 5, lr)
    assert step == 1
    assert np.allclose(p0 - p1, lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-18)
    assert np.allclose(m1, 0.1 * g) and np.allclose(m2, 0.001 * g * g)


def test_adam_epochs_fit_a_smooth_target():
    sizes = (3, 16, 16, 16, 1)
    rng = np.random.default_rng(9)
    X = rng.normal(size=(400, 3))
    z = 0.5 * np.tanh(X[:, 0]) - 0.3 * X[:, 1] + 0.2 * X[:, 1] * X[:, 2]
    p = _random_params(sizes, 10, 0.3)
    m1, m2, step = np.zeros_like(p), np.zeros_like(p), 0
    mean, scale = D.normalisation(X)
    l0, _ = D.loss_and_gradient(p, sizes, mean, scale, X, z)
    for ep in range(40):
        order = np.random.default_rng(100 + ep).permutation(400)
        p, m1, m2, step, _ = D.adam_epoch(p, m1, m2, step, sizes, mean, scale, X, z, order, 32, 3e-3)
    l1, _ = D.loss_and_gradient(p, sizes, mean, scale, X, z)
    assert l1 < 0.1 * l0


def test_finite_differences_catch_a_planted_backprop_mistake():
    """A copy of the back-propagation with the tanh derivative written as (1 - a) instead
    of (1 - a^2): the finite-difference pin above would reject it."""
    sizes = (3, 4, 4, 4, 1)
    rng = np.random.default_rng(11)
    params = _random_params(sizes, 12)
    X, z = rng.normal(size=(7, 3)), rng.normal(size=7)
    mean, scale = np.zeros(3), np.ones(3)

    def wrong_gradient(p):
        y, acts = D.forward(p, sizes, mean, scale, X)
        layers = D.unpack(p, sizes)
        delta = ((y - z) / z.size)[:, None]
        grads = [None] * len(layers)
        for l in range(len(layers) - 1, -1, -1):
            grads[l] = (delta.T @ acts[l], delta.sum(axis=0))
            if l > 0:
                delta = (delta @ layers[l][0]) * (1.0 - acts[l])   # the planted mistake
        return D.pack(grads)

    g_fd = _fd_gradient(params, sizes, mean, scale, X, z)
    assert np.max(np.abs(wrong_gradient(params) - g_fd)) > 1e-3 * np.max(np.abs(g_fd))
