"""Pins for the oracle MLP: finite differences, closed forms and Adam's first step."""
import math

import numpy as np

from oracle import mlp


def _problem(seed=0, B=6, F=16, C=5):
    rng = np.random.default_rng(seed)
    params = mlp.init_params(F, C, rng)
    X = rng.standard_normal((B, F))
    Y = np.zeros((B, C))
    Y[np.arange(B), rng.integers(0, C, B)] = 1.0
    return params, X, Y


def test_gradient_matches_central_differences():
    params, X, Y = _problem()
    loss, grads = mlp.loss_and_grad(params, X, Y)
    rng = np.random.default_rng(1)
    h = 1e-6
    for li, p in enumerate(params):
        for _ in range(6):
            idx = tuple(rng.integers(0, n) for n in p.shape)
            old = p[idx]
            p[idx] = old + h
            lp, _ = mlp.loss_and_grad(params, X, Y)
            p[idx] = old - h
            lm, _ = mlp.loss_and_grad(params, X, Y)
            p[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[li][idx]) <= 1e-6 * max(1.0, abs(fd)), (li, idx)


def test_soft_targets_gradient():
    params, X, _ = _problem(seed=3)
    rng = np.random.default_rng(4)
    Y = rng.random((X.shape[0], 5))
    Y /= Y.sum(axis=1, keepdims=True)
    _, grads = mlp.loss_and_grad(params, X, Y)
    h = 1e-6
    p = params[-1]
    old = p[2]
    p[2] = old + h
    lp, _ = mlp.loss_and_grad(params, X, Y)
    p[2] = old - h
    lm, _ = mlp.loss_and_grad(params, X, Y)
    p[2] = old
    assert abs((lp - lm) / (2 * h) - grads[-1][2]) < 1e-7


def test_uniform_logits_loss_is_log_classes():
    params, X, Y = _problem(C=7)
    for l in range(mlp.LAYERS):
        params[2 * l][:] = 0
        params[2 * l + 1][:] = 0
    loss, grads = mlp.loss_and_grad(params, X, Y)
    assert abs(loss - math.log(7)) < 1e-15
    # with zero hidden activations only the output bias gets a gradient: mean(p - y)
    assert np.allclose(grads[-1], (np.full_like(Y, 1 / 7) - Y).mean(axis=0), atol=1e-15)
    assert np.all(grads[-2] == 0)


def test_adam_first_step_is_lr_times_sign():
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -4.0, 1e-3])]
    z = [np.zeros(3)]
    newp, m, v = mlp.adam_step(p, g, z, z, t=1, lr=0.01, eps=1e-12)
    assert np.allclose(newp[0], p[0] - 0.01 * np.sign(g[0]), atol=1e-9)
    assert np.allclose(m[0], 0.1 * g[0]) and np.allclose(v[0], 0.001 * g[0] ** 2)


def test_adam_weight_decay_is_the_l2_gradient():
    # decay alone (zero loss gradient): the first step moves each parameter
    # by lr against its own sign, and m holds (1 - beta1) * wd * p
    p = [np.array([1.0, -2.0, 0.0])]
    z = [np.zeros(3)]
    newp, m, _ = mlp.adam_step(p, z, z, z, t=1, lr=0.01, eps=1e-12, weight_decay=0.5)
    assert np.allclose(newp[0], [0.99, -1.99, 0.0], atol=1e-9)
    assert np.allclose(m[0], 0.1 * 0.5 * p[0])


def test_training_reduces_loss():
    params, X, Y = _problem(seed=7, B=32)
    m = [np.zeros_like(p) for p in params]
    v = [np.zeros_like(p) for p in params]
    l0, _ = mlp.loss_and_grad(params, X, Y)
    for t in range(1, 101):
        _, g = mlp.loss_and_grad(params, X, Y)
        params, m, v = mlp.adam_step(params, g, m, v, t, lr=1e-2)
    l1, _ = mlp.loss_and_grad(params, X, Y)
    assert l1 < 0.2 * l0
