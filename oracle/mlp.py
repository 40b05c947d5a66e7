"""Oracle: the schedule selector's MLP in FP64.  Test infrastructure.

The selector maps a standardised feature vector x to logits over candidate
schedules through three hidden layers of 64 ReLU units:

    h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), h3 = relu(W3 h2 + b3),
    z  = W4 h3 + b4

and is trained on measured runtimes with softmax cross-entropy against a
target distribution y over the candidates (one-hot on the fastest candidate,
or soft):  loss = mean_batch( -sum_c y_c log softmax(z)_c ).

Gradients are the textbook backpropagation of that loss; parameters are updated
with Adam (bias-corrected first and second moments).  Weights are stored
row-major as [out][in].
"""
from __future__ import annotations

import numpy as np

HIDDEN = 64
LAYERS = 4          # three hidden layers + the output layer
__all__ = ["HIDDEN", "init_params", "forward", "loss_and_grad", "adam_step", "softmax"]


def init_params(n_in: int, n_out: int, rng: np.random.Generator):
    """He-uniform initialisation (weights), zero biases."""
    sizes = [n_in, HIDDEN, HIDDEN, HIDDEN, n_out]
    params = []
    for l in range(LAYERS):
        fan_in = sizes[l]
        lim = np.sqrt(6.0 / fan_in)
        W = rng.uniform(-lim, lim, size=(sizes[l + 1], sizes[l]))
        b = np.zeros(sizes[l + 1])
        params += [W, b]
    return params


def softmax(z):
    z = np.asarray(z, dtype=np.float64)
    e = np.exp(z - z.max(axis=1, keepdims=True))
    return e / e.sum(axis=1, keepdims=True)


def forward(params, X):
    """Returns (logits, activations) for a batch X (B x n_in)."""
    acts = [np.asarray(X, dtype=np.float64)]
    h = acts[0]
    for l in range(LAYERS):
        W, b = params[2 * l], params[2 * l + 1]
        a = h @ W.T + b
        h = np.maximum(a, 0.0) if l < LAYERS - 1 else a
        acts.append(h)
    return h, acts


def loss_and_grad(params, X, Y):
    """Mean softmax cross-entropy of the batch against target rows Y and the
    gradient of that loss with respect to every parameter."""
    z, acts = forward(params, X)
    Y = np.asarray(Y, dtype=np.float64)
    Bn = z.shape[0]
    zs = z - z.max(axis=1, keepdims=True)
    logp = zs - np.log(np.exp(zs).sum(axis=1, keepdims=True))
    loss = float(-(Y * logp).sum() / Bn)
    p = np.exp(logp)
    g = (p * Y.sum(axis=1, keepdims=True) - Y) / Bn       # dloss/dz
    grads = [None] * (2 * LAYERS)
    for l in range(LAYERS - 1, -1, -1):
        W = params[2 * l]
        grads[2 * l] = g.T @ acts[l]
        grads[2 * l + 1] = g.sum(axis=0)
        if l > 0:
            g = (g @ W) * (acts[l] > 0)
    return loss, grads


def adam_step(params, grads, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
              weight_decay=0.0):
    """One Adam update (step number t >= 1) of the objective L + (wd/2)|p|^2,
    whose gradient is g + wd * p.  Returns new (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    for p, g, mm, vv in zip(params, grads, m, v):
        g = g + weight_decay * p
        mm = beta1 * mm + (1 - beta1) * g
        vv = beta2 * vv + (1 - beta2) * g * g
        mhat = mm / (1 - beta1 ** t)
        vhat = vv / (1 - beta2 ** t)
        out_p.append(p - lr * mhat / (np.sqrt(vhat) + eps))
        out_m.append(mm)
        out_v.append(vv)
    return out_p, out_m, out_v
