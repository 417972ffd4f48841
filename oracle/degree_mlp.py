"""Oracle for the learned per-vector filter degree (TEST INFRASTRUCTURE ONLY).

The paper has no learned component; its Section 3.1 discusses the trade-off between the
block size and the polynomial degree of the filter, which the library's adaptive degree
rule makes per vector.  The learned form predicts, for every active Ritz vector, the log
of the filter degree that would bring its residual below the locking threshold in one
loop, from the vector's residual history, its Ritz-value position and the filter bounds.

This module restates, in plain float64 NumPy with no blocking or fusion, what the library's
CUDA kernels compute for that model: the perceptron's forward pass, the gradient of the
mean squared error by back-propagation layer by layer, and epochs of Adam (Kingma & Ba,
2015) over minibatches in a given sample order.  Only the tests may import it; the library
never does, and it shares no code with the library.

Parameters are one flat vector in the order of the C structure chfsi_mlp: for each layer l
(hidden layers with tanh, then a linear output) the weight matrix W_l row by row (row j
holds the weights of unit j) followed by the bias b_l.  The input is normalised as
(x - mean) * scale before the first layer.  Layer sizes are an argument so that tiny
networks can be checked against finite differences and hand-worked cases; the library's
network has sizes [8, 64, 64, 64, 1].
"""
from __future__ import annotations

import numpy as np

LIBRARY_SIZES = (8, 64, 64, 64, 1)


def param_count(sizes) -> int:
    """Number of trainable parameters of a network with the given layer sizes."""
    return sum(sizes[l + 1] * sizes[l] + sizes[l + 1] for l in range(len(sizes) - 1))


def unpack(params, sizes):
    """Split the flat parameter vector into [(W_l, b_l)] (W_l of shape out x in)."""
    p = np.asarray(params, dtype=np.float64)
    if p.size != param_count(sizes):
        raise ValueError("parameter vector does not match the layer sizes")
    layers, o = [], 0
    for l in range(len(sizes) - 1):
        n_in, n_out = sizes[l], sizes[l + 1]
        W = p[o:o + n_out * n_in].reshape(n_out, n_in)
        o += n_out * n_in
        b = p[o:o + n_out]
        o += n_out
        layers.append((W, b))
    return layers


def pack(layers) -> np.ndarray:
    """Inverse of unpack."""
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def forward(params, sizes, mean, scale, X):
    """Network output y (one value per sample) and the activations of every layer.

    Returns (y [n], acts) where acts[0] is the normalised input and acts[l] the tanh
    activations of hidden layer l."""
    X = np.asarray(X, dtype=np.float64)
    a = (X - np.asarray(mean, np.float64)) * np.asarray(scale, np.float64)
    acts = [a]
    layers = unpack(params, sizes)
    for l, (W, b) in enumerate(layers):
        pre = a @ W.T + b
        if l < len(layers) - 1:
            a = np.tanh(pre)
            acts.append(a)
        else:
            a = pre
    return a[:, 0], acts


def loss_and_gradient(params, sizes, mean, scale, X, z):
    """L = 1/(2n) sum_k (y_k - z_k)^2 and dL/dparams (flat, parameter order) by the chain
    rule applied layer by layer from the output back to the first layer."""
    z = np.asarray(z, dtype=np.float64)
    n = z.size
    y, acts = forward(params, sizes, mean, scale, X)
    layers = unpack(params, sizes)
    loss = 0.5 * float(np.sum((y - z) ** 2)) / n
    delta = ((y - z) / n)[:, None]          # dL/d(pre-activation) of the output layer
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        a_in = acts[l]                       # input of layer l
        grads[l] = (delta.T @ a_in, delta.sum(axis=0))
        if l > 0:
            # back through W_l, then through the tanh of hidden layer l (derivative 1 - a^2)
            delta = (delta @ W) * (1.0 - acts[l] ** 2)
    return loss, pack(grads)


def adam_epoch(params, m1, m2, step, sizes, mean, scale, X, z, order, batch, lr,
               beta1=0.9, beta2=0.999, eps=1e-8):
    """One epoch of Adam: the samples in `order` taken in minibatches of `batch`, each
    minibatch's gradient of its own mean squared error (the loss above over the minibatch)
    followed by the bias-corrected update.  Returns (params, m1, m2, step, mean loss of the
    epoch), the loss being 1/(2n) sum over all samples of the squared errors seen during
    the epoch."""
    p = np.array(params, dtype=np.float64)
    m1 = np.array(m1, dtype=np.float64)
    m2 = np.array(m2, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    order = np.asarray(order)
    n = order.size
    sq = 0.0
    for b0 in range(0, n, batch):
        idx = order[b0:b0 + batch]
        lb, g = loss_and_gradient(p, sizes, mean, scale, X[idx], z[idx])
        sq += 2.0 * lb * idx.size
        step += 1
        m1 = beta1 * m1 + (1.0 - beta1) * g
        m2 = beta2 * m2 + (1.0 - beta2) * g * g
        mhat = m1 / (1.0 - beta1 ** step)
        vhat = m2 / (1.0 - beta2 ** step)
        p = p - lr * mhat / (np.sqrt(vhat) + eps)
    return p, m1, m2, step, 0.5 * sq / n


def normalisation(X):
    """Per-feature mean and scale = 1 / standard deviation (1 where the deviation is below
    1e-12) of the training inputs, as the training sets them before the first epoch."""
    X = np.asarray(X, dtype=np.float64)
    mean = X.mean(axis=0)
    sd = X.std(axis=0)
    scale = np.where(sd > 1e-12, 1.0 / np.where(sd > 1e-12, sd, 1.0), 1.0)
    return mean, scale
