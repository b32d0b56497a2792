"""Multilayer perceptron of the PAH emission surrogate -- oracle (plain FP64 numpy).

TEST INFRASTRUCTURE ONLY: forward pass, mean-squared-error loss and its exact
gradients by the chain rule, for checking the library's tensor-core kernels. The
parameter layout is the library's: for each layer l, W_l [n_out][n_in] row-major
then b_l [n_out], layers in order.

Network: a_0 = x; z_l = a_{l-1} W_l^T + b_l; a_l = silu(z_l) = z_l / (1 + e^{-z_l})
for the hidden layers; the output layer is linear. Loss = mean over the batch and
the output of (y - t)^2.
"""
from __future__ import annotations

import numpy as np


def layer_shapes(n_in: int, n_hidden: int, n_layers: int, n_out: int):
    dims = [n_in] + [n_hidden] * n_layers + [n_out]
    return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]


def unpack(params, shapes):
    out, o = [], 0
    for (r, c) in shapes:
        W = params[o:o + r * c].reshape(r, c)
        o += r * c
        b = params[o:o + r]
        o += r
        out.append((W, b))
    assert o == params.size
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, shapes, x):
    layers = unpack(np.asarray(params, dtype=np.float64), shapes)
    a = np.asarray(x, dtype=np.float64)
    cache = []
    for i, (W, b) in enumerate(layers):
        z = a @ W.T + b
        cache.append((a, z))
        a = silu(z) if i < len(layers) - 1 else z
    return a, cache


def loss_and_grad(params, shapes, x, t):
    """Loss and its gradient with respect to the flat parameter vector."""
    y, cache = forward(params, shapes, x)
    t = np.asarray(t, dtype=np.float64)
    n = y.size
    loss = float(((y - t) ** 2).sum() / n)
    layers = unpack(np.asarray(params, dtype=np.float64), shapes)
    grads = []
    d = 2.0 * (y - t) / n                       # dL/dz of the output layer
    for i in range(len(layers) - 1, -1, -1):
        a_prev, z = cache[i]
        W, _ = layers[i]
        if i < len(layers) - 1:
            d = d * dsilu(z)                    # through the activation
        grads.append((d.T @ a_prev, d.sum(axis=0)))
        d = d @ W                               # to the previous layer's output
    flat = []
    for gW, gb in reversed(grads):
        flat.append(gW.ravel())
        flat.append(gb)
    return loss, np.concatenate(flat)
