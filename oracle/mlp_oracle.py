"""FP64 oracle of the wake-surrogate multilayer perceptron.

TEST INFRASTRUCTURE ONLY (tests/ may import it; the product never does).
Network: n_in -> width (x n_hidden, GELU) -> n_out, linear output; loss: mean
squared error over every output of the batch.  GELU(z) = z Phi(z) with Phi the
standard normal distribution function; its derivative is Phi(z) + z phi(z).
Parameter vector (same layout as the product): for each layer, W [out][in]
row-major, then b [out].  Backward pass by the chain rule written out layer by
layer.  Pinned by central finite differences of the loss and by the GELU
identities (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

SQRT2 = np.sqrt(2.0)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    Phi = 0.5 * (1.0 + erf(z / SQRT2))
    phi = np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)
    return Phi + z * phi


def layer_dims(n_in, width, n_hidden, n_out):
    dims = []
    for l in range(n_hidden + 1):
        dims.append((n_in if l == 0 else width, n_out if l == n_hidden else width))
    return dims


def n_params(n_in, width, n_hidden, n_out):
    return sum(i * o + o for i, o in layer_dims(n_in, width, n_hidden, n_out))


def unpack(params, dims):
    out, off = [], 0
    p = np.asarray(params, dtype=np.float64)
    for i, o in dims:
        W = p[off:off + i * o].reshape(o, i)
        off += i * o
        b = p[off:off + o]
        off += o
        out.append((W, b))
    return out


def forward(params, X, dims):
    """Returns the output and the per-layer (input, pre-activation) pairs."""
    layers = unpack(params, dims)
    A = np.asarray(X, dtype=np.float64)
    cache = []
    for l, (W, b) in enumerate(layers):
        Z = A @ W.T + b
        cache.append((A, Z))
        A = gelu(Z) if l < len(layers) - 1 else Z
    return A, cache


def loss_grad(params, X, T, dims):
    """Mean squared error and its gradient w.r.t. the parameter vector."""
    Y, cache = forward(params, X, dims)
    T = np.asarray(T, dtype=np.float64)
    n = Y.size
    loss = float(np.sum((Y - T) ** 2) / n)
    dA = 2.0 * (Y - T) / n            # d loss / d output
    layers = unpack(params, dims)
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        A_in, Z = cache[l]
        W, _ = layers[l]
        dZ = dA if l == len(layers) - 1 else dA * gelu_grad(Z)
        grads[l] = (dZ.T @ A_in, dZ.sum(axis=0))
        dA = dZ @ W
    g = np.concatenate([np.concatenate([gW.reshape(-1), gb]) for gW, gb in grads])
    return loss, g
