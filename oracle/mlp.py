"""FP64 restatement of the bound proposer's MLP, for checking the GPU
forward and backward kernels (test infrastructure only).

y = relu(relu(x W1 + b1) W2 + b2) W3 + b3, loss = mean over batch x out of
(y - t)^2; parameters packed [W1 (in x h), b1, W2 (h x h), b2, W3 (h x out), b3]
row-major.  The gradient follows the chain rule written out layer by layer.
"""
from __future__ import annotations

import numpy as np


def unpack(p, nin, h, out):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + nin * h].reshape(nin, h); o += nin * h
    b1 = p[o:o + h]; o += h
    W2 = p[o:o + h * h].reshape(h, h); o += h * h
    b2 = p[o:o + h]; o += h
    W3 = p[o:o + h * out].reshape(h, out); o += h * out
    b3 = p[o:o + out]; o += out
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


def forward(p, dims, X):
    W1, b1, W2, b2, W3, b3 = unpack(p, *dims)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(X @ W1 + b1, 0.0)
    h2 = np.maximum(h1 @ W2 + b2, 0.0)
    return h2 @ W3 + b3


def loss(p, dims, X, T):
    return float(np.mean((forward(p, dims, X) - np.asarray(T, dtype=np.float64)) ** 2))


def grad(p, dims, X, T):
    W1, b1, W2, b2, W3, b3 = unpack(p, *dims)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    a1 = X @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ W3 + b3
    dy = 2.0 * (y - T) / y.size
    gW3, gb3 = h2.T @ dy, dy.sum(axis=0)
    dh2 = (dy @ W3.T) * (a2 > 0)
    gW2, gb2 = h1.T @ dh2, dh2.sum(axis=0)
    dh1 = (dh2 @ W2.T) * (a1 > 0)
    gW1, gb1 = X.T @ dh1, dh1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3]), float(np.mean((y - T) ** 2))
